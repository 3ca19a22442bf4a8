// order.cu -- the order in which a scan runs its queries.
//
// A scan runs one CTA per query and every CTA touches only its own query's
// state, so results do not depend on the order in which the CTAs run.  The
// order does decide how the concurrently running queries share L2: queries
// whose nearest list is the same have largely the same probe sets, and run
// side by side they read the same list rows while those are still cached.
// This file sorts the queries by their first probed list (counting sort:
// histogram, exclusive scan, scatter); the scan kernels read their query
// index from the resulting permutation.
#include <algorithm>

#include "internal.cuh"

namespace dade {

namespace {

__global__ void k_order_hist(const int32_t *__restrict__ probe, int64_t nq, int nprobe, int *__restrict__ cnt) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[probe[q * nprobe]], 1);
}

// Exclusive prefix sum of cnt[0..n) in place, one CTA of 1024 threads: each
// thread sums a contiguous run, a shared-memory scan of the run totals gives
// each run its offset, and the runs are rewritten.
__global__ void __launch_bounds__(1024) k_order_scan(int *__restrict__ cnt, int n) {
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int b = min(n, t * per), e = min(n, b + per);
    int s = 0;
    for (int i = b; i < e; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = b; i < e; ++i) {
        const int c = cnt[i];
        cnt[i] = run;
        run += c;
    }
}

__global__ void k_order_scatter(const int32_t *__restrict__ probe, int64_t nq, int nprobe, int *__restrict__ off,
                                int32_t *__restrict__ order) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x)
        order[atomicAdd(&off[probe[q * nprobe]], 1)] = (int32_t)q;
}

} // namespace

// Exclusive prefix sum of a[0..n) in place (n small: one CTA).
dade_status exclusive_scan_int(int *a, int n, cudaStream_t s) {
    if (n <= 0) return DADE_OK;
    k_order_scan<<<1, 1024, 0, s>>>(a, n);
    return launch_check("k_order_scan");
}

dade_status order_queries(const dade_index *ix, const int32_t *probe, int64_t nq, int32_t nprobe, int32_t *order,
                          cudaStream_t s) {
    if (nq == 0) return DADE_OK;
    DADE_TRY(ws(ix).ordcnt.ensure(sizeof(int) * (size_t)ix->nc));
    int *cnt = ws(ix).ordcnt.as<int>();
    DADE_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)ix->nc, s));
    const unsigned g = (unsigned)std::min<int64_t>((nq + 255) / 256, 152 * 8);
    k_order_hist<<<g, 256, 0, s>>>(probe, nq, nprobe, cnt);
    DADE_TRY(launch_check("k_order_hist"));
    k_order_scan<<<1, 1024, 0, s>>>(cnt, ix->nc);
    DADE_TRY(launch_check("k_order_scan"));
    k_order_scatter<<<g, 256, 0, s>>>(probe, nq, nprobe, cnt, order);
    return launch_check("k_order_scatter");
}

} // namespace dade
