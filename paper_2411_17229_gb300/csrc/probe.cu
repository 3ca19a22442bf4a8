// probe.cu -- IVF coarse probe (Section 3.4): the nprobe inverted lists whose
// centroids are nearest to each rotated query, ordered by (distance, list id).
//
// Step 1 writes the query x centroid squared-distance matrix
// ||q||^2 + ||c||^2 - 2 <q, c> with the tensor-core GEMM of tc_gemm.cu
// (3xTF32, FP32-accurate).
// Step 2 selects, per query, the nprobe smallest 64-bit keys
// (float bits of the distance << 32 | list id): a value-histogram threshold
// and a rank sort of the keys below it (k_probe_hist), and, for the rows where
// ties overflow that pass, an 8-pass radix select over 8-bit digits (keys are
// unique, so exactly nprobe keys are <= the selected one).  Both give the
// same, deterministic order.
#include <mutex>
#include <string>

#include "internal.cuh"
#include "tiles.cuh"

namespace dade {

namespace {

__global__ void k_row_sqnorm(const float *__restrict__ X, int n, int ld, int kdim, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    float s = 0.f;
    for (int k = lane; k < kdim; k += 32) s = fmaf(X[(int64_t)w * ld + k], X[(int64_t)w * ld + k], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[w] = s;
}

constexpr int SEL_THREADS = 256;

__device__ __forceinline__ unsigned long long probe_key(const float *row, int j) {
    return ((unsigned long long)__float_as_uint(row[j]) << 32) | (unsigned)j;
}

__global__ void __launch_bounds__(SEL_THREADS) k_probe_select(const float *__restrict__ dist, int nc, int nprobe,
                                                              int32_t *__restrict__ out, const int *__restrict__ only) {
    if (only && !only[blockIdx.x]) return;   // row already selected by k_probe_hist
    extern __shared__ unsigned long long sel[];        // [nprobe]
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned s_rank, s_cnt;
    const int tid = threadIdx.x, lane = tid & 31;
    const float *row = dist + (int64_t)blockIdx.x * nc;
    unsigned long long prefix = 0, mask = 0;
    unsigned rank = (unsigned)nprobe;                  // 1-based rank sought among keys matching prefix
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        hist[tid] = 0;
        __syncthreads();
        // Distances of one query share their leading bytes, so most keys of a
        // pass fall into a few bins: lanes with equal bins add once per warp.
        for (int j0 = 0; j0 < nc; j0 += SEL_THREADS) {
            const int j = j0 + tid;
            const unsigned long long k = j < nc ? probe_key(row, j) : 0ull;
            const bool in = j < nc && (k & mask) == prefix;
            const unsigned bin = in ? (unsigned)((k >> shift) & 255u) : 256u;
            const unsigned peers = __match_any_sync(0xffffffffu, bin);
            if (in && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
        }
        __syncthreads();
        if (tid < 32) {   // warp 0: find the digit where the cumulative count reaches rank
            unsigned loc[8], s = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) { loc[t] = hist[lane * 8 + t]; s += loc[t]; }
            unsigned inc = s;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                unsigned v = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc += v;
            }
            unsigned before = inc - s;
            bool here = before < rank && inc >= rank;
            if (here) {
                unsigned c = before;
                int t = 0;
                while (c + loc[t] < rank) { c += loc[t]; ++t; }
                s_prefix = prefix | ((unsigned long long)(lane * 8 + t) << shift);
                s_rank = rank - c;
            }
        }
        __syncthreads();
        prefix = s_prefix;
        rank = s_rank;
        mask |= 255ull << shift;
        const unsigned here_cnt = hist[(prefix >> shift) & 255u];
        __syncthreads();
        // After the four distance bytes: if every key with the selected
        // distance is needed (no tie to break by id), select all keys whose
        // distance is at most it.
        if (pass == 3 && here_cnt == rank) {
            prefix |= 0xffffffffull;
            break;
        }
    }
    // prefix is now the nprobe-th smallest key; gather the keys <= it
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    for (int j = tid; j < nc; j += SEL_THREADS) {
        unsigned long long k = probe_key(row, j);
        if (k <= prefix) {
            const unsigned slot = atomicAdd(&s_cnt, 1u);
            if (slot < (unsigned)nprobe) sel[slot] = k;   // exactly nprobe keys qualify (keys are unique)
        }
    }
    __syncthreads();
    const int nsel = min((int)s_cnt, nprobe);
    for (int t = tid; t < nsel; t += SEL_THREADS) {
        unsigned long long k = sel[t];
        int r = 0;
        for (int u = 0; u < nsel; ++u) r += sel[u] < k;
        out[(int64_t)blockIdx.x * nprobe + r] = (int32_t)(k & 0xffffffffu);
    }
}

// Selection by value histogram: the row's distances are binned uniformly
// between their minimum and maximum (a monotone map, so every distance below
// the nprobe-th smallest falls in a bin at or below that one's), the bin
// where the cumulative count reaches nprobe gives a threshold, and the keys at
// or below it (typically nprobe plus part of one bin) are collected and
// rank-sorted by (distance, id).  Three passes over the row, few barriers.  A
// row whose threshold bin holds more than HCAP keys (massive ties) sets
// *overflow for the radix path.
constexpr int HBINS = 1024, HCAP = 1024;

__global__ void __launch_bounds__(SEL_THREADS) k_probe_hist(const float *__restrict__ dist, int nc, int nprobe,
                                                            int32_t *__restrict__ out, int *__restrict__ overflow) {
    if (threadIdx.x == 0) overflow[blockIdx.x] = 0;
    __shared__ unsigned hist[HBINS];
    __shared__ unsigned long long cand[HCAP];
    __shared__ float s_min[SEL_THREADS / 32], s_max[SEL_THREADS / 32];
    __shared__ int s_bin, s_cnt;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float *row = dist + (int64_t)blockIdx.x * nc;
    float lo = INFINITY, hi = -INFINITY;
    for (int j = tid; j < nc; j += SEL_THREADS) {
        const float v = row[j];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    for (int off = 16; off > 0; off >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (lane == 0) { s_min[warp] = lo; s_max[warp] = hi; }
    for (int b = tid; b < HBINS; b += SEL_THREADS) hist[b] = 0;
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    lo = s_min[0];
    hi = s_max[0];
    for (int w = 1; w < SEL_THREADS / 32; ++w) { lo = fminf(lo, s_min[w]); hi = fmaxf(hi, s_max[w]); }
    const float scale = hi > lo ? (float)(HBINS - 1) / (hi - lo) : 0.f;
    auto bin_of = [&](float v) { return min(HBINS - 1, (int)((v - lo) * scale)); };
    for (int j = tid; j < nc; j += SEL_THREADS) atomicAdd(&hist[bin_of(row[j])], 1u);
    __syncthreads();
    if (warp == 0) {   // the bin where the cumulative count reaches nprobe
        const int per = HBINS / 32;
        unsigned loc = 0;
        for (int t = 0; t < per; ++t) loc += hist[lane * per + t];
        unsigned inc = loc;
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += v;
        }
        const unsigned before = inc - loc;
        if (before < (unsigned)nprobe && inc >= (unsigned)nprobe) {
            unsigned c = before;
            int t = 0;
            while (c + hist[lane * per + t] < (unsigned)nprobe) { c += hist[lane * per + t]; ++t; }
            s_bin = lane * per + t;
        }
    }
    __syncthreads();
    const int bstar = s_bin;
    for (int j = tid; j < nc; j += SEL_THREADS) {
        const float v = row[j];
        if (bin_of(v) <= bstar) {
            const int slot = atomicAdd(&s_cnt, 1);
            if (slot < HCAP) cand[slot] = ((unsigned long long)__float_as_uint(v) << 32) | (unsigned)j;
        }
    }
    __syncthreads();
    const int n = s_cnt;
    if (n > HCAP) {
        if (tid == 0) overflow[blockIdx.x] = 1;
        return;
    }
    for (int t = tid; t < n; t += SEL_THREADS) {
        const unsigned long long k = cand[t];
        int r = 0;
        for (int u = 0; u < n; ++u) r += cand[u] < k;
        if (r < nprobe) out[(int64_t)blockIdx.x * nprobe + r] = (int32_t)(k & 0xffffffffu);
    }
}

} // namespace

dade_status centroid_norms(dade_index *ix, cudaStream_t s) {
    DADE_TRY(ix->cnorm.alloc(sizeof(float) * (size_t)ix->nc));
    k_row_sqnorm<<<(unsigned)((ix->nc * 32 + 255) / 256), 256, 0, s>>>(ix->cent.as<float>(), ix->nc, ix->dp, ix->d,
                                                                      ix->cnorm.as<float>());
    return launch_check("k_row_sqnorm");
}

dade_status probe(const dade_index *ix, const float *q_rot, int64_t nq, int32_t q_stride, int32_t nprobe,
                  int32_t *probe_out, cudaStream_t s) {
    if (nq == 0) return DADE_OK;
    DADE_TRY(ws(ix).dist.ensure(sizeof(float) * (size_t)nq * ix->nc));
    DADE_TRY(probe_distances(ix, q_rot, nq, q_stride, ws(ix).dist.as<float>(), s));
    int *flags = nullptr;
    if (nprobe <= HCAP) {
        DADE_TRY(ws(ix).selflag.ensure(sizeof(int) * (size_t)nq));
        flags = ws(ix).selflag.as<int>();
        k_probe_hist<<<(unsigned)nq, SEL_THREADS, 0, s>>>(ws(ix).dist.as<float>(), ix->nc, nprobe, probe_out, flags);
        DADE_TRY(launch_check("k_probe_hist"));
    }
    // radix select for the rows the histogram pass could not settle (or all rows)
    size_t smem = sizeof(unsigned long long) * (size_t)nprobe;
    if (smem > 48 * 1024)
        DADE_TRY_CUDA(cudaFuncSetAttribute(k_probe_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_probe_select<<<(unsigned)nq, SEL_THREADS, smem, s>>>(ws(ix).dist.as<float>(), ix->nc, nprobe, probe_out, flags);
    return launch_check("k_probe_select");
}

// ------------------------------------------------------------------------------
// Probe without device allocations.
//
// dade_probe() keeps its query x centroid distance matrix in the index's
// workspace, which grows with cudaMalloc on demand.  Some callers must not
// allocate device memory at all: a serving path that must not block on or
// fail in the allocator in the middle of a request, or a process whose device
// memory is owned by another framework's arena.  dade_probe_noalloc() keeps
// the distance matrix in the fixed array below instead, computes it with a
// GEMM kernel that stages its operands itself (no operand images), with the
// same products and the same query norms as dade_probe's kernels (the same
// bits), and selects the nearest lists with the same exact radix select.
//
// The array is a file-scope device variable: every GPU that loads this
// library reserves DADE_PROBE_NOALLOC_MAX floats (16 MiB) for it until the
// process exits.  Host code cannot pass the variable's name to a kernel (in
// host code it is only a stand-in for the symbol), so the first call on each
// device looks up the array's device address with cudaGetSymbolAddress, with
// that device current, and caches it.  All calls share the one array: calls
// whose work overlaps on the GPU (different streams, no ordering between
// them) race on it.  Every entry that a call reads was written by the same
// call first, so nothing needs clearing between calls.
static __device__ __align__(256) float g_probe_scratch[DADE_PROBE_NOALLOC_MAX];

namespace {
constexpr int kMaxDevices = 64;
float *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

dade_status scratch_address(float **out) {
    int dev = 0;
    DADE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("dade_probe_noalloc: device ordinal beyond the supported range");
        return DADE_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_probe_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error(std::string("dade_probe_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return DADE_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[dev];
    return DADE_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}
} // namespace

} // namespace dade

extern "C" dade_status dade_probe_noalloc(const dade_index *ix, const float *q_rot, int64_t nq, int32_t nprobe,
                                          int32_t *probe, dade_stream stream) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(ix != nullptr, "index is NULL");
    DADE_CHECK_ARG(nq >= 0, "nq < 0");
    DADE_CHECK_ARG(nprobe >= 1 && nprobe <= ix->nc && nprobe <= 8192, "nprobe outside 1..min(n_clusters, 8192)");
    if (nq == 0) return DADE_OK;
    DADE_CHECK_ARG(q_rot != nullptr && probe != nullptr, "NULL pointer");
    if (nq * (int64_t)ix->nc > (int64_t)DADE_PROBE_NOALLOC_MAX) {
        set_error("invalid argument: dade_probe_noalloc handles at most DADE_PROBE_NOALLOC_MAX (4194304) "
                  "query x list distances per call (nq * n_clusters = " + std::to_string(nq * (int64_t)ix->nc) +
                  "); split the batch");
        return DADE_EINVAL;
    }
    DADE_CHECK_ARG(on_device(q_rot) && on_device(probe),
                   "dade_probe_noalloc takes device pointers only (host buffers would need staging memory)");
    float *dist = nullptr;
    DADE_TRY(scratch_address(&dist));
    cudaStream_t s = (cudaStream_t)stream;
    DADE_TRY(probe_distances_direct(ix, q_rot, nq, ix->d, dist, s));
    size_t smem = sizeof(unsigned long long) * (size_t)nprobe;
    if (smem > 48 * 1024)
        DADE_TRY_CUDA(cudaFuncSetAttribute(k_probe_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_probe_select<<<(unsigned)nq, SEL_THREADS, smem, s>>>(dist, ix->nc, nprobe, probe, nullptr);
    return launch_check("k_probe_select");
}
