// shard.cu -- the IVF index split by inverted lists over several GPUs.
//
// The inverted lists are the unit of work of the IVF search (Section 3.4):
// a query's result is the K nearest of the candidates of its probed lists.
// Lists are therefore dealt to G shards, balanced by rows (dade_shard_lists);
// a shard (dade_index_subset) keeps everything the search reads besides the
// rows -- the mean and basis (Section 3.2), the eigenvalue sums and the
// sampled rho_d behind eps_d (Eq. 13-14), every centroid -- and the rows of
// its own lists only, so that every shard probes the same global lists and
// scans the probed lists it holds with its own threshold.  A shard's search
// is the IVF loop restricted to its lists; the K nearest of the shards'
// results (dade_merge_shards, one (distance, id) list of K per shard and
// query, as an all-gather delivers them) is the sharded search's result.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "internal.cuh"

namespace dade {

namespace {

// Order-preserving 64-bit key of (distance, id): the float's bits mapped so
// that unsigned comparison follows the float order, then the id (an empty
// place, id -1, gets the largest low word).
__device__ __forceinline__ unsigned long long shard_key(float d, int64_t id) {
    uint32_t u = __float_as_uint(d);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)u << 32) | (uint32_t)(id < 0 ? 0xffffffffu : (uint32_t)id);
}

// Places of the row's K keys that are < x (strict) or <= x (!strict), by
// binary search (the row is ascending).
__device__ __forceinline__ int count_below(const float *d, const int64_t *ids, int k, unsigned long long x, bool strict) {
    int lo = 0, hi = k;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const unsigned long long y = shard_key(d[mid], ids[mid]);
        if (strict ? y < x : y <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One CTA per query: every (shard, place) key finds its rank among all the
// shards' keys (its place in its own row plus, in every other row, the keys
// below it; equal keys rank by shard), and the K lowest ranks are written.
__global__ void k_merge_shards(const int64_t *__restrict__ ids, const float *__restrict__ dists, int g, int64_t nq,
                               int k, int64_t *__restrict__ out_ids, float *__restrict__ out_d) {
    const int64_t q = blockIdx.x;
    for (int e = threadIdx.x; e < g * k; e += blockDim.x) {
        const int a = e / k, i = e % k;
        const int64_t row = ((int64_t)a * nq + q) * k;
        const unsigned long long x = shard_key(dists[row + i], ids[row + i]);
        int rank = i;
        for (int b = 0; b < g; ++b) {
            if (b == a) continue;
            const int64_t rb = ((int64_t)b * nq + q) * k;
            rank += count_below(dists + rb, ids + rb, k, x, b > a);
        }
        if (rank < k) {
            out_ids[q * k + rank] = ids[row + i];
            out_d[q * k + rank] = dists[row + i];
        }
    }
}

bool device_buffer(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
dade_status copy_buf(DevBuf &dst, const DevBuf &src, size_t bytes, cudaStream_t s) {
    DADE_TRY(dst.alloc(std::max<size_t>(bytes, 16)));
    if (bytes) DADE_TRY_CUDA(cudaMemcpyAsync(dst.p, src.p, bytes, cudaMemcpyDeviceToDevice, s));
    return DADE_OK;
}

dade_status make_subset(const dade_index *ix, const int32_t *owner, int32_t shard, dade_index *sub, cudaStream_t s) {
    const int nc = ix->nc, dp = ix->dp;
    sub->n = ix->n;
    sub->d = ix->d;
    sub->dp = dp;
    sub->nb = ix->nb;
    sub->nc = nc;
    sub->mu = ix->mu;
    sub->W = ix->W;
    sub->lam = ix->lam;
    sub->Lam = ix->Lam;
    sub->rho = ix->rho;
    sub->eps_kept = ix->eps_kept;
    sub->assign = ix->assign;
    sub->kmeans_obj = ix->kmeans_obj;
    sub->shard = shard;
    // the kept lists, packed in list order as the build packs them
    sub->lists.assign(nc, ListMeta{0, 0, 0, 0});
    int64_t base = 0, slot = 0;
    int32_t mx = 0;
    for (int c = 0; c < nc; ++c) {
        ListMeta m{base, slot, 0, 0};
        if (owner[c] == shard) {
            m.len = ix->lists[c].len;
            m.np = ix->lists[c].np;
            base += ((int64_t)m.np * dp + 63) / 64 * 64;
            slot += m.np;
            mx = std::max(mx, m.len);
        }
        sub->lists[c] = m;
    }
    sub->max_list = mx;
    sub->data_floats = std::max<int64_t>(base, 64);
    sub->slots = std::max<int64_t>((slot + 3) / 4 * 4, 4);
    DADE_TRY(sub->data.alloc(sizeof(float) * (size_t)sub->data_floats));
    DADE_TRY(sub->ids.alloc(sizeof(int32_t) * (size_t)sub->slots));
    DADE_TRY_CUDA(cudaMemsetAsync(sub->data.p, 0, sizeof(float) * (size_t)sub->data_floats, s));
    DADE_TRY_CUDA(cudaMemsetAsync(sub->ids.p, 0xff, sizeof(int32_t) * (size_t)sub->slots, s));
    const int es = ix->lead_format == DADE_LEAD_BF16 ? 2 : 1, lnb = ix->lead_nb;
    if (ix->lead_format != DADE_LEAD_NONE) {
        sub->lead_format = ix->lead_format;
        sub->lead_dims = ix->lead_dims;
        sub->lead_nb = lnb;
        const size_t code_bytes = (size_t)sub->slots * lnb * 16 * es;
        DADE_TRY(sub->lead.alloc(code_bytes));
        DADE_TRY(sub->lead_err.alloc(sizeof(float) * (size_t)sub->slots * lnb));
        DADE_TRY_CUDA(cudaMemsetAsync(sub->lead.p, 0, code_bytes, s));
        DADE_TRY_CUDA(cudaMemsetAsync(sub->lead_err.p, 0, sizeof(float) * (size_t)sub->slots * lnb, s));
        DADE_TRY(copy_buf<float>(sub->lead_scale, ix->lead_scale, sizeof(float) * (size_t)nc * lnb, s));
    }
    if (ix->tail_nb0 > 0) {
        sub->tail_nb0 = ix->tail_nb0;
        sub->tail_w = ix->tail_w;
        DADE_TRY(sub->tail.alloc(sizeof(float) * (size_t)sub->slots * ix->tail_w));
        DADE_TRY_CUDA(cudaMemsetAsync(sub->tail.p, 0, sizeof(float) * (size_t)sub->slots * ix->tail_w, s));
    }
    for (int c = 0; c < nc; ++c) {
        if (owner[c] != shard || ix->lists[c].np == 0) continue;
        const ListMeta &f = ix->lists[c], &t = sub->lists[c];
        DADE_TRY_CUDA(cudaMemcpyAsync(sub->data.as<float>() + t.base, ix->data.as<float>() + f.base,
                                      sizeof(float) * (size_t)f.np * dp, cudaMemcpyDeviceToDevice, s));
        DADE_TRY_CUDA(cudaMemcpyAsync(sub->ids.as<int32_t>() + t.slot, ix->ids.as<int32_t>() + f.slot,
                                      sizeof(int32_t) * (size_t)f.np, cudaMemcpyDeviceToDevice, s));
        if (ix->lead_format != DADE_LEAD_NONE) {
            const size_t per = (size_t)lnb * 16 * es;   // code bytes per slot
            DADE_TRY_CUDA(cudaMemcpyAsync(sub->lead.as<unsigned char>() + t.slot * per,
                                          ix->lead.as<unsigned char>() + f.slot * per, per * (size_t)f.np,
                                          cudaMemcpyDeviceToDevice, s));
            for (int b = 0; b < lnb; ++b)
                DADE_TRY_CUDA(cudaMemcpyAsync(sub->lead_err.as<float>() + (int64_t)b * sub->slots + t.slot,
                                              ix->lead_err.as<float>() + (int64_t)b * ix->slots + f.slot,
                                              sizeof(float) * (size_t)f.np, cudaMemcpyDeviceToDevice, s));
        }
        if (ix->tail_nb0 > 0)
            DADE_TRY_CUDA(cudaMemcpyAsync(sub->tail.as<float>() + t.slot * ix->tail_w,
                                          ix->tail.as<float>() + f.slot * ix->tail_w,
                                          sizeof(float) * (size_t)f.np * ix->tail_w, cudaMemcpyDeviceToDevice, s));
    }
    DADE_TRY(copy_buf<float>(sub->cent, ix->cent, sizeof(float) * (size_t)nc * dp, s));
    DADE_TRY(copy_buf<float>(sub->cnorm, ix->cnorm, sizeof(float) * (size_t)nc, s));
    DADE_TRY(upload_basis(sub, s));
    DADE_TRY(prepare_tensor_operands(sub, s));
    DADE_TRY(make_data_tmap(sub));
    DADE_TRY(sub->meta.alloc(sizeof(ListMeta) * (size_t)nc));
    DADE_TRY_CUDA(cudaMemcpyAsync(sub->meta.p, sub->lists.data(), sizeof(ListMeta) * (size_t)nc,
                                  cudaMemcpyHostToDevice, s));
    DADE_TRY(sub->errflag.alloc(sizeof(int32_t) * 4));
    DADE_TRY_CUDA(cudaMemsetAsync(sub->errflag.p, 0, sizeof(int32_t) * 4, s));
    DADE_TRY_CUDA(cudaStreamSynchronize(s));
    return DADE_OK;
}

} // namespace

} // namespace dade

using namespace dade;

extern "C" {

dade_status dade_shard_lists(const int64_t *list_rows, int32_t n_lists, int32_t n_shards, int32_t *owner) {
    set_error(std::string());
    DADE_CHECK_ARG(list_rows != nullptr && owner != nullptr, "NULL pointer");
    DADE_CHECK_ARG(n_lists >= 1 && n_shards >= 1, "n_lists and n_shards must be >= 1");
    for (int32_t c = 0; c < n_lists; ++c) DADE_CHECK_ARG(list_rows[c] >= 0, "negative list size");
    // longest lists first (ties by list id), each to the shard with the fewest rows so
    // far (ties by shard id)
    std::vector<int32_t> order(n_lists);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return list_rows[a] > list_rows[b]; });
    std::vector<int64_t> load(n_shards, 0);
    for (int32_t c : order) {
        const int32_t g = (int32_t)(std::min_element(load.begin(), load.end()) - load.begin());
        owner[c] = g;
        load[g] += list_rows[c];
    }
    return DADE_OK;
}

dade_status dade_index_subset(const dade_index *ix, const int32_t *owner, int32_t shard, dade_index **out) {
    set_error(std::string());
    DADE_CHECK_ARG(ix != nullptr && owner != nullptr && out != nullptr, "NULL pointer");
    DADE_CHECK_ARG(ix->shard < 0, "the index is already a shard");
    DADE_CHECK_ARG(shard >= 0, "shard < 0");
    *out = nullptr;
    dade_index *sub = new (std::nothrow) dade_index();
    if (!sub) {
        set_error("host allocation of the shard failed");
        return DADE_ENOMEM;
    }
    dade_status st;
    try {
        st = make_subset(ix, owner, shard, sub, 0);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed while making the shard");
        st = DADE_ENOMEM;
    }
    if (st != DADE_OK) {
        delete sub;
        return st;
    }
    *out = sub;
    return DADE_OK;
}

dade_status dade_merge_shards(const int64_t *ids, const float *dists, int32_t n_shards, int64_t nq, int32_t k,
                              int64_t *out_ids, float *out_dists, dade_stream stream) {
    set_error(std::string());
    DADE_CHECK_ARG(n_shards >= 1 && nq >= 0 && k >= 1 && k <= DADE_MAX_K, "n_shards, nq or k out of range");
    if (nq == 0) return DADE_OK;
    DADE_CHECK_ARG(ids && dists && out_ids && out_dists, "NULL pointer");
    DADE_CHECK_ARG(device_buffer(ids) && device_buffer(dists) && device_buffer(out_ids) && device_buffer(out_dists),
                   "dade_merge_shards takes device buffers");
    DADE_CHECK_ARG(nq <= 0x7fffffffLL, "nq above 2^31 - 1");
    k_merge_shards<<<(unsigned)nq, 128, 0, (cudaStream_t)stream>>>(ids, dists, n_shards, nq, k, out_ids, out_dists);
    return launch_check("k_merge_shards");
}

} // extern "C"
