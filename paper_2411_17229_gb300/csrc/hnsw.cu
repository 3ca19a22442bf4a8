// hnsw.cu -- HNSW* (Section 3.4): greedy beam search on a layer-0 graph with
// one DADE DCO (Algorithm 1, the test of Section 3.3) per neighbour, and the
// construction of that graph.
//
// Search: one warp per query (four per thread block, persistent over the
// batch).  The result set R (at most ef objects, ascending by (squared
// distance, id)) lives in the warp's shared memory with an "expanded" bit per
// entry; the search set S of the method is represented by R's unexpanded
// entries.  Under the (distance, id) order this pops the same objects: an
// object that left R is farther than every object R holds, so whenever it
// would be the nearest of S, R has no unexpanded object left and the method's
// stop compare ends the search at that pop.  Each step takes the nearest
// unexpanded entry c, reads r = the farthest distance in R (+inf while R holds
// fewer than ef: the threshold is read once per expanded object, the schedule
// the oracle calls NODE), and gives each of c's M0 <= 32 neighbour slots to a
// lane: the lane claims the neighbour in the query's visited set and runs the
// DCO on it; the accepted neighbours then enter R (the ef nearest are kept).
//
// DCO arithmetic: each lane reads its candidate's row (row-major, rows of dp
// floats, 16-byte loads) and sums (q_k - o_k)^2 in dimension order with every
// subtraction, product and sum rounded to FP32 (no contraction), the
// arithmetic of the paper's scalar implementation; at each tested d < D it
// prunes iff P_d > c_j r^2 (the product rounded to FP32), at d = D it accepts
// iff P_D <= r^2.  Dims D..dp-1 of every row and query are zero, so running
// the last increment to dp adds exact zeros.
//
// Visited set: per warp slot, an open-addressing table in global memory of
// 64-bit words (query tag << 32 | object id).  A word whose tag is not the
// current query's counts as empty, so nothing is cleared between queries; the
// host advances the tags per call and zeroes the tables when they would wrap.
// The table holds at least twice the objects a query can visit (the visit
// budget, one expansion past it, the entry objects), so probing always ends.
//
// Graph (dade_hnsw_build): candidates from the index's own FDScanning search
// (the kc nearest of every object among its nprobe nearest lists; exact when
// nprobe = n_clusters), HNSW's neighbour heuristic (Malkov and Yashunin,
// Algorithm 4) keeping at most M on the GPU, reverse links and the degree cap
// M0 (the heuristic again over lists longer than M0) -- the graph the oracle
// defines, from approximate candidates when nprobe < n_clusters.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int HW = 4;                // warps per thread block of the search kernel
constexpr int HMAX_EF = 1024;
constexpr int HMAX_ENTRY = 64;
constexpr unsigned FULL = 0xffffffffu;

bool dev_ptr(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Shared bytes of one warp: the query (dp floats), R's distances and ids (ef
// each) and expanded bits (ef bytes).
__host__ __device__ inline size_t warp_bytes(int dp, int ef) { return align16((size_t)dp * 4) + 2 * align16((size_t)ef * 4) + align16(ef); }

struct HnswArgs {
    const float *X;             // [n][dp] rotated objects, dims >= d zero
    const int32_t *nbr;         // [n][m0] neighbour ids, -1 unused
    int64_t n;
    int32_t d, dp, m0;
    const float *q;             // [nq][d] rotated queries
    int64_t nq;
    int32_t k, ef, delta_d;
    const float *coef;          // [tested increments] c_j, or nullptr (FDScanning)
    const int64_t *entry;       // [nq][n_entry] entry ids, or nullptr (entry0 for every query)
    int32_t n_entry;
    int64_t entry0;
    int64_t max_visits;         // DCOs after which no further object is expanded
    unsigned long long *hash;   // per warp slot: 1 << hbits words
    int32_t hbits;
    unsigned tag0;              // query qi uses tag tag0 + qi + 1
    int64_t *ids;               // [nq][k]
    float *dists;               // [nq][k]
    int64_t *stats;             // [nq][5] or nullptr
};

// Claims object id for the current query in the warp slot's table: true the
// first time, false when it was visited (or, impossibly, the table is full).
__device__ bool visit_once(unsigned long long *t, unsigned hmask, unsigned tag, int id) {
    const unsigned long long want = ((unsigned long long)tag << 32) | (unsigned)id;
    const unsigned h = (unsigned)id * 2654435761u;   // Knuth's multiplicative hash
    for (unsigned probe = 0; probe <= hmask; ++probe) {
        unsigned long long *w = t + ((h + probe) & hmask);
        unsigned long long cur = __ldcg(w);
        for (int tries = 0; tries < 4; ++tries) {
            if ((unsigned)(cur >> 32) != tag) {          // empty for this query
                const unsigned long long prev = atomicCAS(w, cur, want);
                if (prev == cur) return true;
                cur = prev;                              // another lane of this warp took it: look again
                continue;
            }
            if ((unsigned)cur == (unsigned)id) return false;
            break;                                       // another object of this query: next word
        }
    }
    return false;
}

// One DCO of object e against the squared threshold r2 (see the file comment).
// Returns accept; *dist = P_D when the last increment ran; *dims = dims used.
__device__ bool hnsw_dco(const HnswArgs &a, const float *sq, int64_t e, float r2, float *dist, int *dims) {
    const float4 *x = reinterpret_cast<const float4 *>(a.X + e * a.dp);
    const float4 *qv = reinterpret_cast<const float4 *>(sq);
    float P = 0.f;
    int d = 0, j = 0;
    for (;;) {
        const int dn = min(d + a.delta_d, a.dp);
        for (int k4 = d >> 2; k4 < (dn >> 2); ++k4) {
            const float4 o = __ldg(x + k4);
            const float4 q = qv[k4];
            float t;
            t = __fsub_rn(q.x, o.x);
            P = __fadd_rn(P, __fmul_rn(t, t));
            t = __fsub_rn(q.y, o.y);
            P = __fadd_rn(P, __fmul_rn(t, t));
            t = __fsub_rn(q.z, o.z);
            P = __fadd_rn(P, __fmul_rn(t, t));
            t = __fsub_rn(q.w, o.w);
            P = __fadd_rn(P, __fmul_rn(t, t));
        }
        d = dn;
        if (d >= a.d) break;
        if (a.coef && P > __fmul_rn(a.coef[j], r2)) {
            *dims = d;
            return false;
        }
        ++j;
    }
    *dims = a.d;
    *dist = P;
    return P <= r2;
}

// R (nR entries, ascending by (distance, id)) takes (xd, xi) if it is among
// the ef nearest; the farthest entry drops out when R is full.  Warp-wide.
__device__ void r_insert(float *rd, int *ri, unsigned char *rx, int &nR, int ef, float xd, int xi, int lane) {
    int pos = 0;
    for (int j0 = 0; j0 < nR; j0 += 32) {
        const int j = j0 + lane;
        const bool lt = j < nR && (rd[j] < xd || (rd[j] == xd && ri[j] < xi));
        pos += __popc(__ballot_sync(FULL, lt));
    }
    if (pos >= ef) return;                              // R full and x beyond its farthest
    const int last = min(nR, ef - 1);                   // entries [pos, last) move up by one
    for (int top = last; top > pos; top -= 32) {
        const int j = top - 1 - lane;
        const bool act = j >= pos;
        float vd = 0.f;
        int vi = 0;
        unsigned char vx = 0;
        if (act) {
            vd = rd[j];
            vi = ri[j];
            vx = rx[j];
        }
        __syncwarp();
        if (act) {
            rd[j + 1] = vd;
            ri[j + 1] = vi;
            rx[j + 1] = vx;
        }
        __syncwarp();
    }
    if (lane == 0) {
        rd[pos] = xd;
        ri[pos] = xi;
        rx[pos] = 0;
    }
    nR = min(nR + 1, ef);
    __syncwarp();
}

// The accepted lanes (ballot acc) enter R, in lane order.
__device__ void admit(unsigned acc, float p, int e, float *rd, int *ri, unsigned char *rx, int &nR, int ef,
                      int lane) {
    while (acc) {
        const int b = __ffs(acc) - 1;
        acc &= acc - 1;
        const float xd = __shfl_sync(FULL, p, b);
        const int xi = __shfl_sync(FULL, e, b);
        r_insert(rd, ri, rx, nR, ef, xd, xi, lane);
    }
}

__global__ void __launch_bounds__(HW * 32) k_hnsw_search(HnswArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char *base = smem + (size_t)w * warp_bytes(a.dp, a.ef);
    float *sq = reinterpret_cast<float *>(base);
    float *rd = reinterpret_cast<float *>(base + align16((size_t)a.dp * 4));
    int *ri = reinterpret_cast<int *>(base + align16((size_t)a.dp * 4) + align16((size_t)a.ef * 4));
    unsigned char *rx = base + align16((size_t)a.dp * 4) + 2 * align16((size_t)a.ef * 4);
    const int64_t gw = (int64_t)blockIdx.x * HW + w, nw = (int64_t)gridDim.x * HW;
    unsigned long long *tab = a.hash + ((size_t)gw << a.hbits);
    const unsigned hmask = (1u << a.hbits) - 1u;
    const float INF = __int_as_float(0x7f800000);

    for (int64_t qi = gw; qi < a.nq; qi += nw) {
        const unsigned tag = a.tag0 + (unsigned)qi + 1u;
        for (int k = lane; k < a.dp; k += 32) sq[k] = k < a.d ? a.q[qi * a.d + k] : 0.f;
        __syncwarp();
        int nR = 0;
        long long vis = 0, dims_sum = 0, n_acc = 0, n_pruned = 0, pops = 0;

        // the entry objects: one group against r = +inf
        const int ne = a.entry ? a.n_entry : 1;
        for (int j0 = 0; j0 < ne; j0 += 32) {
            int64_t e = -1;
            if (j0 + lane < ne) e = a.entry ? a.entry[qi * a.n_entry + j0 + lane] : a.entry0;
            const bool fresh = e >= 0 && e < a.n && visit_once(tab, hmask, tag, (int)e);
            float p = INF;
            int dims = 0;
            const bool ok = fresh && hnsw_dco(a, sq, e, INF, &p, &dims);
            vis += __popc(__ballot_sync(FULL, fresh));
            dims_sum += __reduce_add_sync(FULL, (unsigned)dims);
            n_acc += __popc(__ballot_sync(FULL, ok));
            admit(__ballot_sync(FULL, ok), p, (int)e, rd, ri, rx, nR, a.ef, lane);
        }

        for (;;) {
            if (vis >= a.max_visits) break;
            int cpos = -1;                               // the nearest unexpanded entry of R
            for (int j0 = 0; j0 < nR && cpos < 0; j0 += 32) {
                const unsigned b = __ballot_sync(FULL, j0 + lane < nR && rx[j0 + lane] == 0);
                if (b) cpos = j0 + __ffs(b) - 1;
            }
            if (cpos < 0) break;
            const int c = ri[cpos];
            const float r2 = nR == a.ef ? rd[a.ef - 1] : INF;
            __syncwarp();
            if (lane == 0) rx[cpos] = 1;
            __syncwarp();
            ++pops;
            int64_t e = -1;
            bool fresh = false;
            if (lane < a.m0) {
                e = a.nbr[(int64_t)c * a.m0 + lane];
                fresh = e >= 0 && e < a.n && visit_once(tab, hmask, tag, (int)e);
            }
            float p = INF;
            int dims = 0;
            const bool ok = fresh && hnsw_dco(a, sq, e, r2, &p, &dims);
            vis += __popc(__ballot_sync(FULL, fresh));
            dims_sum += __reduce_add_sync(FULL, (unsigned)dims);
            n_acc += __popc(__ballot_sync(FULL, ok));
            n_pruned += __popc(__ballot_sync(FULL, fresh && !ok && dims < a.d));
            admit(__ballot_sync(FULL, ok), p, (int)e, rd, ri, rx, nR, a.ef, lane);
        }

        for (int s = lane; s < a.k; s += 32) {
            a.ids[qi * a.k + s] = s < nR ? (int64_t)ri[s] : -1;
            a.dists[qi * a.k + s] = s < nR ? rd[s] : INF;
        }
        if (a.stats && lane == 0) {
            int64_t *st = a.stats + qi * 5;
            st[0] = vis;
            st[1] = dims_sum;
            st[2] = n_acc;
            st[3] = n_pruned;
            st[4] = pops;
        }
        __syncwarp();
    }
}

}  // namespace

// ------------------------------------------------------------ graph build ----
namespace {

// Squared norms of the rows (the entry object is the one nearest the mean,
// which the rotation moves to the origin).
__global__ void k_hnsw_norms(const float *X, int64_t n, int dp, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 *x = reinterpret_cast<const float4 *>(X + i * dp);
        float s = 0.f;
        for (int k = 0; k < dp / 4; ++k) {
            const float4 v = __ldg(x + k);
            s = fmaf(v.x, v.x, s);
            s = fmaf(v.y, v.y, s);
            s = fmaf(v.z, v.z, s);
            s = fmaf(v.w, v.w, s);
        }
        out[i] = s;
    }
}

// Candidates of rows [row0, row0 + rows): the search results (kq per row,
// ascending by (distance, id)) without the row's own id, the first kc kept.
__global__ void k_hnsw_cand(const int64_t *kid, const float *kd, int64_t n, int kq, int kc, int64_t row0,
                            int64_t rows, int32_t *cid, float *cdist, int32_t *ccnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = row0 + i;
        int m = 0;
        for (int j = 0; j < kq && m < kc; ++j) {
            const int64_t v = kid[i * kq + j];
            if (v < 0 || v >= n || v == u) continue;
            cid[u * kc + m] = (int32_t)v;
            cdist[u * kc + m] = kd[i * kq + j];
            ++m;
        }
        ccnt[u] = m;
        for (int j = m; j < kc; ++j) {
            cid[u * kc + j] = -1;
            cdist[u * kc + j] = 0.f;
        }
    }
}

// HNSW's neighbour heuristic, one warp per list: list li holds cnt[li]
// candidates at off[li] (off == nullptr: at li * stride), ascending by
// (distance to the list's object, id); candidate e is kept iff it is nearer to
// that object than to every candidate kept before it, until cap (<= 32) are
// kept.  Lane s holds the s-th kept candidate and tests e against it.
__global__ void k_hnsw_select(const float *X, int dp, const int64_t *off, int stride, const int32_t *cnt,
                              const int32_t *cid, const float *cdist, int64_t nl, int cap, int32_t *out,
                              float *out_d, int out_stride, int32_t *out_cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t li = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); li < nl; li += (int64_t)gridDim.x * wpb) {
        const int64_t o = off ? off[li] : li * stride;
        const int m = cnt[li];
        int kept = 0, mine = -1;
        float mine_d = 0.f;
        for (int i = 0; i < m && kept < cap; ++i) {
            const int e = cid[o + i];
            const float de = cdist[o + i];
            bool blocks = false;
            if (lane < kept) {
                const float4 *xe = reinterpret_cast<const float4 *>(X + (int64_t)e * dp);
                const float4 *xs = reinterpret_cast<const float4 *>(X + (int64_t)mine * dp);
                float s = 0.f;
                for (int k = 0; k < dp / 4; ++k) {
                    const float4 a = __ldg(xe + k), b = __ldg(xs + k);
                    float t = a.x - b.x;
                    s = fmaf(t, t, s);
                    t = a.y - b.y;
                    s = fmaf(t, t, s);
                    t = a.z - b.z;
                    s = fmaf(t, t, s);
                    t = a.w - b.w;
                    s = fmaf(t, t, s);
                }
                blocks = !(de < s);
            }
            if (__ballot_sync(FULL, blocks) == 0) {
                if (lane == kept) {
                    mine = e;
                    mine_d = de;
                }
                ++kept;
            }
        }
        if (lane < out_stride) {
            out[li * out_stride + lane] = lane < kept ? mine : -1;
            if (out_d) out_d[li * out_stride + lane] = lane < kept ? mine_d : 0.f;
        }
        if (lane == 0 && out_cnt) out_cnt[li] = kept;
    }
}

// Blocks of a grid-stride kernel over `items` (per_block per block), at most
// 32 per SM of the 152.
int grid_for(int64_t items, int per_block) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((items + per_block - 1) / per_block, 152 * 32));
}

}  // namespace

struct dade_hnsw {
    const dade_index *ix = nullptr;   // thresholds and query rotation (may be null for a given graph)
    int64_t n = 0, entry = 0;
    int32_t d = 0, dp = 0, m0 = 0;
    dade::DevBuf X, nbr;
    // per-call scratch (one call at a time per structure)
    dade::DevBuf q, qraw, ids, dists, stats, entries, coef, hash;
    int32_t hash_bits = 0;
    int64_t hash_slots = 0;
    unsigned long long tag_base = 0;
};

using namespace dade;

namespace {

// The device copy of count elements of src: src itself when it is device
// memory, else buf (grown as needed) after an asynchronous copy on s.
template <class T>
const T *to_device(const T *src, size_t count, DevBuf &buf, cudaStream_t s, dade_status *st) {
    *st = DADE_OK;
    if (dev_ptr(src)) return src;
    if ((*st = buf.ensure(sizeof(T) * std::max<size_t>(count, 1))) != DADE_OK) return nullptr;
    const cudaError_t e = cudaMemcpyAsync(buf.p, src, sizeof(T) * count, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
        *st = DADE_ECUDA;
        return nullptr;
    }
    return buf.as<T>();
}

dade_status pick_entry(dade_hnsw *h, cudaStream_t s) {
    DevBuf norms;
    DADE_TRY(norms.alloc(sizeof(float) * (size_t)h->n));
    k_hnsw_norms<<<grid_for(h->n, 256), 256, 0, s>>>(h->X.as<float>(), h->n, h->dp, norms.as<float>());
    DADE_TRY(launch_check("k_hnsw_norms"));
    std::vector<float> v((size_t)h->n);
    DADE_TRY_CUDA(cudaMemcpyAsync(v.data(), norms.p, sizeof(float) * (size_t)h->n, cudaMemcpyDeviceToHost, s));
    DADE_TRY_CUDA(cudaStreamSynchronize(s));
    h->entry = std::min_element(v.begin(), v.end()) - v.begin();   // first of equal minima: lowest id
    return DADE_OK;
}

}  // namespace

extern "C" {

void dade_hnsw_build_opts_default(dade_hnsw_build_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->M = 16;
    o->M0 = 32;
    o->kc = 64;
}

void dade_hnsw_search_opts_default(dade_hnsw_search_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->mode = DADE_MODE_DADE;
}

dade_status dade_hnsw_build(const dade_index *ix, const float *base, int64_t n, const dade_hnsw_build_opts *opts,
                            dade_hnsw **out) {
    set_error("");
    DADE_CHECK_ARG(ix != nullptr && base != nullptr && opts != nullptr && out != nullptr, "NULL pointer");
    *out = nullptr;
    DADE_CHECK_ARG(ix->shard < 0, "a shard of an index holds only some of its objects");
    DADE_CHECK_ARG(n == ix->n, "n must be the index's object count (base = the vectors it was built on)");
    DADE_CHECK_ARG(n >= 2 && n <= INT32_MAX, "n outside 2..2^31-1");
    DADE_CHECK_ARG(opts->M >= 1 && opts->M <= 32, "M outside 1..32");
    DADE_CHECK_ARG(opts->M0 >= opts->M && opts->M0 <= 32, "M0 outside M..32");
    DADE_CHECK_ARG(opts->kc >= opts->M && opts->kc < DADE_MAX_K, "kc outside M..255");
    DADE_CHECK_ARG(opts->nprobe >= 0 && opts->nprobe <= ix->nc, "nprobe outside 0..n_clusters");
    const int nprobe = opts->nprobe ? opts->nprobe : std::min(ix->nc, 64);
    const int M = opts->M, M0 = opts->M0, kc = (int)std::min<int64_t>(opts->kc, n - 1), kq = kc + 1;

    dade_hnsw *h = new (std::nothrow) dade_hnsw();
    if (!h) {
        set_error("host allocation failed");
        return DADE_ENOMEM;
    }
    std::unique_ptr<dade_hnsw> own(h);
    h->ix = ix;
    h->n = n;
    h->d = ix->d;
    h->dp = ix->dp;
    h->m0 = M0;
    cudaStream_t s = nullptr;
    DADE_TRY_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } guard{s};

    // rotated rows, row-major (the index's rotation; dims >= d are zero)
    DADE_TRY(h->X.alloc(sizeof(float) * (size_t)n * h->dp));
    const bool base_dev = dev_ptr(base);
    const int64_t chunk = 65536;
    DevBuf stage, kid, kd, cid, cdist, ccnt;
    if (!base_dev) DADE_TRY(stage.alloc(sizeof(float) * (size_t)std::min(n, chunk) * h->d));
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t rows = std::min(chunk, n - r0);
        const float *src = base + r0 * h->d;
        if (!base_dev) {
            DADE_TRY_CUDA(cudaMemcpyAsync(stage.p, src, sizeof(float) * (size_t)rows * h->d,
                                          cudaMemcpyHostToDevice, s));
            src = stage.as<float>();
        }
        DADE_TRY(rotate(ix, src, rows, h->dp, h->X.as<float>() + r0 * h->dp, s));
    }
    DADE_TRY(pick_entry(h, s));

    // candidates: the kc nearest other objects by the index's FDScanning search
    DADE_TRY(kid.alloc(sizeof(int64_t) * (size_t)std::min(n, chunk) * kq));
    DADE_TRY(kd.alloc(sizeof(float) * (size_t)std::min(n, chunk) * kq));
    DADE_TRY(cid.alloc(sizeof(int32_t) * (size_t)n * kc));
    DADE_TRY(cdist.alloc(sizeof(float) * (size_t)n * kc));
    DADE_TRY(ccnt.alloc(sizeof(int32_t) * (size_t)n));
    dade_search_opts so{};
    so.mode = DADE_MODE_FD;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t rows = std::min(chunk, n - r0);
        DADE_TRY(dade_query(ix, base + r0 * h->d, rows, kq, nprobe, 0.5f, 16, &so, kid.as<int64_t>(),
                            kd.as<float>(), (dade_stream)s));
        k_hnsw_cand<<<grid_for(rows, 256), 256, 0, s>>>(kid.as<int64_t>(), kd.as<float>(), n, kq, kc, r0, rows,
                                                        cid.as<int32_t>(), cdist.as<float>(), ccnt.as<int32_t>());
        DADE_TRY(launch_check("k_hnsw_cand"));
    }
    kid.release();
    kd.release();

    // sel(u): the heuristic over the candidates, at most M kept
    DevBuf sel, seld, selc;
    DADE_TRY(sel.alloc(sizeof(int32_t) * (size_t)n * M));
    DADE_TRY(seld.alloc(sizeof(float) * (size_t)n * M));
    DADE_TRY(selc.alloc(sizeof(int32_t) * (size_t)n));
    k_hnsw_select<<<grid_for(n, 8), 256, 0, s>>>(h->X.as<float>(), h->dp, nullptr, kc, ccnt.as<int32_t>(),
                                                 cid.as<int32_t>(), cdist.as<float>(), n, M, sel.as<int32_t>(),
                                                 seld.as<float>(), M, selc.as<int32_t>());
    DADE_TRY(launch_check("k_hnsw_select"));
    cid.release();
    cdist.release();
    ccnt.release();
    std::vector<int32_t> hs((size_t)n * M), hc((size_t)n);
    std::vector<float> hd((size_t)n * M);
    DADE_TRY_CUDA(cudaMemcpyAsync(hs.data(), sel.p, sizeof(int32_t) * hs.size(), cudaMemcpyDeviceToHost, s));
    DADE_TRY_CUDA(cudaMemcpyAsync(hd.data(), seld.p, sizeof(float) * hd.size(), cudaMemcpyDeviceToHost, s));
    DADE_TRY_CUDA(cudaMemcpyAsync(hc.data(), selc.p, sizeof(int32_t) * hc.size(), cudaMemcpyDeviceToHost, s));
    DADE_TRY_CUDA(cudaStreamSynchronize(s));
    sel.release();
    seld.release();
    selc.release();

    // U(v) = sel(v) and every u with v in sel(u), distinct, ascending by (distance, id)
    std::vector<int64_t> rstart((size_t)n + 1, 0);
    for (int64_t u = 0; u < n; ++u)
        for (int t = 0; t < hc[u]; ++t) rstart[(size_t)hs[(size_t)u * M + t] + 1] += 1;
    for (int64_t v = 0; v < n; ++v) rstart[(size_t)v + 1] += rstart[(size_t)v];
    std::vector<int32_t> rid((size_t)rstart[(size_t)n]);
    std::vector<float> rdist((size_t)rstart[(size_t)n]);
    {
        std::vector<int64_t> fill(rstart.begin(), rstart.end() - 1);
        for (int64_t u = 0; u < n; ++u)
            for (int t = 0; t < hc[u]; ++t) {
                const int32_t v = hs[(size_t)u * M + t];
                rid[(size_t)fill[(size_t)v]] = (int32_t)u;
                rdist[(size_t)fill[(size_t)v]++] = hd[(size_t)u * M + t];
            }
    }
    std::vector<int32_t> nbr((size_t)n * M0, -1);
    std::vector<int64_t> long_off(1, 0), long_node;
    std::vector<int32_t> long_id, long_cnt;
    std::vector<float> long_d;
    std::vector<std::pair<float, int32_t>> U;
    for (int64_t v = 0; v < n; ++v) {
        U.clear();
        for (int t = 0; t < hc[v]; ++t) U.emplace_back(hd[(size_t)v * M + t], hs[(size_t)v * M + t]);
        for (int64_t t = rstart[(size_t)v]; t < rstart[(size_t)v + 1]; ++t) U.emplace_back(rdist[(size_t)t], rid[(size_t)t]);
        // distinct ids (the nearer of two computed distances of one pair), then by (distance, id)
        std::sort(U.begin(), U.end(), [](const std::pair<float, int32_t> &a, const std::pair<float, int32_t> &b) {
            return a.second < b.second || (a.second == b.second && a.first < b.first);
        });
        U.erase(std::unique(U.begin(), U.end(), [](const std::pair<float, int32_t> &a,
                                                   const std::pair<float, int32_t> &b) { return a.second == b.second; }),
                U.end());
        std::sort(U.begin(), U.end());
        if ((int)U.size() <= M0) {
            for (size_t t = 0; t < U.size(); ++t) nbr[(size_t)v * M0 + t] = U[t].second;
        } else {
            long_node.push_back(v);
            long_cnt.push_back((int32_t)U.size());
            for (const auto &p : U) {
                long_id.push_back(p.second);
                long_d.push_back(p.first);
            }
            long_off.push_back((int64_t)long_id.size());
        }
    }
    if (!long_node.empty()) {   // the degree cap: the heuristic over U(v), at most M0 kept
        const int64_t nl = (int64_t)long_node.size();
        DevBuf loff, lid, ld, lcnt, lout;
        DADE_TRY(loff.alloc(sizeof(int64_t) * long_off.size()));
        DADE_TRY(lid.alloc(sizeof(int32_t) * long_id.size()));
        DADE_TRY(ld.alloc(sizeof(float) * long_d.size()));
        DADE_TRY(lcnt.alloc(sizeof(int32_t) * (size_t)nl));
        DADE_TRY(lout.alloc(sizeof(int32_t) * (size_t)nl * M0));
        DADE_TRY_CUDA(cudaMemcpyAsync(loff.p, long_off.data(), sizeof(int64_t) * long_off.size(),
                                      cudaMemcpyHostToDevice, s));
        DADE_TRY_CUDA(cudaMemcpyAsync(lid.p, long_id.data(), sizeof(int32_t) * long_id.size(),
                                      cudaMemcpyHostToDevice, s));
        DADE_TRY_CUDA(cudaMemcpyAsync(ld.p, long_d.data(), sizeof(float) * long_d.size(), cudaMemcpyHostToDevice, s));
        DADE_TRY_CUDA(cudaMemcpyAsync(lcnt.p, long_cnt.data(), sizeof(int32_t) * (size_t)nl, cudaMemcpyHostToDevice,
                                      s));
        k_hnsw_select<<<grid_for(nl, 8), 256, 0, s>>>(h->X.as<float>(), h->dp, loff.as<int64_t>(), 0,
                                                      lcnt.as<int32_t>(), lid.as<int32_t>(), ld.as<float>(), nl, M0,
                                                      lout.as<int32_t>(), nullptr, M0, nullptr);
        DADE_TRY(launch_check("k_hnsw_select"));
        std::vector<int32_t> res((size_t)nl * M0);
        DADE_TRY_CUDA(cudaMemcpyAsync(res.data(), lout.p, sizeof(int32_t) * res.size(), cudaMemcpyDeviceToHost, s));
        DADE_TRY_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < nl; ++i)
            std::copy(res.begin() + i * M0, res.begin() + (i + 1) * M0, nbr.begin() + long_node[(size_t)i] * M0);
    }
    DADE_TRY(h->nbr.alloc(sizeof(int32_t) * nbr.size()));
    DADE_TRY_CUDA(cudaMemcpyAsync(h->nbr.p, nbr.data(), sizeof(int32_t) * nbr.size(), cudaMemcpyHostToDevice, s));
    DADE_TRY_CUDA(cudaStreamSynchronize(s));
    *out = own.release();
    return DADE_OK;
}

dade_status dade_hnsw_create(const dade_index *ix, const float *x_rot, int64_t n, int32_t d, const int32_t *nbr,
                             int32_t m0, int64_t entry, dade_hnsw **out) {
    set_error("");
    DADE_CHECK_ARG(x_rot != nullptr && nbr != nullptr && out != nullptr, "NULL pointer");
    *out = nullptr;
    DADE_CHECK_ARG(n >= 1 && n <= INT32_MAX, "n outside 1..2^31-1");
    DADE_CHECK_ARG(d >= 1 && d <= DADE_MAX_DIM, "d outside 1..DADE_MAX_DIM");
    DADE_CHECK_ARG(!ix || ix->d == d, "d differs from the index's");
    DADE_CHECK_ARG(m0 >= 1 && m0 <= 32, "m0 outside 1..32");
    DADE_CHECK_ARG(entry >= 0 && entry < n, "entry outside 0..n-1");
    dade_hnsw *h = new (std::nothrow) dade_hnsw();
    if (!h) {
        set_error("host allocation failed");
        return DADE_ENOMEM;
    }
    std::unique_ptr<dade_hnsw> own(h);
    h->ix = ix;
    h->n = n;
    h->d = d;
    h->dp = (d + 15) / 16 * 16;
    h->m0 = m0;
    h->entry = entry;
    DADE_TRY(h->X.alloc(sizeof(float) * (size_t)n * h->dp));
    DADE_TRY(h->nbr.alloc(sizeof(int32_t) * (size_t)n * m0));
    DADE_TRY_CUDA(cudaMemset(h->X.p, 0, sizeof(float) * (size_t)n * h->dp));
    DADE_TRY_CUDA(cudaMemcpy2D(h->X.p, sizeof(float) * h->dp, x_rot, sizeof(float) * d, sizeof(float) * d, (size_t)n,
                               cudaMemcpyDefault));
    DADE_TRY_CUDA(cudaMemcpy(h->nbr.p, nbr, sizeof(int32_t) * (size_t)n * m0, cudaMemcpyDefault));
    *out = own.release();
    return DADE_OK;
}

dade_status dade_hnsw_search(dade_hnsw *h, const float *q_rot, int64_t nq, int32_t k, int32_t ef, float alpha,
                             int32_t delta_d, const dade_hnsw_search_opts *opts, int64_t *ids, float *dists,
                             dade_stream stream) {
    set_error("");
    DADE_CHECK_ARG(h != nullptr, "structure is NULL");
    DADE_CHECK_ARG(nq >= 0, "nq < 0");
    DADE_CHECK_ARG(k >= 1 && k <= DADE_MAX_K, "k outside 1..DADE_MAX_K");
    DADE_CHECK_ARG(ef >= k && ef <= HMAX_EF, "ef outside k..1024");
    dade_hnsw_search_opts o;
    dade_hnsw_search_opts_default(&o);
    if (opts) o = *opts;
    DADE_CHECK_ARG(o.mode == DADE_MODE_DADE || o.mode == DADE_MODE_FD, "unknown mode");
    DADE_CHECK_ARG(delta_d >= 16 && delta_d <= DADE_MAX_DIM && delta_d % 16 == 0,
                   "delta_d must be a multiple of 16 in [16, 1024]");
    DADE_CHECK_ARG(o.mode == DADE_MODE_FD || o.coef || (alpha > 0.f && alpha < 1.f), "alpha outside (0, 1)");
    DADE_CHECK_ARG(o.mode == DADE_MODE_FD || o.coef || h->ix, "no index for the thresholds: pass opts.coef");
    DADE_CHECK_ARG(!o.entry || (o.n_entry >= 1 && o.n_entry <= HMAX_ENTRY), "n_entry outside 1..64");
    DADE_CHECK_ARG(o.max_visits >= 0, "max_visits < 0");
    if (nq == 0) return DADE_OK;
    DADE_CHECK_ARG(q_rot != nullptr && ids != nullptr && dists != nullptr, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    dade_status st;

    // thresholds c_j of the tested d = delta_d, 2 delta_d, ... < D
    const int n_test = (h->d + delta_d - 1) / delta_d - 1;
    const float *coef = nullptr;
    if (o.mode == DADE_MODE_DADE && n_test > 0) {
        std::vector<float> c((size_t)n_test);
        if (o.coef) {
            std::copy(o.coef, o.coef + n_test, c.begin());
        } else {
            std::vector<float> t((size_t)h->d + 1);
            coef_table(h->ix, alpha, delta_d, nullptr, t.data());
            std::copy(t.begin(), t.begin() + n_test, c.begin());
        }
        DADE_TRY(h->coef.ensure(sizeof(float) * c.size()));
        DADE_TRY_CUDA(cudaMemcpyAsync(h->coef.p, c.data(), sizeof(float) * c.size(), cudaMemcpyHostToDevice, s));
        coef = h->coef.as<float>();
    }
    const float *qd = to_device(q_rot, (size_t)nq * h->d, h->q, s, &st);
    if (!qd) return st;
    const int ne = o.entry ? o.n_entry : 1;
    const int64_t *ed = nullptr;
    if (o.entry && !(ed = to_device(o.entry, (size_t)nq * o.n_entry, h->entries, s, &st))) return st;
    const bool ids_host = !dev_ptr(ids), dists_host = !dev_ptr(dists);
    const bool stats_host = o.stats && !dev_ptr(o.stats);
    if (ids_host) DADE_TRY(h->ids.ensure(sizeof(int64_t) * (size_t)nq * k));
    if (dists_host) DADE_TRY(h->dists.ensure(sizeof(float) * (size_t)nq * k));
    if (stats_host) DADE_TRY(h->stats.ensure(sizeof(int64_t) * (size_t)nq * 5));

    HnswArgs a{};
    a.X = h->X.as<float>();
    a.nbr = h->nbr.as<int32_t>();
    a.n = h->n;
    a.d = h->d;
    a.dp = h->dp;
    a.m0 = h->m0;
    a.q = qd;
    a.nq = nq;
    a.k = k;
    a.ef = ef;
    a.delta_d = delta_d;
    a.coef = coef;
    a.entry = ed;
    a.n_entry = ne;
    a.entry0 = h->entry;
    a.max_visits = o.max_visits ? o.max_visits : std::min<int64_t>(h->n, 64ll * ef + 1024);
    a.ids = ids_host ? h->ids.as<int64_t>() : ids;
    a.dists = dists_host ? h->dists.as<float>() : dists;
    a.stats = o.stats ? (stats_host ? h->stats.as<int64_t>() : o.stats) : nullptr;

    // grid: persistent, at most the resident blocks; a visited table per warp slot
    const size_t smem = (size_t)HW * warp_bytes(h->dp, ef);
    DADE_TRY(kernel_smem((const void *)k_hnsw_search, smem));
    int blocks = 0;
    DADE_TRY(resident_blocks((const void *)k_hnsw_search, HW * 32, smem, &blocks));
    const int64_t words = 2 * (std::min<int64_t>(a.max_visits, h->n) + h->m0 + ne);
    int bits = 6;
    while ((1ll << bits) < words) ++bits;
    // visited tables of at most 2 GiB in all: fewer warps when a query may visit many objects
    const int64_t max_slots = std::max<int64_t>(HW, (2ll << 30) / (8ll << bits));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>({(int64_t)blocks, (nq + HW - 1) / HW, max_slots / HW}));
    const int64_t slots = grid * HW;
    if (bits != h->hash_bits || slots > h->hash_slots) {
        h->hash.release();
        DADE_TRY(h->hash.alloc(sizeof(unsigned long long) * ((size_t)slots << bits)));
        DADE_TRY_CUDA(cudaMemsetAsync(h->hash.p, 0, sizeof(unsigned long long) * ((size_t)slots << bits), s));
        h->hash_bits = bits;
        h->hash_slots = slots;
        h->tag_base = 0;
    }
    if (h->tag_base + (unsigned long long)nq + 1 >= 0xffffffffull) {   // tags would wrap: forget every visit
        DADE_TRY_CUDA(cudaMemsetAsync(h->hash.p, 0, sizeof(unsigned long long) * ((size_t)h->hash_slots << bits), s));
        h->tag_base = 0;
    }
    a.hash = h->hash.as<unsigned long long>();
    a.hbits = bits;
    a.tag0 = (unsigned)h->tag_base;
    h->tag_base += (unsigned long long)nq;
    k_hnsw_search<<<(unsigned)grid, HW * 32, smem, s>>>(a);
    DADE_TRY(launch_check("k_hnsw_search"));
    if (ids_host)
        DADE_TRY_CUDA(cudaMemcpyAsync(ids, a.ids, sizeof(int64_t) * (size_t)nq * k, cudaMemcpyDeviceToHost, s));
    if (dists_host)
        DADE_TRY_CUDA(cudaMemcpyAsync(dists, a.dists, sizeof(float) * (size_t)nq * k, cudaMemcpyDeviceToHost, s));
    if (stats_host)
        DADE_TRY_CUDA(cudaMemcpyAsync(o.stats, a.stats, sizeof(int64_t) * (size_t)nq * 5, cudaMemcpyDeviceToHost, s));
    if (ids_host || dists_host || stats_host) DADE_TRY_CUDA(cudaStreamSynchronize(s));
    return DADE_OK;
}

dade_status dade_hnsw_query(dade_hnsw *h, const float *q, int64_t nq, int32_t k, int32_t ef, float alpha,
                            int32_t delta_d, const dade_hnsw_search_opts *opts, int64_t *ids, float *dists,
                            dade_stream stream) {
    set_error("");
    DADE_CHECK_ARG(h != nullptr, "structure is NULL");
    DADE_CHECK_ARG(h->ix != nullptr, "no index to rotate the queries with: rotate them and call dade_hnsw_search");
    DADE_CHECK_ARG(nq >= 0, "nq < 0");
    if (nq == 0) return dade_hnsw_search(h, nullptr, 0, k, ef, alpha, delta_d, opts, ids, dists, stream);
    DADE_CHECK_ARG(q != nullptr, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    dade_status st;
    const float *qd = to_device(q, (size_t)nq * h->d, h->qraw, s, &st);
    if (!qd) return st;
    DevBuf &qr = h->q;
    DADE_TRY(qr.ensure(sizeof(float) * (size_t)nq * h->d));
    DADE_TRY(rotate(h->ix, qd, nq, h->d, qr.as<float>(), s));
    return dade_hnsw_search(h, qr.as<float>(), nq, k, ef, alpha, delta_d, opts, ids, dists, stream);
}

dade_status dade_hnsw_info_get(const dade_hnsw *h, dade_hnsw_info *out) {
    set_error("");
    DADE_CHECK_ARG(h != nullptr && out != nullptr, "NULL pointer");
    std::memset(out, 0, sizeof(*out));
    out->n = h->n;
    out->d = h->d;
    out->m0 = h->m0;
    out->entry = h->entry;
    out->device_bytes = (int64_t)(h->X.bytes + h->nbr.bytes);
    return DADE_OK;
}

dade_status dade_hnsw_graph(const dade_hnsw *h, int32_t *nbr) {
    set_error("");
    DADE_CHECK_ARG(h != nullptr && nbr != nullptr, "NULL pointer");
    DADE_TRY_CUDA(cudaMemcpy(nbr, h->nbr.p, sizeof(int32_t) * (size_t)h->n * h->m0, cudaMemcpyDefault));
    return DADE_OK;
}

void dade_hnsw_free(dade_hnsw *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    delete h;
}

}  // extern "C"
