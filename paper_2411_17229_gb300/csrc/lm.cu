// lm.cu -- the seeded schedule (DADE_SCHED_SEEDED): the first S probed lists
// of every query run in the tile schedule (scan.cu); r is then frozen at the
// K-th distance found, and the later lists are scanned list-major.
//
// List-major: the (query, list) pairs of probe positions >= S are grouped by
// list (counting sort), and the groups split into work items of at most 32
// queries.  One persistent launch pops items from a counter.  For an item the
// CTA stages the list's first increment tile by tile (cp.async.bulk, two
// tiles in flight) once, and each warp runs Algorithm 1 for its queries of
// the item against the staged rows: first increment from shared memory, the
// survivors' later blocks gathered from global memory (the list is hot in L2
// while the item runs), the Section 3.3 test against the query's frozen r,
// the exact compare at d = D.  Accepted candidates are appended, as 64-bit
// (distance bits, id) keys, to the query's own region of an accept buffer.
// A candidate's outcome depends only on its query's frozen r, so the order in
// which items and warps run does not change the result.  A final merge per
// query takes the K smallest keys of the first-S-lists result and of its
// accepted candidates (radix select, then rank sort).
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "scan_common.cuh"

namespace dade {

dade_status exclusive_scan_int(int *a, int n, cudaStream_t s);

namespace {
using namespace scanning;

constexpr int LT = 64;          // candidates per staged tile
constexpr int LG = 32;           // queries per work item
constexpr int LNT = 256;         // threads per CTA
constexpr int LNW = LNT / 32;    // warps
constexpr int LNB = 8;           // 16-dim blocks (D in 113..128)

struct LmArgs {
    const float *data;
    const int32_t *ids;
    const ListMeta *meta;
    const float *q_rot;
    const int32_t *lq_items;     // queries grouped by list
    const int *lq_off;           // [nc + 1] first entry of list c in lq_items
    const int *item_off;         // [nc + 1] first work item of list c
    unsigned *ctr;               // work counter
    const float *r2src;          // first-phase squared distances [nq][k]; r^2 = entry k - 1 (k: the query's)
    const int32_t *q_k;          // per-query K (at most k, the row stride), or NULL for k
    unsigned long long *acc;     // [nq][cap] accepted keys
    int *acnt;                   // [nq]
    int64_t *stats;              // [nq][4], added to; or null
    int *err;
    const float *tail;           // row-major tail copy or null
    int64_t cap;
    int q_stride, nc, k, d, tail_nb0, tail_w;
    int nb, n_inc;               // 16-dim blocks of the layout, increments (k_lm_g)
    int chunk_tiles;             // tiles of a list per work item (a long list is several items)
    int lg;                      // queries per work item (k_lm_tc: 32 or 64; the others LG)
    uint64_t wait_ns;            // limit of every bounded wait on a copy or an MMA
    const int *never;            // failure-path check: a device word nothing sets (else NULL)
    int row_lo, row_hi;          // rows [row_lo, min(len, row_hi)) of every list are scanned; tiles
                                 // of LT rows start at row_lo
    // tensor-core prefilter (k_lm_tc)
    int64_t *lead_stats;         // [nq] candidates dropped by the prefilter (added to), or null
    float tc_c1, tc_c2;          // error bound of the expanded partial distance (see k_lm_tc)
    float coef[DADE_MAX_DIM / DADE_BLOCK];   // prune iff P > coef[j] r^2 after increment j
};

// The K of query q (rows of r2src and of the results have k entries).
__device__ __forceinline__ int lm_kq(const LmArgs &a, int64_t q) {
    return a.q_k ? min(max(a.q_k[q], 1), a.k) : a.k;
}

// End of the rows of a list of `len` members that a pass scans.
__device__ __forceinline__ int lm_end(const LmArgs &a, int len) { return min(len, a.row_hi); }

struct LmSmem {
    static constexpr size_t stage(int gb) { return sizeof(float) * (size_t)gb * LT * 16; }
    static size_t total_g(int gb);   // k_lm_g: only the first increment of each query staged (below)
    static size_t total(int gb) {
        return 2 * stage(gb) + sizeof(float) * LG * 16 * LNB + sizeof(Surv) * LNW * LT;
    }
};

__device__ __forceinline__ float quad_sum4(float p) {
    p += __shfl_xor_sync(0xffffffffu, p, 1);
    p += __shfl_xor_sync(0xffffffffu, p, 2);
    return p;
}

// Warp-aggregated append of the lanes with `take` to query q's accept region.
__device__ __forceinline__ void lm_append(const LmArgs &a, bool take, int q, unsigned long long key) {
    const int lane = threadIdx.x & 31;
    const unsigned mk = __ballot_sync(0xffffffffu, take);
    if (mk == 0) return;
    const int leader = __ffs(mk) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&a.acnt[q], __popc(mk));
    base = __shfl_sync(0xffffffffu, base, leader);
    const int64_t pos = (int64_t)base + __popc(mk & ((1u << lane) - 1u));
    if (take) {
        if (pos < a.cap) a.acc[(int64_t)q * a.cap + pos] = key;
        else atomicExch(a.err, (int)DADE_ENOMEM);   // accept buffer full: the call reports it
    }
}

// Per-item K-best staging of accepted keys (K <= KB_K): within one work item a
// query's accepted keys are staged per (warp, query slot) and cut back to its
// K smallest whenever the stage fills; only those reach the query's accept
// buffer.  Exact: the final merge keeps the K smallest keys overall, and a key
// beaten by K others of the same item cannot be among them.  This bounds what
// an item adds per query (K), however many candidates pass a loose r.
constexpr int KB = 64;            // staged keys per (warp, query slot)
constexpr int KB_K = KB - 32;     // largest K staged (one append adds up to 32)
constexpr int QSLOT = LG / LNW;   // query slots per warp: the item's queries warp + LNW * slot

struct KBest {
    unsigned long long key[LNW][QSLOT][KB];
    int cnt[LNW][QSLOT];
};

// Keep the k smallest staged keys of (w, s) at the front (keys are unique). Whole warp.
__device__ void kb_compact(KBest &kb, int w, int s, int k) {
    const int lane = threadIdx.x & 31;
    const int n = kb.cnt[w][s];
    const unsigned long long v0 = lane < n ? kb.key[w][s][lane] : ~0ull;
    const unsigned long long v1 = lane + 32 < n ? kb.key[w][s][lane + 32] : ~0ull;
    int r0 = 0, r1 = 0;
    for (int j = 0; j < n; ++j) {
        const unsigned long long x = kb.key[w][s][j];
        r0 += x < v0;
        r1 += x < v1;
    }
    __syncwarp();
    if (lane < n && r0 < k) kb.key[w][s][r0] = v0;
    if (lane + 32 < n && r1 < k) kb.key[w][s][r1] = v1;
    __syncwarp();
    if (lane == 0) kb.cnt[w][s] = min(n, k);
    __syncwarp();
}

// Stage the keys of the lanes with `take` for (w, s).  Whole warp.
__device__ void kb_take(KBest &kb, int w, int s, int k, bool take, unsigned long long key) {
    const int lane = threadIdx.x & 31;
    const unsigned mk = __ballot_sync(0xffffffffu, take);
    if (mk == 0) return;
    if (kb.cnt[w][s] + __popc(mk) > KB) kb_compact(kb, w, s, k);
    const int n = kb.cnt[w][s];
    __syncwarp();
    if (take) kb.key[w][s][n + __popc(mk & ((1u << lane) - 1u))] = key;
    __syncwarp();
    if (lane == 0) kb.cnt[w][s] = n + __popc(mk);
    __syncwarp();
}

// Move the staged K best of (w, s) to query q's accept buffer.  Whole warp.
__device__ void kb_flush(const LmArgs &a, KBest &kb, int w, int s, int q) {
    const int lane = threadIdx.x & 31;
    if (kb.cnt[w][s] > a.k) kb_compact(kb, w, s, a.k);
    const int n = kb.cnt[w][s];
    for (int b = 0; b < n; b += 32) {
        const bool take = b + lane < n;
        lm_append(a, take, q, take ? kb.key[w][s][b + lane] : 0ull);
    }
    __syncwarp();
    if (lane == 0) kb.cnt[w][s] = 0;
    __syncwarp();
}

template <int GB, bool STATS>
__global__ void __launch_bounds__(LNT, 3) k_lm(const LmArgs a) {
    constexpr int NINC = (LNB + GB - 1) / GB;
    constexpr int NREST = LNB - GB;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_item, s_q[LG];
    __shared__ float s_r2[LG];
    float *stage = reinterpret_cast<float *>(smem);
    float *qs = reinterpret_cast<float *>(smem + 2 * LmSmem::stage(GB));
    Surv *survs = reinterpret_cast<Surv *>(smem + 2 * LmSmem::stage(GB) + sizeof(float) * LG * 16 * LNB);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quad = lane >> 2, lq = lane & 3;

    if (tid == 0) {
        mbar_init(su32(&bars[0]), 1);
        mbar_init(su32(&bars[1]), 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t used[2] = {0u, 0u};   // completed waits per buffer (the same on every thread)
    const int total = a.item_off[a.nc];

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(a.ctr, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        int lo = 0, hi = a.nc;   // the list c with item_off[c] <= item < item_off[c + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.item_off[mid] <= item) lo = mid;
            else hi = mid;
        }
        const int c = lo;
        // item = (chunk of the list's tiles) x (group of up to LG of its queries)
        const int ngroups = (a.lq_off[c + 1] - a.lq_off[c] + LG - 1) / LG;
        const int local = item - a.item_off[c];
        const int qb = a.lq_off[c] + (local % ngroups) * LG;
        const int ng = min(LG, a.lq_off[c + 1] - qb);
        const ListMeta m = a.meta[c];
        const int rend = lm_end(a, m.len);   // tile t: rows [row_lo + t LT, ...) up to rend
        const int t0 = (local / ngroups) * a.chunk_tiles;
        const int ntile = min(max(0, (rend - a.row_lo + LT - 1) / LT), t0 + a.chunk_tiles);   // end of this item's tiles
        auto issue = [&](int t) {   // thread 0: first-increment slabs of tile t
            const int buf = t & 1, i0 = a.row_lo + t * LT, tn = min(LT, rend - i0);
            const uint32_t bar = su32(&bars[buf]);
            mbar_expect_tx(bar, (uint32_t)(GB * tn * 64));
            for (int b = 0; b < GB; ++b)
                bulk_g2s(su32(stage + (size_t)buf * GB * LT * 16 + (size_t)b * LT * 16),
                         a.data + m.base + (int64_t)b * m.np * 16 + (int64_t)i0 * 16, (uint32_t)(tn * 64), bar);
        };
        if (tid == 0)
            for (int t = t0; t < t0 + 2 && t < ntile; ++t) issue(t);
        for (int g = tid; g < ng; g += LNT) {
            const int q = a.lq_items[qb + g];
            s_q[g] = q;
            s_r2[g] = a.r2src[(int64_t)q * a.k + lm_kq(a, q) - 1];
        }
        for (int e = tid; e < ng * 16 * LNB; e += LNT) {
            const int g = e / (16 * LNB), kk = e % (16 * LNB);
            qs[e] = kk < a.d ? a.q_rot[(int64_t)a.lq_items[qb + g] * a.q_stride + kk] : 0.f;
        }
        __syncthreads();

        for (int t = t0; t < ntile; ++t) {
            const int buf = t & 1;
            if (!wait_block(su32(&bars[buf]), used[buf] & 1u, a.wait_ns, (used[0] | used[1]) == 0 ? a.never : nullptr)) {
                if (tid == 0) {   // both buffers' copies may still be in flight: let them land (bounded)
                    atomicExch(a.err, (int)DADE_ETIMEOUT);
                    wait_bounded(su32(&bars[buf]), used[buf] & 1u, 10000000ull);
                    if (t + 1 < ntile) wait_bounded(su32(&bars[buf ^ 1]), used[buf ^ 1] & 1u, 10000000ull);
                }
                return;
            }
            ++used[buf];
            const int i0 = a.row_lo + t * LT, tn = min(LT, rend - i0);
            const float *st = stage + (size_t)buf * GB * LT * 16;
            for (int g = warp; g < ng; g += LNW) {
                const int q = s_q[g];
                const float r2 = s_r2[g];
                const float *qv = qs + g * 16 * LNB;
                float4 qa[GB];
#pragma unroll
                for (int b = 0; b < GB; ++b) qa[b] = *reinterpret_cast<const float4 *>(qv + b * 16 + lq * 4);
                Surv *sv = survs + warp * LT;
                int nsv = 0;
                unsigned long long st_c = 0, st_d = 0, st_a = 0, st_p = 0;
                const float c0 = a.coef[0] * r2;
                for (int k0 = 0; k0 < tn; k0 += 16) {
                    float pp[2];
                    bool aa[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int cand = k0 + 8 * h + quad;
                        aa[h] = cand < tn;
                        float p = 0.f;
                        if (aa[h]) {
#pragma unroll
                            for (int b = 0; b < GB; ++b)
                                p += sqd4(qa[b], *reinterpret_cast<const float4 *>(st + ((size_t)b * LT + cand) * 16 + lq * 4));
                        }
                        pp[h] = p;
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int cand = k0 + 8 * h + quad;
                        const bool act = aa[h];
                        const float p = quad_sum4(pp[h]);
                        const bool lead = act && lq == 0;
                        if (NINC == 1) {
                            const bool take = lead && p <= r2;
                            const int id = take ? a.ids[m.slot + i0 + cand] : 0;
                            lm_append(a, take, q, ((unsigned long long)__float_as_uint(p) << 32) | (unsigned)id);
                            if (STATS && lead) { ++st_c; st_d += a.d; st_a += take; }
                        } else {
                            const bool keep = lead && !(p > c0);
                            const unsigned mk = __ballot_sync(0xffffffffu, keep);
                            if (keep) sv[nsv + __popc(mk & ((1u << lane) - 1u))] = Surv{cand, p};
                            nsv += __popc(mk);
                            if (STATS && lead) {
                                ++st_c;
                                if (!keep) { st_d += min(GB * 16, a.d); ++st_p; }
                            }
                        }
                    }
                }
                __syncwarp();
                if (NINC > 1) {
                    for (int r0 = 0; r0 < nsv; r0 += 8) {
                        const int sidx = r0 + quad;
                        const bool act = sidx < nsv;
                        const Surv v = act ? sv[sidx] : Surv{0, 0.f};
                        const int64_t i = i0 + v.idx;
                        const float *row = a.data + m.base + i * 16 + lq * 4;
                        const float *trow =
                            a.tail ? a.tail + (m.slot + i) * a.tail_w + lq * 4 - (int64_t)a.tail_nb0 * 16 : nullptr;
                        float4 o[NREST > 0 ? NREST : 1];
#pragma unroll
                        for (int u = 0; u < NREST; ++u) {
                            const int b = GB + u;
                            const float *src = (trow && b >= a.tail_nb0) ? trow + b * 16 : row + (int64_t)b * m.np * 16;
                            o[u] = act ? __ldg(reinterpret_cast<const float4 *>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        float p = v.p;
                        bool alive = act;
#pragma unroll
                        for (int j = 1; j < NINC; ++j) {
                            float part = 0.f;
#pragma unroll
                            for (int b = j * GB; b < (j + 1) * GB && b < LNB; ++b)
                                part += sqd4(*reinterpret_cast<const float4 *>(qv + b * 16 + lq * 4), o[b - GB]);
                            part = quad_sum4(part);
                            p += part;
                            if (j < NINC - 1 && alive && p > a.coef[j] * r2) {
                                alive = false;
                                if (STATS && lq == 0) { st_d += min((j + 1) * GB * 16, a.d); ++st_p; }
                            }
                        }
                        const bool take = alive && lq == 0 && p <= r2;
                        if (STATS && alive && lq == 0) { st_d += a.d; st_a += take; }
                        const int id = take ? a.ids[m.slot + i] : 0;
                        lm_append(a, take, q, ((unsigned long long)__float_as_uint(p) << 32) | (unsigned)id);
                    }
                }
                if (STATS) {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        st_c += __shfl_xor_sync(0xffffffffu, st_c, off);
                        st_d += __shfl_xor_sync(0xffffffffu, st_d, off);
                        st_a += __shfl_xor_sync(0xffffffffu, st_a, off);
                        st_p += __shfl_xor_sync(0xffffffffu, st_p, off);
                    }
                    if (lane == 0) {
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 0]), st_c);
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 1]), st_d);
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 2]), st_a);
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 3]), st_p);
                    }
                }
                __syncwarp();   // this warp's survivor list is reused by its next query
            }
            __syncthreads();    // every warp is done with buffer buf
            if (tid == 0 && t + 2 < ntile) issue(t + 2);
        }
    }
}

// Survivors a warp has queued over the tiles of an item, finished in bulk:
// entries (query slot g << 26 | row of the list, FP32 partial distance over
// the first increment; with FIRST the first increment is still to be summed
// from the FP32 rows, in the plain kernels' order, and tested).  One quad per
// entry, eight entries per step: the later increments are walked in windows
// of WB blocks (one round trip each, the query's blocks read through L1),
// testing at every increment boundary against the entry's query's frozen
// r^2, then the exact compare at d = D; accepted keys go to the query's
// K-best stage (or its accept region).  Queueing takes the survivors' global
// round trips out of the per-tile barrier: the warp that queued them drains
// them when its queue fills or the item ends.
constexpr int QCAP = 256;         // survivors queued per warp
// A queued survivor's idx packs the item's query slot (6 bits, 0..63) above its row in the
// list (26 bits), read as an unsigned word: the list-major passes need lists below 2^26 rows.
constexpr int QROW_BITS = 26;
__device__ __forceinline__ int surv_key(int g, int row) {
    return (int)(((unsigned)g << QROW_BITS) | (unsigned)row);
}

inline size_t LmSmem::total_g(int gb) {
    return 2 * stage(gb) + sizeof(float) * LG * 16 * gb + sizeof(Surv) * LNW * QCAP;
}

// NSL: query slots per warp (the item's queries g = warp + LNW * slot); kb: the
// per-item K-best stage, or NULL (accepted keys go straight to the accept buffers).
template <int GB, bool STATS, bool FIRST, int NSL = QSLOT>
__device__ void lm_drain(const LmArgs &a, const ListMeta &m, const Surv *sv, int n, const int *s_q, const float *s_r2,
                         const float *s_thr, const float *qs, KBest *kb) {
    constexpr int WB = 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quad = lane >> 2, lq = lane & 3;
    const int nb = a.nb, n_inc = a.n_inc;
    for (int r0 = 0; r0 < n; r0 += 8) {
        const int sidx = r0 + quad;
        const bool act = sidx < n;
        const Surv v = act ? sv[sidx] : Surv{0, 0.f};
        const int g = (int)((unsigned)v.idx >> QROW_BITS);
        const int64_t i = v.idx & ((1 << QROW_BITS) - 1);
        const int q = s_q[g];
        const float r2 = s_r2[g];
        const float *row = a.data + m.base + i * 16 + lq * 4;
        float p = v.p;
        bool alive = act;
        if (FIRST) {
            p = 0.f;
            if (act) {
#pragma unroll
                for (int b = 0; b < GB; ++b)
                    p += sqd4(*reinterpret_cast<const float4 *>(qs + g * 16 * GB + b * 16 + lq * 4),
                              __ldg(reinterpret_cast<const float4 *>(row + (int64_t)b * m.np * 16)));
            }
            p = quad_sum4(p);
            if (alive && p > s_thr[g]) {
                alive = false;
                if (STATS && lq == 0) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 1]),
                              (unsigned long long)min(GB * 16, a.d));
                    atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 3]), 1ull);
                }
            }
        }
        const float *qrow = a.q_rot + (int64_t)q * a.q_stride;
        const float *trow = a.tail ? a.tail + (m.slot + i) * a.tail_w + lq * 4 - (int64_t)a.tail_nb0 * 16 : nullptr;
        float part = 0.f;
        int jj = 1, bend = min(2 * GB, nb);
        for (int wb = GB; wb < nb; wb += WB) {
            if (!__any_sync(0xffffffffu, alive)) break;
            float4 o[WB];
#pragma unroll
            for (int u = 0; u < WB; ++u) {
                const int b = wb + u;
                const float *src = (trow && b >= a.tail_nb0) ? trow + b * 16 : row + (int64_t)b * m.np * 16;
                o[u] = (b < nb && alive) ? __ldg(reinterpret_cast<const float4 *>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < WB; ++u) {
                const int b = wb + u;
                if (b < nb) {
                    float qv[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int kk = b * 16 + lq * 4 + t;
                        qv[t] = kk < a.d ? __ldg(qrow + kk) : 0.f;
                    }
                    part += sqd4(make_float4(qv[0], qv[1], qv[2], qv[3]), o[u]);
                    if (b + 1 == bend) {   // end of increment jj
                        part = quad_sum4(part);
                        if (alive) {
                            p += part;
                            if (jj < n_inc - 1 && p > a.coef[jj] * r2) {
                                alive = false;
                                if (STATS && lq == 0) {
                                    atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 1]),
                                              (unsigned long long)min((jj + 1) * GB * 16, a.d));
                                    atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 3]), 1ull);
                                }
                            }
                        }
                        part = 0.f;
                        ++jj;
                        bend = min(bend + GB, nb);
                    }
                }
            }
        }
        const bool take = alive && lq == 0 && p <= r2;
        if (STATS && alive && lq == 0) {
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 1]), (unsigned long long)a.d);
            if (take) atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 2]), 1ull);
        }
        const int id = take ? a.ids[m.slot + i] : 0;
        const unsigned long long key = ((unsigned long long)__float_as_uint(p) << 32) | (unsigned)id;
        // the warp's queries are slots g = warp + LNW s; stage each slot's accepted keys together
#pragma unroll
        for (int sl = 0; sl < NSL; ++sl) {
            const bool ts = take && g == warp + LNW * sl;
            if (kb) kb_take(*kb, warp, sl, a.k, ts, key);
            else lm_append(a, ts, s_q[warp + LNW * sl], key);
        }
    }
}

// The list-major kernel for any D (blocks nb > GB): the same items, tiles
// and phase A as k_lm, with only the first increment of each query staged in
// shared memory; phase B walks a survivor's later blocks in windows of 8
// (one round trip each, its query's blocks read through L1), testing at
// every increment boundary, and a warp stops as soon as its 8 survivors are
// all pruned.
template <int GB, bool STATS>
__global__ void __launch_bounds__(LNT, 3) k_lm_g(const LmArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_item, s_q[LG];
    __shared__ float s_r2[LG], s_thr[LG];
    __shared__ KBest kb;
    const bool kbest = a.k <= KB_K;   // stage per item (small K), else append directly
    float *stage = reinterpret_cast<float *>(smem);
    float *qs = reinterpret_cast<float *>(smem + 2 * LmSmem::stage(GB));
    Surv *survs = reinterpret_cast<Surv *>(smem + 2 * LmSmem::stage(GB) + sizeof(float) * LG * 16 * GB);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quad = lane >> 2, lq = lane & 3;
    Surv *queue = survs + warp * QCAP;   // this warp's survivors, drained when full or at the item's end
    int qn = 0;                          // entries queued (the same on every lane of the warp)

    if (tid == 0) {
        mbar_init(su32(&bars[0]), 1);
        mbar_init(su32(&bars[1]), 1);
        fence_mbar_init();
    }
    if (tid < LNW * QSLOT) kb.cnt[tid / QSLOT][tid % QSLOT] = 0;
    __syncthreads();
    uint32_t used[2] = {0u, 0u};
    const int total = a.item_off[a.nc];

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(a.ctr, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        int lo = 0, hi = a.nc;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.item_off[mid] <= item) lo = mid;
            else hi = mid;
        }
        const int c = lo;
        // item = (chunk of the list's tiles) x (group of up to LG of its queries)
        const int ngroups = (a.lq_off[c + 1] - a.lq_off[c] + LG - 1) / LG;
        const int local = item - a.item_off[c];
        const int qb = a.lq_off[c] + (local % ngroups) * LG;
        const int ng = min(LG, a.lq_off[c + 1] - qb);
        const ListMeta m = a.meta[c];
        const int rend = lm_end(a, m.len);   // tile t: rows [row_lo + t LT, ...) up to rend
        const int t0 = (local / ngroups) * a.chunk_tiles;
        const int ntile = min(max(0, (rend - a.row_lo + LT - 1) / LT), t0 + a.chunk_tiles);   // end of this item's tiles
        auto issue = [&](int t) {
            const int buf = t & 1, i0 = a.row_lo + t * LT, tn = min(LT, rend - i0);
            const uint32_t bar = su32(&bars[buf]);
            mbar_expect_tx(bar, (uint32_t)(GB * tn * 64));
            for (int b = 0; b < GB; ++b)
                bulk_g2s(su32(stage + (size_t)buf * GB * LT * 16 + (size_t)b * LT * 16),
                         a.data + m.base + (int64_t)b * m.np * 16 + (int64_t)i0 * 16, (uint32_t)(tn * 64), bar);
        };
        if (tid == 0)
            for (int t = t0; t < t0 + 2 && t < ntile; ++t) issue(t);
        for (int g = tid; g < ng; g += LNT) {
            const int q = a.lq_items[qb + g];
            s_q[g] = q;
            const float r2 = a.r2src[(int64_t)q * a.k + lm_kq(a, q) - 1];
            s_r2[g] = r2;
            s_thr[g] = a.coef[0] * r2;
        }
        for (int e = tid; e < ng * 16 * GB; e += LNT) {
            const int g = e / (16 * GB), kk = e % (16 * GB);
            qs[e] = kk < a.d ? a.q_rot[(int64_t)a.lq_items[qb + g] * a.q_stride + kk] : 0.f;
        }
        for (int t = t0; t < ntile; ++t) {
            const int buf = t & 1;
            if (!wait_block(su32(&bars[buf]), used[buf] & 1u, a.wait_ns, (used[0] | used[1]) == 0 ? a.never : nullptr)) {
                if (tid == 0) {   // both buffers' copies may still be in flight: let them land (bounded)
                    atomicExch(a.err, (int)DADE_ETIMEOUT);
                    wait_bounded(su32(&bars[buf]), used[buf] & 1u, 10000000ull);
                    if (t + 1 < ntile) wait_bounded(su32(&bars[buf ^ 1]), used[buf ^ 1] & 1u, 10000000ull);
                }
                return;
            }
            ++used[buf];
            const int i0 = a.row_lo + t * LT, tn = min(LT, rend - i0);
            const float *st = stage + (size_t)buf * GB * LT * 16;
            for (int g = warp; g < ng; g += LNW) {
                if (qn + LT > QCAP) {   // room for this query's survivors of the tile
                    lm_drain<GB, STATS, false>(a, m, queue, qn, s_q, s_r2, s_thr, qs, kbest ? &kb : nullptr);
                    qn = 0;
                    __syncwarp();
                }
                const int q = s_q[g];
                float4 qa[GB];
#pragma unroll
                for (int b = 0; b < GB; ++b)
                    qa[b] = *reinterpret_cast<const float4 *>(qs + g * 16 * GB + b * 16 + lq * 4);
                unsigned long long st_c = 0, st_d = 0, st_a = 0, st_p = 0;
                const float c0 = s_thr[g];
                for (int k0 = 0; k0 < tn; k0 += 8) {
                    const int cand = k0 + quad;
                    const bool act = cand < tn;
                    float p = 0.f;
                    if (act) {
#pragma unroll
                        for (int b = 0; b < GB; ++b)
                            p += sqd4(qa[b], *reinterpret_cast<const float4 *>(st + ((size_t)b * LT + cand) * 16 + lq * 4));
                    }
                    p = quad_sum4(p);
                    const bool lead = act && lq == 0;
                    const bool keep = lead && !(p > c0);
                    const unsigned mk = __ballot_sync(0xffffffffu, keep);
                    if (keep) queue[qn + __popc(mk & ((1u << lane) - 1u))] = Surv{surv_key(g, i0 + cand), p};
                    qn += __popc(mk);
                    if (STATS && lead) {
                        ++st_c;
                        if (!keep) { st_d += min(GB * 16, a.d); ++st_p; }
                    }
                }
                if (STATS) {
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        st_c += __shfl_xor_sync(0xffffffffu, st_c, off);
                        st_d += __shfl_xor_sync(0xffffffffu, st_d, off);
                        st_a += __shfl_xor_sync(0xffffffffu, st_a, off);
                        st_p += __shfl_xor_sync(0xffffffffu, st_p, off);
                    }
                    if (lane == 0) {
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 0]), st_c);
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 1]), st_d);
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 2]), st_a);
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 3]), st_p);
                    }
                }
                __syncwarp();
            }
            __syncthreads();
            if (tid == 0 && t + 2 < ntile) issue(t + 2);
        }
        __syncwarp();
        lm_drain<GB, STATS, false>(a, m, queue, qn, s_q, s_r2, s_thr, qs, kbest ? &kb : nullptr);
        qn = 0;
        __syncwarp();
        if (kbest)   // the item's K best per query go to the accept buffers
            for (int g = warp; g < ng; g += LNW) kb_flush(a, kb, warp, g / LNW, s_q[g]);
    }
}

// ---- the first increment on the tensor cores (list-major passes) -----------------------
// For a tile of LTC candidates of one list and the item's queries (up to LGT),
// the partial distance over the first increment is expanded as
//     X = ||q'||^2 + ||o'||^2 - 2 q'.o'   (FP32 rows q', o' of the index).
// The tile's FP32 rows arrive by TMA in the tensor cores' canonical K-major
// layout without swizzle: per 16-dim block b and 4-float chunk kc, a box of
// 4 floats x 128 rows (16 B per row; core matrices of 8 rows contiguous).  One
// thread issues tcgen05.mma kind::tf32 (A = the tile, M = 128 candidates, read
// by the tensor core as TF32; B = the item's queries rounded to TF32, N = 64;
// K = 8 dims per instruction; FP32 accumulation in tensor memory),
// two accumulators in turn, so that the MMA of the next tile runs while the
// threads read this one's (tcgen05.ld).  Every (query, candidate) pair is then
// tested with a certified bound: X - E is a lower bound of the exact partial
// distance, E = c1 (||q'||^2 + ||o'||^2) + c2 ||q'|| ||o'|| covering the TF32
// reading of the rows (2^-10), the rounding of the queries to TF32 (2^-11), the FP32 sums
// and the tensor-core accumulation (host-side constants); a pair is dropped
// only when X - E exceeds the FP32 threshold by 2^-15 relative, more than the
// rounding of the FP32 path's own partial sum, so the FP32 test would drop it
// too.  Every other pair runs the FP32 path from the staged rows (the same
// float4 per lane and the same order as the plain kernels) and its
// survivors are queued for the later increments: results and counters are
// those of the FP32 list-major path.
constexpr int LTC = 128;            // candidates per tile: M of the MMA
constexpr int LGT = 64;             // queries per work item of k_lm_tc
constexpr int TCN = LGT;            // N of the MMA: the item's queries, one TF32 part each
constexpr uint32_t TC_COLS = 128;   // tensor-memory columns: two FP32 accumulators of N = 64

// Instruction descriptor of kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N / 8 at bits 17-22,
// M / 16 at bits 24-28.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TCN >> 3) << 17) |
                              ((uint32_t)(LTC >> 4) << 24);

// Staged tiles of k_lm_tc: a ring of four for increments of up to 32 dims, two
// for 64 dims (two blocks per SM must fit; see the tile loop).
constexpr int tc_ring(int gb) { return gb >= 4 ? 2 : 4; }

struct TcSmem {   // dynamic shared memory of k_lm_tc (1024-byte aligned base)
    static constexpr size_t a_bytes(int gb) { return (size_t)gb * 4 * LTC * 16; }   // FP32 rows of one tile
    static constexpr size_t b_off(int gb) { return tc_ring(gb) * a_bytes(gb); }     // the ring of tiles
    static constexpr size_t b_bytes(int gb) { return (size_t)gb * 4 * TCN * 16; }
    static constexpr size_t qs_off(int gb) { return b_off(gb) + b_bytes(gb); }
    static constexpr size_t sv_off(int gb) { return qs_off(gb) + sizeof(float) * LGT * 16 * gb; }
    static constexpr size_t mask_off(int gb) { return sv_off(gb) + sizeof(Surv) * LNW * QCAP; }
    // the kept-pair masks of a tile (two query halves of 32 bits), one buffer per tile parity with the ring of four
    static constexpr size_t total(int gb) { return mask_off(gb) + (tc_ring(gb) > 2 ? 4 : 2) * sizeof(unsigned) * LTC; }
};

// Shared-memory matrix descriptor without swizzle: start address / 16 (bits
// 0-13), K-direction core-matrix stride / 16 (bits 16-29), M/N-direction
// 8-row group stride / 16 (bits 32-45), the fixed 0b001 at bits 46-48.
__device__ __forceinline__ uint64_t lt_desc(uint32_t addr, uint32_t kstride, uint32_t mstride) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kstride >> 4) << 16) | ((uint64_t)(mstride >> 4) << 32) |
           (1ull << 46);
}
__device__ __forceinline__ void lt_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void lt_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void lt_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void lt_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void lt_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void lt_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 2D TMA load of one box (x = float within the 16-float row, y = row) into shared memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ uint32_t tf32_rna_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// The list of work item `item`: the last c with item_off[c] <= item (warp-wide,
// every lane returns it).  A block takes items in increasing order, so the search
// starts at the list of its previous item (`from`, with item_off[from] <= item):
// one round trip when the item is in one of the next 32 lists, then a 32-way
// search (each step one round trip, the range shrinking 32-fold).
__device__ __forceinline__ int find_list(const int *__restrict__ off, int nc, int item, int from, int lane) {
    {
        const int idx = from + 1 + lane;
        const int cnt = __popc(__ballot_sync(0xffffffffu, idx < nc && __ldg(off + idx) <= item));
        if (cnt < 32) return from + cnt;
    }
    int lo = from + 32, hi = nc;
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int idx = lo + (lane + 1) * step;
        lo += __popc(__ballot_sync(0xffffffffu, idx < hi && __ldg(off + idx) <= item)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

template <int GB, bool STATS>
__global__ void __launch_bounds__(LNT, 2) k_lm_tc(const LmArgs a, const __grid_constant__ CUtensorMap tmap) {
    constexpr int NA = tc_ring(GB);                 // staged tiles
    constexpr int PRE = 2;                          // tiles queued before an item's first MMA
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[NA], mdone[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_item, s_next, s_c, s_q[LGT];
    __shared__ float s_r2[LGT], s_thr[LGT];
    __shared__ float4 s_qc[LGT];   // per query: ||q'||^2, ||q'||, the bound's threshold thr (1 + 2^-15)
    __shared__ unsigned s_any[2][4][2];   // per tile parity, row quarter, query half: queries with a kept row
    unsigned char *abuf = smem;
    unsigned char *bsm = smem + TcSmem::b_off(GB);
    float *qs = reinterpret_cast<float *>(smem + TcSmem::qs_off(GB));
    Surv *survs = reinterpret_cast<Surv *>(smem + TcSmem::sv_off(GB));
    unsigned *mask = reinterpret_cast<unsigned *>(smem + TcSmem::mask_off(GB));   // [parity][half][LTC]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, quad = lane >> 2, lq = lane & 3;
    Surv *queue = survs + warp * QCAP;   // this warp's survivors, drained when full or at the item's end
    int qn = 0;                          // entries queued (the same on every lane of the warp)

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < NA; ++b) mbar_init(su32(&full[b]), 1);
        for (int b = 0; b < 2; ++b) mbar_init(su32(&mdone[b]), 1);
        fence_mbar_init();
        s_item = (int)atomicAdd(a.ctr, 1u);
    }
    lt_fence_before();
    __syncthreads();
    lt_fence_after();
    const uint32_t tmem = tmem_base;
    uint32_t used[NA], mph[2] = {0u, 0u};   // completed waits per staged tile / accumulator
    int inflight[NA];                       // thread 0: copies issued and not waited on
#pragma unroll
    for (int b = 0; b < NA; ++b) {
        used[b] = 0u;
        inflight[b] = 0;
    }
    bool mpend[2] = {false, false};         // thread 0: MMAs committed and not waited on
    bool failed = false;
    const int total = a.item_off[a.nc];
    int c = 0;                              // the list of the previous item

    for (;;) {
        __syncthreads();   // s_item is set; the previous item's shared state is no longer read
        const int item = s_item;
        if (item >= total) break;
        if (tid == 32) s_next = (int)atomicAdd(a.ctr, 1u);   // the next item, fetched while this one runs
        if (warp == 0) {
            const int cl = find_list(a.item_off, a.nc, item, c, lane);
            if (lane == 0) s_c = cl;
        }
        __syncthreads();
        c = s_c;
        const int ngroups = (a.lq_off[c + 1] - a.lq_off[c] + a.lg - 1) / a.lg;
        const int local = item - a.item_off[c];
        const int qb = a.lq_off[c] + (local % ngroups) * a.lg;
        const int ng = min(a.lg, a.lq_off[c + 1] - qb);
        const ListMeta m = a.meta[c];
        const int rend = lm_end(a, m.len);
        const int t0 = (local / ngroups) * a.chunk_tiles;
        const int ntile = min(max(0, (rend - a.row_lo + LTC - 1) / LTC), t0 + a.chunk_tiles);
        const int64_t brow = m.base >> 4;   // row (16 floats) of block 0, member 0 of list c
        auto issue = [&](int t) {   // thread 0: the tile's FP32 rows, GB blocks x 4 boxes
            const int buf = t % NA, i0 = a.row_lo + t * LTC;
            const uint32_t bar = su32(&full[buf]);
            mbar_expect_tx(bar, (uint32_t)(GB * 4 * LTC * 16));
            unsigned char *dst = abuf + (size_t)buf * TcSmem::a_bytes(GB);
            for (int b = 0; b < GB; ++b)
                for (int kc = 0; kc < 4; ++kc)
                    tma_load_2d(su32(dst + (size_t)(b * 4 + kc) * LTC * 16), &tmap, kc * 4,
                                (int)(brow + (int64_t)b * m.np + i0), bar);
            ++inflight[buf];
        };
        auto mma = [&](int t) -> bool {   // thread 0: wait for tile t's rows, then its MMAs
            const int buf = t % NA;
            if (a.never != nullptr && (used[0] | used[1]) == 0 && !wait_word(a.never, a.wait_ns)) return false;
            if (!wait_bounded(su32(&full[buf]), used[buf] & 1u, a.wait_ns)) return false;
            ++used[buf];
            --inflight[buf];
            lt_fence_after();
            const uint32_t ab = su32(abuf + (size_t)buf * TcSmem::a_bytes(GB)), bb = su32(bsm);
            const uint32_t d = tmem + (uint32_t)((t & 1) * TCN);
#pragma unroll
            for (int b = 0; b < GB; ++b)
#pragma unroll
                for (int s2 = 0; s2 < 2; ++s2)
                    lt_mma(d, lt_desc(ab + (uint32_t)((b * 4 + 2 * s2) * LTC * 16), LTC * 16, 128),
                           lt_desc(bb + (uint32_t)((b * 4 + 2 * s2) * TCN * 16), TCN * 16, 128),
                           (b > 0 || s2 > 0) ? 1u : 0u);
            lt_commit(su32(&mdone[t & 1]));
            mpend[t & 1] = true;
            return true;
        };
        if (tid == 0)
            for (int t = t0; t < t0 + PRE && t < ntile; ++t) issue(t);
        for (int g = tid; g < LGT; g += LNT) {
            const bool in = g < ng;
            const int q = in ? a.lq_items[qb + g] : 0;
            const float r2 = in ? a.r2src[(int64_t)q * a.k + lm_kq(a, q) - 1] : 0.f;
            const float thr = a.coef[0] * r2;
            s_q[g] = q;
            s_r2[g] = r2;
            s_thr[g] = thr;
            s_qc[g].z = thr * (1.f + 0x1p-15f);
        }
        // the queries' first increment: FP32 for the FP32 path, rounded to TF32 for the MMA
        // (B row g, K-major core matrices of 8 rows x 4 floats)
        for (int e = tid; e < LGT * 16 * GB; e += LNT) {
            const int g = e / (16 * GB), kk = e % (16 * GB);
            const bool in = g < ng && kk < a.d;
            const float qv = in ? a.q_rot[(int64_t)a.lq_items[qb + g] * a.q_stride + kk] : 0.f;
            qs[e] = qv;
            const int b = kk >> 4, kc = (kk >> 2) & 3, el = kk & 3;
            reinterpret_cast<uint32_t *>(bsm + ((size_t)(b * 4 + kc) * TCN + g) * 16)[el] = tf32_rna_bits(qv);
        }
        __syncthreads();
        for (int g = warp; g < LGT; g += LNW) {   // ||q'||^2 over the increment
            float acc = 0.f;
            for (int kk = lane; kk < 16 * GB; kk += 32) acc = fmaf(qs[g * 16 * GB + kk], qs[g * 16 * GB + kk], acc);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) {
                s_qc[g].x = acc;
                s_qc[g].y = sqrtf(acc);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B, written by threads, read by the MMA
        __syncthreads();
        if (tid == 0 && t0 < ntile && !mma(t0)) failed = true;

        // Tile t's epilogue (every warp): candidate mrow against the queries of half qh,
        // from accumulator t & 1; the kept pairs as bits of the tile's masks.
        auto epilogue = [&](int t) {
            const int i0 = a.row_lo + t * LTC, tn = min(LTC, rend - i0);
            const float *af = reinterpret_cast<const float *>(abuf + (size_t)(t % NA) * TcSmem::a_bytes(GB));
            unsigned *mk_t = mask + (NA > 2 ? (t & 1) : 0) * 2 * LTC;
            // warp half qh takes the item's queries 16 qh + j and 32 + 16 qh + j (bits j and
            // 16 + j of its masks), the second block only when the item has more than 32
            const int mrow = 32 * (warp & 3) + lane, qh = warp >> 2;
            const int nblk = ng > 32 ? 2 : 1;   // uniform over the block
            unsigned bits = 0u;
            uint32_t dv[32];
            const uint32_t tb = tmem + (uint32_t)((t & 1) * TCN) + ((uint32_t)(32 * (warp & 3)) << 16);
            lt_ld16(tb + (uint32_t)(qh * 16), *reinterpret_cast<uint32_t(*)[16]>(dv));
            if (nblk == 2) lt_ld16(tb + (uint32_t)(32 + qh * 16), *reinterpret_cast<uint32_t(*)[16]>(dv + 16));
            if (mrow < tn) {
                float on = 0.f;   // ||o'||^2 over the increment, from the staged rows
#pragma unroll
                for (int b = 0; b < GB; ++b)
#pragma unroll
                    for (int kc = 0; kc < 4; ++kc) {
                        const float4 v = *reinterpret_cast<const float4 *>(af + ((size_t)(b * 4 + kc) * LTC + mrow) * 4);
                        on = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, on))));
                    }
                const float ocn = sqrtf(on);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    if (j >= 16 * nblk) break;
                    const int g = (j < 16 ? 0 : 32 - 16) + qh * 16 + j;
                    const float dot = __uint_as_float(dv[j]);
                    const float4 qc = s_qc[g];
                    const float sq = qc.x + on;
                    const float pt = fmaf(-2.f, dot, sq);
                    const float err = fmaf(a.tc_c1, sq, a.tc_c2 * (qc.y * ocn));
                    const bool drop = pt - err > qc.z;
                    bits |= (unsigned)(g < ng && !drop) << j;
                }
            }
            mk_t[qh * LTC + mrow] = bits;
            const unsigned any = __reduce_or_sync(0xffffffffu, bits);   // the warp's 32 rows
            if (lane == 0) s_any[NA > 2 ? (t & 1) : 0][warp & 3][qh] = any;
        };
        // Tile t's kept pairs (warp per query): the FP32 first increment from the staged
        // rows, and the survivors of its test to the warp's queue.
        auto recheck = [&](int t) {
            const int i0 = a.row_lo + t * LTC, tn = min(LTC, rend - i0);
            const float *af = reinterpret_cast<const float *>(abuf + (size_t)(t % NA) * TcSmem::a_bytes(GB));
            const unsigned *mk_t = mask + (NA > 2 ? (t & 1) : 0) * 2 * LTC;
            for (int g = warp; g < ng; g += LNW) {
                if (qn + LTC > QCAP) {
                    lm_drain<GB, STATS, false, LGT / LNW>(a, m, queue, qn, s_q, s_r2, s_thr, qs, nullptr);
                    qn = 0;
                    __syncwarp();
                }
                const int gg = g & 31, qh = gg >> 4, jb = (gg & 15) + (g >= 32 ? 16 : 0);
                Surv *cand_list = queue + qn;   // kept candidates, compacted in place into survivors
                int nk = 0;
                for (int m0 = 0; m0 < tn; m0 += 32) {
                    if (!((s_any[NA > 2 ? (t & 1) : 0][m0 >> 5][qh] >> jb) & 1u)) continue;   // nothing kept
                    const int mm = m0 + lane;
                    const bool keep = mm < tn && ((mk_t[qh * LTC + mm] >> jb) & 1u);
                    const unsigned mk = __ballot_sync(0xffffffffu, keep);
                    if (keep) cand_list[nk + __popc(mk & ((1u << lane) - 1u))] = Surv{mm, 0.f};
                    nk += __popc(mk);
                }
                __syncwarp();
                float4 qa[GB];
#pragma unroll
                for (int b = 0; b < GB; ++b)
                    qa[b] = *reinterpret_cast<const float4 *>(qs + g * 16 * GB + b * 16 + lq * 4);
                const float c0 = s_thr[g];
                int ns = 0;
                for (int r0 = 0; r0 < nk; r0 += 8) {   // the FP32 partial, as the plain kernels sum it
                    const int sidx = r0 + quad;
                    const bool act = sidx < nk;
                    const int cand = act ? cand_list[sidx].idx : 0;
                    float p = 0.f;
                    if (act) {
#pragma unroll
                        for (int b = 0; b < GB; ++b)
                            p += sqd4(qa[b], *reinterpret_cast<const float4 *>(af + ((size_t)(b * 4 + lq) * LTC + cand) * 4));
                    }
                    p = quad_sum4(p);
                    const bool lead = act && lq == 0;
                    const bool keep = lead && !(p > c0);
                    __syncwarp();   // every lane has read its entry before the list is compacted in place
                    const unsigned mk = __ballot_sync(0xffffffffu, keep);
                    if (keep) cand_list[ns + __popc(mk & ((1u << lane) - 1u))] = Surv{surv_key(g, i0 + cand), p};
                    ns += __popc(mk);
                }
                qn += ns;
                if (lane == 0) {
                    const int q = s_q[g];
                    const unsigned long long pruned = (unsigned long long)(tn - ns);
                    if (STATS) {   // every candidate the tile tested; pruned at the first test
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 0]),
                                  (unsigned long long)tn);
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 1]),
                                  pruned * (unsigned long long)min(GB * 16, a.d));
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[(int64_t)q * 4 + 3]), pruned);
                    }
                    if (a.lead_stats && tn > nk)
                        atomicAdd(reinterpret_cast<unsigned long long *>(&a.lead_stats[q]), (unsigned long long)(tn - nk));
                }
                __syncwarp();
            }
        };
        // thread 0: tile t's MMAs done (bounded); the block meets (false: every thread leaves)
        auto tile_ready = [&](int t) -> bool {
            bool ok = !failed;
            if (tid == 0 && ok) {
                ok = wait_bounded(su32(&mdone[t & 1]), mph[t & 1] & 1u, a.wait_ns);
                if (ok) {
                    ++mph[t & 1];
                    mpend[t & 1] = false;
                }
            }
            return !__syncthreads_or(!ok);
        };

        if constexpr (NA > 2) {
            // Ring of four, one block barrier per tile.  Iteration t: tile t's MMAs done and
            // the block met, so every warp is past tile t - 1's epilogue and tile t - 2's
            // FP32 pass; thread 0 then queues tile t + 1's MMAs into accumulator (t + 1) & 1
            // (tile t - 1's, read) and tile t + 2's rows into tile t - 2's slot; the warps
            // read tile t's accumulator into its masks (a buffer per tile parity) and run the
            // FP32 pass of tile t - 1, whose rows and masks nothing touches before the next
            // meeting.  Tile t's slot holds its rows through tile t + 1's pass.
            for (int t = t0; t < ntile; ++t) {
                if (!tile_ready(t)) {
                    failed = true;
                    break;
                }
                if (tid == 0) {
                    if (t + 1 < ntile && !mma(t + 1)) failed = true;   // the next meeting reports it
                    if (t + 2 < ntile) issue(t + 2);
                }
                lt_fence_after();
                epilogue(t);
                lt_fence_before();
                if (t > t0) recheck(t - 1);
            }
            if (!failed && t0 < ntile) {
                __syncthreads();   // the last tile's masks
                recheck(ntile - 1);
            }
        } else {
            // Ring of two: tile t + 1's MMAs queued, tile t's waited for, the block meets;
            // the epilogue, a second barrier, the FP32 pass; a third barrier frees tile t's
            // slot, the masks and accumulator t & 1 for tile t + 2.
            for (int t = t0; t < ntile; ++t) {
                if (tid == 0 && !failed && t + 1 < ntile && !mma(t + 1)) failed = true;   // overlaps this tile's reads
                if (!tile_ready(t)) {
                    failed = true;
                    break;
                }
                lt_fence_after();
                epilogue(t);
                lt_fence_before();
                __syncthreads();
                recheck(t);
                __syncthreads();
                if (tid == 0 && t + 2 < ntile) issue(t + 2);
            }
        }
        if (failed) break;
        __syncwarp();
        lm_drain<GB, STATS, false, LGT / LNW>(a, m, queue, qn, s_q, s_r2, s_thr, qs, nullptr);
        qn = 0;
        __syncwarp();
        if (tid == 32) s_item = s_next;
    }
    if (failed && tid == 0) {   // let the copies and MMAs in flight finish (bounded) before leaving
        atomicExch(a.err, (int)DADE_ETIMEOUT);
        for (int b = 0; b < NA; ++b)
            if (inflight[b] > 0) wait_bounded(su32(&full[b]), used[b] & 1u, 10000000ull);
        for (int b = 0; b < 2; ++b)
            if (mpend[b]) wait_bounded(su32(&mdone[b]), mph[b] & 1u, 10000000ull);
    }
    lt_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
}

// ---- work list -------------------------------------------------------------------
// (query, list) pairs of probe positions [c0, c1) (probe rows of nprobe).
__global__ void k_lm_count(const int32_t *__restrict__ probe, int64_t nq, int nprobe, int c0, int c1,
                           const int32_t *__restrict__ q_np, int *__restrict__ cnt) {
    const int64_t total = nq * (int64_t)(c1 - c0);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / (c1 - c0);
        const int j = c0 + (int)(e % (c1 - c0));
        if (q_np && j >= q_np[q]) continue;   // past this query's own nprobe
        atomicAdd(&cnt[probe[q * nprobe + j]], 1);
    }
}

// items[c] = ceil(cnt[c] / lg) query groups x ceil(tiles of c in the row
// window / chunk_tiles) chunks (none when the window holds no row of c);
// both arrays get a trailing 0 for the scans.  off is written only when
// `with_off` (the query groups do not change between the rounds of a pass).
__global__ void k_lm_items(const int *__restrict__ cnt, const ListMeta *__restrict__ meta, int nc, int chunk_tiles,
                           int tile_rows, int lg, int row_lo, int row_hi, int with_off, int *__restrict__ off,
                           int *__restrict__ items) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= nc; c += gridDim.x * blockDim.x) {
        const int v = c < nc ? cnt[c] : 0;
        if (with_off) off[c] = v;
        const int rows = c < nc ? min(meta[c].len, row_hi) - row_lo : 0;
        const int tiles = rows > 0 ? (rows + tile_rows - 1) / tile_rows : 0;
        items[c] = (v > 0 && tiles > 0) ? ((v + lg - 1) / lg) * ((tiles + chunk_tiles - 1) / chunk_tiles) : 0;
    }
}

__global__ void k_lm_scatter(const int32_t *__restrict__ probe, int64_t nq, int nprobe, int c0, int c1,
                             const int32_t *__restrict__ q_np, int *__restrict__ fill, int32_t *__restrict__ lq_items) {
    const int64_t total = nq * (int64_t)(c1 - c0);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e / (c1 - c0);
        const int j = c0 + (int)(e % (c1 - c0));
        if (q_np && j >= q_np[q]) continue;
        lq_items[atomicAdd(&fill[probe[q * nprobe + j]], 1)] = (int32_t)q;
    }
}

// An empty K-nearest state: ids -1, distances +inf (the threshold of a first round).
__global__ void k_lm_reset(int64_t *__restrict__ ids, float *__restrict__ dists, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        ids[e] = -1;
        dists[e] = INFINITY;
    }
}

// ---- final merge: the K smallest keys of the first-phase result and the
// query's accepted keys.  Keys are unique (ids are), so a radix select on the
// 64-bit key finds the K-th smallest exactly; the keys at most it are then
// rank-sorted.  One CTA per query.
constexpr int MT = 256;

__global__ void __launch_bounds__(MT) k_lm_merge(int64_t *__restrict__ ids, float *__restrict__ dists, int k,
                                                 const unsigned long long *__restrict__ acc,
                                                 const int *__restrict__ acnt, int64_t cap,
                                                 const int32_t *__restrict__ q_k) {
    __shared__ unsigned long long s1[DADE_MAX_K], sel[DADE_MAX_K];
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ unsigned s_rank, s_cnt;
    __shared__ int s_n1;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t q = blockIdx.x;
    if (acnt[q] == 0) return;   // nothing accepted in this pass: the row is already the K nearest, sorted
    const int kq = q_k ? min(max(q_k[q], 1), k) : k;   // this query's K; rows have k entries
    if (tid == 0) s_n1 = 0;
    __syncthreads();
    for (int j = tid; j < k; j += MT) {   // first-phase results: a sorted prefix of valid entries
        const int64_t id = ids[q * k + j];
        if (id >= 0) {
            s1[j] = ((unsigned long long)__float_as_uint(dists[q * k + j]) << 32) | (unsigned)id;
            atomicAdd(&s_n1, 1);
        }
    }
    __syncthreads();
    const int n1 = s_n1, n2 = (int)min((int64_t)acnt[q], cap), n = n1 + n2;
    const unsigned long long *a2 = acc + q * cap;
    auto key = [&](int j) { return j < n1 ? s1[j] : a2[j - n1]; };
    unsigned long long bound = ~0ull;   // select every key when n <= kq
    if (n > kq) {
        unsigned long long prefix = 0, mask = 0;
        unsigned rank = (unsigned)kq;
        for (int pass = 0; pass < 8; ++pass) {
            const int shift = 56 - 8 * pass;
            hist[tid] = 0;
            __syncthreads();
            for (int j0 = 0; j0 < n; j0 += MT) {
                const int j = j0 + tid;
                const unsigned long long kk = j < n ? key(j) : 0ull;
                const bool in = j < n && (kk & mask) == prefix;
                const unsigned bin = in ? (unsigned)((kk >> shift) & 255u) : 256u;
                const unsigned peers = __match_any_sync(0xffffffffu, bin);
                if (in && lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (unsigned)__popc(peers));
            }
            __syncthreads();
            if (tid < 32) {
                unsigned loc[8], s = 0;
#pragma unroll
                for (int t = 0; t < 8; ++t) { loc[t] = hist[lane * 8 + t]; s += loc[t]; }
                unsigned inc = s;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned v = __shfl_up_sync(0xffffffffu, inc, off);
                    if (lane >= off) inc += v;
                }
                const unsigned before = inc - s;
                if (before < rank && inc >= rank) {
                    unsigned cc = before;
                    int t = 0;
                    while (cc + loc[t] < rank) { cc += loc[t]; ++t; }
                    s_prefix = prefix | ((unsigned long long)(lane * 8 + t) << shift);
                    s_rank = rank - cc;
                }
            }
            __syncthreads();
            prefix = s_prefix;
            rank = s_rank;
            mask |= 255ull << shift;
            __syncthreads();
        }
        bound = prefix;   // the k-th smallest key
    }
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    for (int j = tid; j < n; j += MT) {
        const unsigned long long kk = key(j);
        if (kk <= bound) {
            const unsigned slot = atomicAdd(&s_cnt, 1u);
            if (slot < (unsigned)kq) sel[slot] = kk;
        }
    }
    __syncthreads();
    const int m = min((int)s_cnt, kq);
    for (int t = tid; t < k; t += MT) {
        if (t < m) {
            const unsigned long long kk = sel[t];
            int r = 0;
            for (int u = 0; u < m; ++u) r += sel[u] < kk;
            ids[q * k + r] = (int64_t)(unsigned)(kk & 0xffffffffu);
            dists[q * k + r] = __uint_as_float((unsigned)(kk >> 32));
        } else {
            ids[q * k + t] = -1;
            dists[q * k + t] = INFINITY;
        }
    }
}

int grid_of(int64_t work, int threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 152 * 16));
}

template <int GB, bool STATS>
dade_status launch_lm(const LmArgs &a, cudaStream_t s) {
    const size_t smem = LmSmem::total(GB);
    int blocks = 1;
    DADE_TRY(resident_blocks((const void *)k_lm<GB, STATS>, LNT, smem, &blocks));
    k_lm<GB, STATS><<<blocks, LNT, smem, s>>>(a);
    return launch_check("k_lm");
}

template <int GB, bool STATS>
dade_status launch_lm_g(const LmArgs &a, cudaStream_t s) {
    const size_t smem = LmSmem::total_g(GB);
    int blocks = 1;
    DADE_TRY(resident_blocks((const void *)k_lm_g<GB, STATS>, LNT, smem, &blocks));
    k_lm_g<GB, STATS><<<blocks, LNT, smem, s>>>(a);
    return launch_check("k_lm_g");
}

template <int GB, bool STATS>
dade_status launch_lm_tc(const LmArgs &a, const CUtensorMap &tmap, cudaStream_t s) {
    const size_t smem = TcSmem::total(GB);
    int blocks = 1, dev = 0, sms = 0;
    DADE_TRY(resident_blocks((const void *)k_lm_tc<GB, STATS>, LNT, smem, &blocks));
    DADE_TRY_CUDA(cudaGetDevice(&dev));
    DADE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the kernel is sized for two blocks per SM (registers and shared memory; two
    // accumulators of 128 tensor-memory columns each); the occupancy query answers one
    // for it, so launch at least two per SM: a persistent block beyond what fits only
    // starts when another leaves and then finds the work counter exhausted
    blocks = std::max(blocks, 2 * sms);
    k_lm_tc<GB, STATS><<<blocks, LNT, smem, s>>>(a, tmap);
    return launch_check("k_lm_tc");
}

template <bool STATS>
dade_status launch_lm_tc_gb(const LmArgs &a, const CUtensorMap &tmap, int gb, cudaStream_t s) {
    switch (gb) {
    case 1: return launch_lm_tc<1, STATS>(a, tmap, s);
    case 2: return launch_lm_tc<2, STATS>(a, tmap, s);
    default: return launch_lm_tc<4, STATS>(a, tmap, s);
    }
}

template <bool STATS>
dade_status launch_lm_gen(const LmArgs &a, int gb, cudaStream_t s) {
    switch (gb) {
    case 1: return launch_lm_g<1, STATS>(a, s);
    case 2: return launch_lm_g<2, STATS>(a, s);
    case 4: return launch_lm_g<4, STATS>(a, s);
    default: return launch_lm_g<8, STATS>(a, s);
    }
}

template <bool STATS>
dade_status launch_lm_gb(const LmArgs &a, int gb, cudaStream_t s) {
    switch (gb) {
    case 1: return launch_lm<1, STATS>(a, s);
    case 2: return launch_lm<2, STATS>(a, s);
    case 4: return launch_lm<4, STATS>(a, s);
    default: return launch_lm<8, STATS>(a, s);
    }
}

} // namespace

// The tensor-core prefilter runs a list-major DADE pass when the search asks
// for it, the first increment is 1, 2 or 4 blocks and not the last one, and
// the list-major kernels apply (D > 112).
bool tc_applies(const dade_index *ix, const ScanParams &p, int gb) {
    return p.use_tc && p.mode == DADE_MODE_DADE && ix->data_tmap_ok && (gb == 1 || gb == 2 || gb == 4) &&
           ix->nb > gb && ix->nb >= LNB;
}

// Error bound of the expanded partial distance of k_lm_tc over K = 16 gb dims,
// E = c1 (||q'||^2 + ||o'||^2) + c2 ||q'|| ||o'|| (FP32 rows q', o'), u = 2^-24:
//   - the FP32 sums ||q'||^2 (lane-strided FMAs and an xor tree), ||o'||^2
//     (one FMA chain of K terms) and s = ||q'||^2 + ||o'||^2: relative
//     (K + 8) u together, with the rounding of s - 2 dot: c1;
//   - the tensor core reads each row value o as TF32 (at most 2^-10 relative
//     off, truncated or rounded), the query is rounded to TF32 (2^-11
//     relative), products of TF32 values are exact in FP32, and the K
//     products of a column are accumulated in FP32: allowed 4 x 2u per
//     addition (truncating adds with a factor 4 to spare), K + 2 of them:
//     |dot - q'.o'| <= (2^-10 + 2^-11 + (K + 2) 2^-21) sum |q'_k||o'_k|,
//     at most that times ||q'|| ||o'||; twice it for -2 dot: c2.
// Both are rounded up and carry a further 2^-20 for their own FP32 evaluation.
void tc_constants(int gb, float *c1, float *c2) {
    const double u = std::ldexp(1.0, -24), K = 16.0 * gb;
    const double cs = (K + 8.0) * u * 1.01 + 3.0 * u;
    const double cd = std::ldexp(1.0, -10) + std::ldexp(1.0, -11) + (K + 2.0) * std::ldexp(1.0, -21);
    const double grow = 1.0 + std::ldexp(1.0, -20);
    *c1 = std::nextafter((float)(cs * grow), INFINITY);
    *c2 = std::nextafter((float)(2.0 * cd * (1.0 + std::ldexp(1.0, -10)) * grow), INFINITY);
}

// One list-major round: the lists at probe positions [c0, c1) of every query,
// each candidate tested against the query's r^2 = dists[q][k - 1] as it is
// when the round starts (frozen for the round), then the K nearest of the
// previous result and the round's accepted candidates.  gb = 8 with no
// pruning (coef +inf) is FDScanning.
// Accept-buffer entries per query for a pass over `lists` probe positions:
// every candidate (lists x longest list) up to 65,536; a pass that accepts
// more for one query (r = +inf over very long lists) reports DADE_ENOMEM.
int64_t accept_cap(const dade_index *ix, int lists) {
    return std::min<int64_t>((int64_t)lists * std::max(ix->max_list, 1), 1 << 16);
}

// rows [row_lo, min(len, row_hi)) of every list (the row-rounds schedule);
// `lists` = false reuses the (list, query) groups of the previous call with
// the same probe positions and rebuilds only the work items of the window.
dade_status lm_round(const dade_index *ix, int64_t nq, const ScanParams &p, int c0, int c1, int gb, bool prune,
                     cudaStream_t s, int row_lo = 0, int row_hi = INT_MAX, bool lists = true) {
    const int nc = ix->nc, np = p.nprobe;
    const int64_t pairs = nq * (int64_t)(c1 - c0);
    Workspace &w = ws(ix);
    DADE_TRY(w.lm_cnt.ensure(sizeof(int) * (size_t)(nc + 1) * 4));
    int *cnt = w.lm_cnt.as<int>(), *off = cnt + (nc + 1), *items = off + (nc + 1), *fill = items + (nc + 1);
    DADE_TRY(w.lm_items.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(pairs, 1) + 16));
    int32_t *lq_items = w.lm_items.as<int32_t>();
    unsigned *ctr = reinterpret_cast<unsigned *>(lq_items + std::max<int64_t>(pairs, 1));
    const int64_t cap = accept_cap(ix, c1 - c0);
    DADE_TRY(w.lm_acc.ensure(sizeof(unsigned long long) * (size_t)(nq * cap)));
    DADE_TRY(w.lm_acnt.ensure(sizeof(int) * (size_t)nq));
    if (lists) DADE_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(nc + 1), s));
    DADE_TRY_CUDA(cudaMemsetAsync(w.lm_acnt.p, 0, sizeof(int) * (size_t)nq, s));
    DADE_TRY_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned), s));
    if (lists) {
        k_lm_count<<<grid_of(pairs, 256), 256, 0, s>>>(p.probe, nq, np, c0, c1, p.q_np, cnt);
        DADE_TRY(launch_check("k_lm_count"));
    }
    // the tensor-core bound needs a finite threshold: not in a first round (r = +inf)
    // and, in the row rounds, only for windows of at least tc_min_rows rows
    const bool tc = prune && tc_applies(ix, p, gb) && !(row_lo == 0 && c0 == 0 && p.schedule == DADE_SCHED_ROUNDS) &&
                    (p.schedule != DADE_SCHED_ROUNDS || (int64_t)row_hi - row_lo >= p.tc_min_rows);
    const int tile_rows = tc ? LTC : LT;
    const int chunk_tiles = std::max(1, (p.list_chunk > 0 ? p.list_chunk : 4096) / tile_rows);
    // queries per work item: the tensor-core kernel takes 64 where the window spans at least 32
    // work items of a list (only long lists reach it, with many queries each, and items stay
    // plentiful), 32 elsewhere
    const int lg = tc && (int64_t)row_hi - row_lo >= 32ll * chunk_tiles * tile_rows ? LGT : LG;
    k_lm_items<<<grid_of(nc + 1, 256), 256, 0, s>>>(cnt, ix->meta.as<ListMeta>(), nc, chunk_tiles, tile_rows,
                                                    lg, row_lo, row_hi, lists ? 1 : 0, off, items);
    DADE_TRY(launch_check("k_lm_items"));
    if (lists) DADE_TRY(exclusive_scan_int(off, nc + 1, s));
    DADE_TRY(exclusive_scan_int(items, nc + 1, s));
    if (lists) {
        DADE_TRY_CUDA(cudaMemcpyAsync(fill, off, sizeof(int) * (size_t)(nc + 1), cudaMemcpyDeviceToDevice, s));
        k_lm_scatter<<<grid_of(pairs, 256), 256, 0, s>>>(p.probe, nq, np, c0, c1, p.q_np, fill, lq_items);
        DADE_TRY(launch_check("k_lm_scatter"));
    }
    LmArgs a{};
    a.data = ix->data.as<float>();
    a.ids = ix->ids.as<int32_t>();
    a.meta = ix->meta.as<ListMeta>();
    a.q_rot = p.q_rot;
    a.lq_items = lq_items;
    a.lq_off = off;
    a.item_off = items;
    a.ctr = ctr;
    a.r2src = p.dists;
    a.q_k = p.q_k;
    a.acc = w.lm_acc.as<unsigned long long>();
    a.acnt = w.lm_acnt.as<int>();
    a.stats = p.stats;
    a.err = ix->errflag.as<int>();
    a.cap = cap;
    a.q_stride = p.q_stride;
    a.chunk_tiles = chunk_tiles;
    a.lg = lg;
    a.row_lo = row_lo;
    a.row_hi = row_hi;
    a.wait_ns = p.wait_ns > 0 ? (uint64_t)p.wait_ns : WAIT_NS;
    a.never = p.check_timeout ? ix->errflag.as<int>() + 3 : nullptr;
    a.nc = nc;
    a.k = p.k;
    a.d = ix->d;
    if (p.use_tail && ix->tail_nb0 > 0) {
        a.tail = ix->tail.as<float>();
        a.tail_nb0 = ix->tail_nb0;
        a.tail_w = ix->tail_w;
    }
    const int n_inc = (ix->nb + gb - 1) / gb;
    a.nb = ix->nb;
    a.n_inc = n_inc;
    for (int j = 0; j < DADE_MAX_DIM / DADE_BLOCK; ++j) a.coef[j] = (prune && j < n_inc - 1) ? p.coef[j] : INFINITY;
    if (tc) {
        a.lead_stats = p.lead_stats;
        tc_constants(gb, &a.tc_c1, &a.tc_c2);
        DADE_TRY(p.stats ? launch_lm_tc_gb<true>(a, ix->data_tmap, gb, s)
                         : launch_lm_tc_gb<false>(a, ix->data_tmap, gb, s));
    } else if (ix->nb == LNB)
        DADE_TRY(p.stats ? launch_lm_gb<true>(a, gb, s) : launch_lm_gb<false>(a, gb, s));
    else
        DADE_TRY(p.stats ? launch_lm_gen<true>(a, gb, s) : launch_lm_gen<false>(a, gb, s));
    k_lm_merge<<<(unsigned)nq, MT, 0, s>>>(p.ids, p.dists, p.k, a.acc, a.acnt, cap, p.q_k);
    return launch_check("k_lm_merge");
}

// The seeded schedule with the lists after the seeds run query-major.  The
// first S lists: in the tile schedule, straight into the outputs; or, with
// whole-list tiles, as S threshold epochs (list j of every query tested
// against r after lists 0..j-1, r = +inf for list 0).  Then every query's
// later lists, with r frozen at the K-th distance after the seeds.  Wherever
// r is frozen the candidates are independent, so those passes run the tile
// kernel in split mode: each query's lists cut into parts over several CTAs
// (enough for about eight waves), each appending what it accepts to the
// query's buffer, then one merge into the K best.  The execution tile there
// does not change the results (128 rows for whole-list epochs).
static dade_status seeded_split(const dade_index *ix, int64_t nq, const ScanParams &p, cudaStream_t s) {
    const int S = p.seed_lists, np = p.nprobe, late = np - S;
    const bool whole = p.tile >= ix->max_list;
    Workspace &w = ws(ix);
    const int64_t cap = accept_cap(ix, late);
    DADE_TRY(w.lm_acc.ensure(sizeof(unsigned long long) * (size_t)(nq * cap)));
    DADE_TRY(w.lm_acnt.ensure(sizeof(int) * (size_t)nq));
    int dev = 0, sms = 0;
    DADE_TRY_CUDA(cudaGetDevice(&dev));
    DADE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t slots = (int64_t)sms * (768 / (p.threads == 256 ? 256 : 128));
    ScanParams base = p;
    base.schedule = DADE_SCHED_TILE;
    base.seed_split = 0;
    base.pstride = np;
    if (whole) base.tile = 128;
    base.r2src = p.dists;
    base.acc = w.lm_acc.as<unsigned long long>();
    base.acnt = w.lm_acnt.as<int>();
    base.cap = cap;
    auto frozen_pass = [&](int c0, int n, int parts) -> dade_status {
        DADE_TRY_CUDA(cudaMemsetAsync(w.lm_acnt.p, 0, sizeof(int) * (size_t)nq, s));
        ScanParams q = base;
        q.c0 = c0;
        q.nprobe = n;
        q.parts = parts;
        DADE_TRY(scan(ix, nq, q, s));
        k_lm_merge<<<(unsigned)nq, MT, 0, s>>>(p.ids, p.dists, p.k, base.acc, base.acnt, cap, nullptr);
        return launch_check("k_lm_merge");
    };
    if (whole) {
        k_lm_reset<<<grid_of(nq * (int64_t)p.k, 256), 256, 0, s>>>(p.ids, p.dists, nq * (int64_t)p.k);
        DADE_TRY(launch_check("k_lm_reset"));
        if (p.stats) DADE_TRY_CUDA(cudaMemsetAsync(p.stats, 0, sizeof(int64_t) * 4 * (size_t)nq, s));
        if (p.lead_stats) DADE_TRY_CUDA(cudaMemsetAsync(p.lead_stats, 0, sizeof(int64_t) * (size_t)nq, s));
        for (int j = 0; j < S; ++j) DADE_TRY(frozen_pass(j, 1, 1));
    } else {
        ScanParams p1 = p;
        p1.nprobe = S;
        p1.pstride = np;
        p1.schedule = DADE_SCHED_TILE;
        p1.seed_split = 0;
        DADE_TRY(scan(ix, nq, p1, s));
    }
    return frozen_pass(S, late, (int)std::min<int64_t>(late, std::max<int64_t>(1, (8 * slots + nq - 1) / nq)));
}

// The seeded schedule for queries [0, nq) of p (see the file comment).  When
// the tile holds every list (tile >= longest list), each of the first S lists
// is one threshold epoch: list j of every query is tested against r after
// lists 0..j-1.  Those lists then run list-major too, as S rounds: round 0
// with r = +inf (every candidate exact, so FDScanning), round j against r
// after round j - 1.  Otherwise the first S lists run in the tile schedule.
dade_status scan_seeded(const dade_index *ix, int64_t nq, const ScanParams &p, cudaStream_t s) {
    if (nq == 0) return DADE_OK;
    const int S = p.seed_lists;
    const int np = p.nprobe;
    const bool fd = p.mode == DADE_MODE_FD;
    const int gb = fd ? LNB : std::min(p.delta_d / 16, ix->nb);
    const bool whole = p.tile >= ix->max_list;
    const bool ok = (ix->nb == LNB ? (gb == 1 || gb == 2 || gb == 4 || gb == 8)
                                   : (ix->nb > LNB && (gb == 1 || gb == 2 || gb == 4 || gb == 8))) &&
                    ix->max_list < (1 << QROW_BITS);
    // the list-major kernels cover D > 112 with delta_d of 1, 2, 4 or 8 blocks; elsewhere
    // the passes with r frozen run query-major (the same tests, thresholds and results)
    if (p.seed_split || !ok) return seeded_split(ix, nq, p, s);
    if (whole) {
        k_lm_reset<<<grid_of(nq * (int64_t)p.k, 256), 256, 0, s>>>(p.ids, p.dists, nq * (int64_t)p.k);
        DADE_TRY(launch_check("k_lm_reset"));
        if (p.stats) DADE_TRY_CUDA(cudaMemsetAsync(p.stats, 0, sizeof(int64_t) * 4 * (size_t)nq, s));
        DADE_TRY(lm_round(ix, nq, p, 0, 1, std::min(LNB, ix->nb), false, s));   // r = +inf: exact
        for (int j = 1; j < S; ++j) DADE_TRY(lm_round(ix, nq, p, j, j + 1, gb, !fd, s));
    } else {
        ScanParams p1 = p;   // the first S lists, tile schedule, straight into the outputs
        p1.nprobe = S;
        p1.pstride = np;
        p1.schedule = DADE_SCHED_TILE;
        DADE_TRY(scan(ix, nq, p1, s));
    }
    return lm_round(ix, nq, p, S, np, gb, !fd, s);
}

// TMA view of the packed FP32 data: rows of 16 floats (64 B), row base_c / 16
// + b np_c + i for block b of member i of list c; boxes of 4 floats x 128 rows
// land in shared memory as 128 contiguous 16-byte rows (core matrices of the
// MMA's K-major layout without swizzle).
dade_status make_data_tmap(dade_index *ix) {
    ix->data_tmap_ok = false;
    if (!ix->data.p || ix->data_floats == 0) return DADE_OK;
    typedef CUresult (*encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static encode_fn encode = nullptr;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!encode) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q{};
            DADE_TRY_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
            if (q != cudaDriverEntryPointSuccess || !fn) {
                set_error("cuTensorMapEncodeTiled is not available from the driver");
                return DADE_ECUDA;
            }
            encode = reinterpret_cast<encode_fn>(fn);
        }
    }
    const uint64_t rows = (uint64_t)ix->data_floats / 16;
    if (rows >= (1ull << 31)) return DADE_OK;   // beyond the kernels' 32-bit row coordinates: no prefilter
    const cuuint64_t dims[2] = {16, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {64};   // bytes between rows
    const cuuint32_t box[2] = {4, (cuuint32_t)LTC};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&ix->data_tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ix->data.p, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed for the packed data (CUresult " + std::to_string((int)r) + ")");
        return DADE_ECUDA;
    }
    ix->data_tmap_ok = true;
    return DADE_OK;
}

// The row-rounds schedule (DADE_SCHED_ROUNDS): round e holds rows
// [R_e, R_{e+1}) of every probed list, R_0 = 0, R_1 = p.tile, R_{e+1} = 2 R_e,
// and every candidate of the round is tested against the query's r after the
// earlier rounds (r = +inf in round 0).  Within a round r is frozen, so the
// round runs list-major (each list window staged once for all the queries
// that probe it, a long window cut into chunks over many thread blocks) or,
// where the list-major kernels do not apply and with DADE_FLAG_SEED_SPLIT,
// query-major with each query's lists split over thread blocks; then the K
// nearest are merged.  Rounds continue until they pass the longest list.
dade_status scan_rounds(const dade_index *ix, int64_t nq, const ScanParams &p, cudaStream_t s) {
    if (nq == 0) return DADE_OK;
    const int np = p.nprobe;
    const bool fd = p.mode == DADE_MODE_FD;
    const int gb = fd ? std::min(LNB, ix->nb) : std::min(p.delta_d / 16, ix->nb);
    const bool lm_ok = (ix->nb == LNB ? (gb == 1 || gb == 2 || gb == 4 || gb == 8)
                                      : (ix->nb > LNB && (gb == 1 || gb == 2 || gb == 4 || gb == 8))) &&
                       ix->max_list < (1 << QROW_BITS);
    k_lm_reset<<<grid_of(nq * (int64_t)p.k, 256), 256, 0, s>>>(p.ids, p.dists, nq * (int64_t)p.k);
    DADE_TRY(launch_check("k_lm_reset"));
    if (p.stats) DADE_TRY_CUDA(cudaMemsetAsync(p.stats, 0, sizeof(int64_t) * 4 * (size_t)nq, s));
    if (p.lead_stats) DADE_TRY_CUDA(cudaMemsetAsync(p.lead_stats, 0, sizeof(int64_t) * (size_t)nq, s));
    const int64_t longest = std::max(ix->max_list, 1);
    const int64_t r1 = std::max(p.tile, 1);
    if (lm_ok && !p.seed_split && !p.use_lead) {
        bool first = true;
        for (int64_t lo = 0, hi = r1; lo < longest; lo = hi, hi *= 2) {
            DADE_TRY(lm_round(ix, nq, p, 0, np, fd ? LNB : gb, !fd, s, (int)lo, (int)std::min<int64_t>(hi, INT_MAX),
                              first));
            first = false;
        }
        return DADE_OK;
    }
    // query-major: every round over all probe positions, each query's lists in parts over thread blocks
    if (p.q_k || p.q_np) {
        set_error("per-query K and nprobe under the row rounds need the list-major passes (D > 112, delta_d of "
                  "16, 32, 64 or 128 dims, no DADE_FLAG_SEED_SPLIT or DADE_FLAG_LEAD)");
        return DADE_EUNSUPPORTED;
    }
    Workspace &w = ws(ix);
    const int64_t cap = accept_cap(ix, np);
    DADE_TRY(w.lm_acc.ensure(sizeof(unsigned long long) * (size_t)(nq * cap)));
    DADE_TRY(w.lm_acnt.ensure(sizeof(int) * (size_t)nq));
    int dev = 0, sms = 0;
    DADE_TRY_CUDA(cudaGetDevice(&dev));
    DADE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t slots = (int64_t)sms * (768 / (p.threads == 256 ? 256 : 128));
    ScanParams q = p;
    q.schedule = DADE_SCHED_TILE;
    q.seed_split = 0;
    q.pstride = np;
    q.tile = 128;
    q.r2src = p.dists;
    q.acc = w.lm_acc.as<unsigned long long>();
    q.acnt = w.lm_acnt.as<int>();
    q.cap = cap;
    q.c0 = 0;
    q.parts = (int)std::min<int64_t>(np, std::max<int64_t>(1, (8 * slots + nq - 1) / nq));
    for (int64_t lo = 0, hi = r1; lo < longest; lo = hi, hi *= 2) {
        DADE_TRY_CUDA(cudaMemsetAsync(w.lm_acnt.p, 0, sizeof(int) * (size_t)nq, s));
        q.row_lo = (int)lo;
        q.row_hi = (int)std::min<int64_t>(hi, INT_MAX);
        DADE_TRY(scan(ix, nq, q, s));
        k_lm_merge<<<(unsigned)nq, MT, 0, s>>>(p.ids, p.dists, p.k, q.acc, q.acnt, cap, nullptr);
        DADE_TRY(launch_check("k_lm_merge"));
    }
    return DADE_OK;
}

} // namespace dade
