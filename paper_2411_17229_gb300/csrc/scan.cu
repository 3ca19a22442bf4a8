// scan.cu -- the DADE-IVF hot path: one DCO (Algorithm 1 with the test of
// Section 3.3) per (query, candidate of a probed list), feeding a per-query
// top-K (Section 3.4).
//
// One CTA owns one query.  It walks the probed lists in probe order and each
// list in tiles of `tile` candidates (ascending base id).  For every tile:
//   1. the first increment's blocks (delta_d dims = delta_d/16 slabs of
//      tile x 64 B, contiguous in the dimension-blocked layout) arrive in
//      shared memory by cp.async.bulk on an mbarrier, issued NS tiles ahead;
//   2. four lanes (a quad) per candidate compute P_d with 128-bit loads and
//      two shuffles; the test keeps a candidate iff P_d <= coef_j * r^2, the
//      squared form of dis' <= (1 + eps_d) r with dis'^2 = Lambda_D/Lambda_d
//      P_d (Eq. 13), coef_j = (1 + eps_d)^2 Lambda_d / Lambda_D;
//   3. survivors are compacted into a shared list (warp-aggregated atomics)
//      and the next increment gathers only their 64-byte block rows straight
//      from global memory, until d = D, where a candidate is accepted iff
//      P_D <= r^2 (Definition 1);
//   4. accepted candidates are rank-sorted by (squared distance, id) and
//      merged into the K-best list in shared memory; r^2 is refreshed from the
//      K-th entry once per tile (a stale r can only prune less).
// FDScanning (exact full-D distance for every candidate) streams every
// increment through the same bulk-copy ring and applies only the final test.
//
// Every mbarrier wait is bounded (2 s on %globaltimer); on expiry the CTA
// records DADE_ETIMEOUT in the index's error word, waits (bounded) for its
// own copies in flight and exits without writing results.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace dade {

namespace {

constexpr int MAX_TILE = 256;
constexpr int GCHUNK = 4;          // survivors per lane whose loads are issued together
constexpr uint64_t WAIT_NS = 2000000000ull;

struct Surv {
    int idx;      // candidate index within the tile
    float p;      // partial squared distance so far
};

struct ScanArgs {
    const float *data;
    const int32_t *ids;
    const ListMeta *meta;
    const float *q_rot;
    const int32_t *probe;
    int64_t *out_ids;
    float *out_d;
    int64_t *stats;
    int *err;
    int q_stride, nprobe, d, dp, nb, k, tile, gb, n_inc, ns, delta_d, stage;
    float coef[DADE_MAX_DIM / DADE_BLOCK];
};

// ---------------------------------------------------------- PTX helpers ----
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ bool wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar, parity))
        if (gtimer() - t0 > limit_ns) return false;
    return true;
}

__device__ __forceinline__ float sqd4(float4 q, float4 o) {
    float a = q.x - o.x, b = q.y - o.y, c = q.z - o.z, e = q.w - o.w;
    return fmaf(a, a, fmaf(b, b, fmaf(c, c, e * e)));
}

// Append (idx, p) for every quad leader with `want`; one atomic per warp.
__device__ __forceinline__ void push(bool want, Surv *list, int *cnt, int idx, float p) {
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (m == 0) return;
    int base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (want) list[base + __popc(m & ((1u << lane) - 1u))] = Surv{idx, p};
}

// Per-probe list descriptor kept in shared memory: x = base / 64 (the data
// offset in 256-byte units), y = first id slot, z = length, w = padded length.
constexpr int PMETA = 1024;   // probes whose descriptors are preloaded

__device__ __forceinline__ int4 meta_of(const ScanArgs &a, const int4 *sm, const int32_t *plist, int p) {
    if (p < PMETA) return sm[p];
    const ListMeta m = a.meta[plist[p]];
    return make_int4((int)(m.base >> 6), (int)m.slot, m.len, m.np);
}

// Tile cursor: probe position p, first candidate i0, increment j.
struct Cur {
    int p, i0, j;
};

__device__ __forceinline__ void normalize(Cur &c, const ScanArgs &a, const int4 *sm, const int32_t *plist) {
    while (c.p < a.nprobe && c.i0 >= meta_of(a, sm, plist, c.p).z) {
        ++c.p;
        c.i0 = 0;
        c.j = 0;
    }
}

// Advance over units: `units` staged increments per tile.
__device__ __forceinline__ void advance(Cur &c, int units, const ScanArgs &a, const int4 *sm, const int32_t *plist) {
    if (++c.j < units) return;
    c.j = 0;
    c.i0 += a.tile;
    normalize(c, a, sm, plist);
}

__device__ __forceinline__ const float *list_base(const ScanArgs &a, int4 m) {
    return a.data + ((int64_t)(unsigned)m.x << 6);
}

// Queue the bulk copies of one unit (tile c.i0 of probe c.p, increment c.j) into `slot`.
__device__ void issue(const ScanArgs &a, const int4 *sm, const int32_t *plist, const Cur &c, int slot, float *stage,
                      uint64_t *bars) {
    const int4 m = meta_of(a, sm, plist, c.p);
    const int tn = min(a.tile, m.z - c.i0);
    const int b0 = c.j * a.gb, b1 = min(b0 + a.gb, a.nb);
    const uint32_t bar = su32(&bars[slot]);
    mbar_expect_tx(bar, (uint32_t)((b1 - b0) * tn * 64));
    float *dst = stage + (size_t)slot * a.tile * a.gb * 16;
    const float *src = list_base(a, m) + (int64_t)c.i0 * 16;
    for (int b = b0; b < b1; ++b)
        bulk_g2s(su32(dst + (size_t)(b - b0) * a.tile * 16), src + (int64_t)b * m.w * 16, (uint32_t)(tn * 64), bar);
}

__device__ __forceinline__ int lower_bound_u64(const unsigned long long *v, int n, unsigned long long key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (v[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

struct SmemLayout {
    size_t meta, qv, stage, l0, l1, fl, fraw, fsort, top, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout layout(int dp, int tile, int gb, int ns, int k, int nprobe) {
    SmemLayout L;
    size_t o = 64;                                  // mbarriers (up to 8)
    L.meta = o;  o = align_up(o + sizeof(int4) * (size_t)min(nprobe, PMETA), 16);
    L.qv = o;    o = align_up(o + sizeof(float) * dp, 128);
    L.stage = o; o = align_up(o + sizeof(float) * (size_t)ns * tile * gb * 16, 128);
    L.l0 = o;    o += sizeof(Surv) * tile;
    L.l1 = o;    o += sizeof(Surv) * tile;
    L.fl = o;    o += sizeof(Surv) * tile;
    L.fraw = o;  o += 8 * (size_t)tile;
    L.fsort = o; o += 8 * (size_t)tile;
    L.top = o;   o += 16 * (size_t)k;
    L.total = align_up(o, 128);
    return L;
}

// Partial squared distance of one candidate row over blocks [b0, b1) (4 dims per lane).
__device__ __forceinline__ float row_part(const float *row, int64_t bstride, const float *qv, int b0, int b1, int lq,
                                          bool global_mem) {
    float p = 0.f;
    for (int b = b0; b < b1; ++b) {
        const float *src = row + (int64_t)(b - (global_mem ? 0 : b0)) * bstride;
        float4 o = global_mem ? __ldg(reinterpret_cast<const float4 *>(src)) : *reinterpret_cast<const float4 *>(src);
        float4 q = *reinterpret_cast<const float4 *>(qv + b * 16 + lq * 4);
        p += sqd4(q, o);
    }
    return p;
}

template <int NT, bool FD, bool STATS>
__global__ void __launch_bounds__(NT, 1024 / NT) k_scan(const ScanArgs a) {
    constexpr int NQUAD = NT / 4;              // candidates per pass
    constexpr int MAXIT = MAX_TILE / NQUAD;    // passes over a full tile
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_cnt[2], s_cntF, s_ntop, s_cur;
    __shared__ float s_r2;
    __shared__ unsigned long long s_stats[4];

    const int tid = threadIdx.x, quad = tid >> 2, lq = tid & 3;
    const int64_t qi = blockIdx.x;
    const SmemLayout L = layout(a.dp, a.tile, a.gb, a.ns, a.k, a.nprobe);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int4 *smeta = reinterpret_cast<int4 *>(smem + L.meta);
    float *qv = reinterpret_cast<float *>(smem + L.qv);
    float *stage = reinterpret_cast<float *>(smem + L.stage);
    Surv *l0 = reinterpret_cast<Surv *>(smem + L.l0);
    Surv *l1 = reinterpret_cast<Surv *>(smem + L.l1);
    Surv *fl = reinterpret_cast<Surv *>(smem + L.fl);
    unsigned long long *fraw = reinterpret_cast<unsigned long long *>(smem + L.fraw);
    unsigned long long *fsort = reinterpret_cast<unsigned long long *>(smem + L.fsort);
    unsigned long long *top0 = reinterpret_cast<unsigned long long *>(smem + L.top);
    unsigned long long *top1 = top0 + a.k;

    const int32_t *plist = a.probe + qi * a.nprobe;
    for (int k = tid; k < a.dp; k += NT) qv[k] = k < a.d ? a.q_rot[qi * a.q_stride + k] : 0.f;
    for (int p = tid; p < min(a.nprobe, PMETA); p += NT) {
        const ListMeta m = a.meta[plist[p]];
        smeta[p] = make_int4((int)(m.base >> 6), (int)m.slot, m.len, m.np);
    }
    if (tid == 0) {
        for (int s = 0; s < a.ns; ++s) mbar_init(su32(&bars[s]), 1);
        fence_mbar_init();
        s_ntop = 0;
        s_cur = 0;
        s_r2 = INFINITY;
    }
    if (STATS && tid < 4) s_stats[tid] = 0;
    __syncthreads();

    const int units = FD ? a.n_inc : min(a.stage, a.n_inc);   // staged increments per tile
    Cur cc{0, 0, 0};
    normalize(cc, a, smeta, plist);
    Cur ic = cc;          // issue cursor (thread 0 only)
    int issued = 0;       // units issued (thread 0 only)
    if (tid == 0)
        for (int s = 0; s < a.ns && ic.p < a.nprobe; ++s) {
            issue(a, smeta, plist, ic, s, stage, bars);
            advance(ic, units, a, smeta, plist);
            ++issued;
        }
    unsigned long long st_cand = 0, st_dims = 0, st_acc = 0, st_prn = 0;
    int unit = 0;
    bool aborted = false;

    while (cc.p < a.nprobe) {
        const int4 m = meta_of(a, smeta, plist, cc.p);
        const int tn = min(a.tile, m.z - cc.i0);
        const int nit = (tn + NQUAD - 1) / NQUAD;
        const float *lbase = list_base(a, m);
        const int64_t bstride = (int64_t)m.w * 16;     // floats between block slabs of this list
        if (tid == 0) {
            s_cnt[0] = 0;
            s_cntF = 0;
        }
        float r2 = 0.f;

        if (FD) {
            // ---- FDScanning: every increment staged, partials kept per lane ------
            float acc[MAXIT];
#pragma unroll
            for (int it = 0; it < MAXIT; ++it) acc[it] = 0.f;
            for (int j = 0; j < a.n_inc; ++j) {
                const int slot = unit % a.ns;
                const bool ok = wait_bounded(su32(&bars[slot]), (uint32_t)((unit / a.ns) & 1), WAIT_NS);
                if (__syncthreads_or(!ok)) { aborted = true; break; }
                if (j == 0) r2 = s_r2;
                const float *st = stage + (size_t)slot * a.tile * a.gb * 16;
                const int b0 = j * a.gb, b1 = min(b0 + a.gb, a.nb);
#pragma unroll
                for (int it = 0; it < MAXIT; ++it) {
                    const int c = quad + it * NQUAD;
                    if (it < nit && c < tn) acc[it] += row_part(st + c * 16 + lq * 4, (int64_t)a.tile * 16, qv, b0, b1, lq, false);
                }
                __syncthreads();
                if (tid == 0 && ic.p < a.nprobe) {
                    issue(a, smeta, plist, ic, slot, stage, bars);
                    advance(ic, units, a, smeta, plist);
                    ++issued;
                }
                ++unit;
            }
            if (aborted) break;
            for (int it = 0; it < nit; ++it) {
                const int c = quad + it * NQUAD;
                float p = acc[it];
                p += __shfl_xor_sync(0xffffffffu, p, 1);
                p += __shfl_xor_sync(0xffffffffu, p, 2);
                const bool act = c < tn;
                const bool take = act && lq == 0 && p <= r2;
                push(take, fl, &s_cntF, c, p);
                if (STATS && act && lq == 0) { ++st_cand; st_dims += a.d; st_acc += take; }
            }
            __syncthreads();
        } else {
            // ---- DADE, increment 0 over the whole tile (staged) --------------------
            int slot = unit % a.ns;
            bool ok = wait_bounded(su32(&bars[slot]), (uint32_t)((unit / a.ns) & 1), WAIT_NS);
            if (__syncthreads_or(!ok)) { aborted = true; break; }
            r2 = s_r2;
            {
                const float *st = stage + (size_t)slot * a.tile * a.gb * 16;
                const int b1 = min(a.gb, a.nb);
                const bool last0 = a.n_inc == 1;
                const int d0 = min(a.delta_d, a.d);
                const float c0 = a.coef[0] * r2;
                for (int it = 0; it < nit; ++it) {
                    const int c = quad + it * NQUAD;
                    const bool act = c < tn;
                    float p = act ? row_part(st + c * 16 + lq * 4, (int64_t)a.tile * 16, qv, 0, b1, lq, false) : 0.f;
                    p += __shfl_xor_sync(0xffffffffu, p, 1);
                    p += __shfl_xor_sync(0xffffffffu, p, 2);
                    const bool lead = act && lq == 0;
                    const bool toF = lead && last0 && p <= r2;
                    const bool toN = lead && !last0 && !(p > c0);
                    push(toF, fl, &s_cntF, c, p);
                    push(toN, l0, &s_cnt[0], c, p);
                    if (STATS && lead) {
                        ++st_cand;
                        if (last0) { st_dims += a.d; st_acc += toF; }
                        else if (!toN) { st_dims += d0; ++st_prn; }
                    }
                }
            }
            __syncthreads();
            if (tid == 0 && ic.p < a.nprobe) {
                issue(a, smeta, plist, ic, slot, stage, bars);
                advance(ic, units, a, smeta, plist);
                ++issued;
            }
            ++unit;
            // ---- later increments: staged (j < units) or gathered ------------------
            int ns_cur = s_cnt[0];
            for (int j = 1; j < a.n_inc; ++j) {
                const bool staged = j < units;
                if (!staged && ns_cur == 0) break;
                const int src = (j - 1) & 1, dst = j & 1;
                if (tid == 0) s_cnt[dst] = 0;
                if (staged) {
                    slot = unit % a.ns;
                    ok = wait_bounded(su32(&bars[slot]), (uint32_t)((unit / a.ns) & 1), WAIT_NS);
                    if (__syncthreads_or(!ok)) { aborted = true; break; }
                } else {
                    __syncthreads();
                }
                if (ns_cur > 0) {
                    const int b0 = j * a.gb, b1 = min(b0 + a.gb, a.nb);
                    const bool last = j == a.n_inc - 1;
                    const int dj = min((j + 1) * a.delta_d, a.d);
                    const float cj = a.coef[j] * r2;
                    const Surv *in = src ? l1 : l0;
                    Surv *out = dst ? l1 : l0;
                    const float *st = stage + (size_t)slot * a.tile * a.gb * 16;
                    const int nits = (ns_cur + NQUAD - 1) / NQUAD;
                    for (int it0 = 0; it0 < nits; it0 += GCHUNK) {
                        // all loads of this lane's survivors first, then the reductions
                        Surv sv[GCHUNK];
                        float part[GCHUNK];
#pragma unroll
                        for (int u = 0; u < GCHUNK; ++u) {
                            const int s = quad + (it0 + u) * NQUAD;
                            const bool act = it0 + u < nits && s < ns_cur;
                            sv[u] = act ? in[s] : Surv{-1, 0.f};
                            part[u] = 0.f;
                            if (act)
                                part[u] = staged
                                    ? row_part(st + sv[u].idx * 16 + lq * 4, (int64_t)a.tile * 16, qv, b0, b1, lq, false)
                                    : row_part(lbase + (int64_t)(cc.i0 + sv[u].idx) * 16 + lq * 4, bstride, qv, b0, b1,
                                               lq, true);
                        }
#pragma unroll
                        for (int u = 0; u < GCHUNK; ++u) {
                            if (it0 + u >= nits) break;
                            float pp = part[u];
                            pp += __shfl_xor_sync(0xffffffffu, pp, 1);
                            pp += __shfl_xor_sync(0xffffffffu, pp, 2);
                            const float p = sv[u].p + pp;
                            const bool lead = sv[u].idx >= 0 && lq == 0;
                            const bool toF = lead && last && p <= r2;
                            const bool toN = lead && !last && !(p > cj);
                            push(toF, fl, &s_cntF, sv[u].idx, p);
                            push(toN, out, &s_cnt[dst], sv[u].idx, p);
                            if (STATS && lead) {
                                if (last) { st_dims += a.d; st_acc += toF; }
                                else if (!toN) { st_dims += dj; ++st_prn; }
                            }
                        }
                    }
                }
                __syncthreads();
                if (staged) {
                    if (tid == 0 && ic.p < a.nprobe) {
                        issue(a, smeta, plist, ic, slot, stage, bars);
                        advance(ic, units, a, smeta, plist);
                        ++issued;
                    }
                    ++unit;
                }
                ns_cur = j == a.n_inc - 1 ? 0 : s_cnt[dst];
            }
            if (aborted) break;
        }

        // ---- merge accepted candidates into the K best ------------------------------
        const int nF = s_cntF;
        if (nF > 0) {
            for (int t = tid; t < nF; t += NT) {
                const Surv f = fl[t];
                const unsigned id = (unsigned)a.ids[(int64_t)(unsigned)m.y + cc.i0 + f.idx];
                fraw[t] = ((unsigned long long)__float_as_uint(f.p) << 32) | id;
            }
            __syncthreads();
            for (int t = tid; t < nF; t += NT) {
                const unsigned long long kk = fraw[t];
                int r = 0;
                for (int u = 0; u < nF; ++u) r += fraw[u] < kk;
                fsort[r] = kk;
            }
            __syncthreads();
            const int nt = s_ntop, cur = s_cur;
            const unsigned long long *A = cur ? top1 : top0;
            unsigned long long *O = cur ? top0 : top1;
            for (int t = tid; t < nt; t += NT) {
                const int pos = t + lower_bound_u64(fsort, nF, A[t]);
                if (pos < a.k) O[pos] = A[t];
            }
            for (int t = tid; t < nF; t += NT) {
                const int pos = t + lower_bound_u64(A, nt, fsort[t]);
                if (pos < a.k) O[pos] = fsort[t];
            }
            __syncthreads();
            if (tid == 0) {
                const int nn = min(a.k, nt + nF);
                s_ntop = nn;
                s_cur = cur ^ 1;
                s_r2 = nn == a.k ? __uint_as_float((unsigned)(O[a.k - 1] >> 32)) : INFINITY;
            }
        }
        __syncthreads();
        cc.j = 0;
        cc.i0 += a.tile;
        normalize(cc, a, smeta, plist);
    }

    if (aborted) {
        if (tid == 0) {
            atomicExch(a.err, (int)DADE_ETIMEOUT);
            for (int u = unit; u < issued; ++u)
                wait_bounded(su32(&bars[u % a.ns]), (uint32_t)((u / a.ns) & 1), 10000000ull);
        }
        return;
    }
    const int nt = s_ntop;
    const unsigned long long *R = s_cur ? top1 : top0;
    for (int t = tid; t < a.k; t += NT) {
        int64_t id = -1;
        float dv = INFINITY;
        if (t < nt) {
            id = (int64_t)(unsigned)(R[t] & 0xffffffffu);
            dv = __uint_as_float((unsigned)(R[t] >> 32));
        }
        a.out_ids[qi * a.k + t] = id;
        a.out_d[qi * a.k + t] = dv;
    }
    if (STATS) {
        if (lq == 0) {
            atomicAdd(&s_stats[0], st_cand);
            atomicAdd(&s_stats[1], st_dims);
            atomicAdd(&s_stats[2], st_acc);
            atomicAdd(&s_stats[3], st_prn);
        }
        __syncthreads();
        if (tid < 4) a.stats[qi * 4 + tid] = (int64_t)s_stats[tid];
    }
}

template <int NT, bool FD, bool STATS>
dade_status launch(const ScanArgs &a, int64_t nq, size_t smem, cudaStream_t s) {
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        DADE_TRY_CUDA(cudaFuncSetAttribute(k_scan<NT, FD, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        configured = smem;
    }
    k_scan<NT, FD, STATS><<<(unsigned)nq, NT, smem, s>>>(a);
    return launch_check(FD ? "k_scan<FD>" : "k_scan<DADE>");
}

template <int NT>
dade_status launch_nt(const ScanArgs &a, int64_t nq, size_t smem, bool fd, bool stats, cudaStream_t s) {
    if (fd) return stats ? launch<NT, true, true>(a, nq, smem, s) : launch<NT, true, false>(a, nq, smem, s);
    return stats ? launch<NT, false, true>(a, nq, smem, s) : launch<NT, false, false>(a, nq, smem, s);
}

} // namespace

dade_status scan(const dade_index *ix, int64_t nq, const ScanParams &p, cudaStream_t s) {
    if (nq == 0) return DADE_OK;
    ScanArgs a{};
    a.data = ix->data.as<float>();
    a.ids = ix->ids.as<int32_t>();
    a.meta = ix->meta.as<ListMeta>();
    a.q_rot = p.q_rot;
    a.probe = p.probe;
    a.out_ids = p.ids;
    a.out_d = p.dists;
    a.stats = p.stats;
    a.err = ix->errflag.as<int>();
    a.q_stride = p.q_stride;
    a.nprobe = p.nprobe;
    a.d = ix->d;
    a.dp = ix->dp;
    a.nb = ix->nb;
    a.k = p.k;
    a.tile = p.tile;
    a.ns = 2;
    a.stage = p.stage;
    const bool fd = p.mode == DADE_MODE_FD;
    if (fd) {
        a.gb = std::min(4, ix->nb);
        a.delta_d = a.gb * 16;
    } else {
        a.gb = std::min(p.delta_d / 16, ix->nb);
        a.delta_d = p.delta_d;
    }
    a.n_inc = (ix->nb + a.gb - 1) / a.gb;
    for (int j = 0; j < DADE_MAX_DIM / DADE_BLOCK; ++j) a.coef[j] = j < p.n_inc ? p.coef[j] : INFINITY;
    const SmemLayout L = layout(a.dp, a.tile, a.gb, a.ns, a.k, a.nprobe);
    if (L.total > 227 * 1024) {
        set_error("scan configuration needs more than 227 KB of shared memory (reduce tile or delta_d)");
        return DADE_EUNSUPPORTED;
    }
    if (p.threads == 256) return launch_nt<256>(a, nq, L.total, fd, p.stats != nullptr, s);
    return launch_nt<128>(a, nq, L.total, fd, p.stats != nullptr, s);
}

} // namespace dade
