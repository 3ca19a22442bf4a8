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

constexpr int NT = 256;            // threads per CTA
constexpr int NQUAD = NT / 4;      // candidates per pass
constexpr int MAXIT = 4;           // tile <= 256 = MAXIT * NQUAD
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
    int q_stride, nprobe, d, dp, nb, k, tile, gb, n_inc, ns, delta_d;
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

// Tile cursor: probe position p, first candidate i0, increment j.
struct Cur {
    int p, i0, j;
};

__device__ __forceinline__ void normalize(Cur &c, const ScanArgs &a, const int32_t *plist) {
    while (c.p < a.nprobe && c.i0 >= a.meta[plist[c.p]].len) {
        ++c.p;
        c.i0 = 0;
        c.j = 0;
    }
}

template <bool FD>
__device__ __forceinline__ void advance(Cur &c, const ScanArgs &a, const int32_t *plist) {
    if (FD && ++c.j < a.n_inc) return;
    c.j = 0;
    c.i0 += a.tile;
    normalize(c, a, plist);
}

// Queue the bulk copies of one unit (a tile's increment c.j) into `slot`.
__device__ void issue(const ScanArgs &a, const int32_t *plist, const Cur &c, int slot, float *stage, uint64_t *bars) {
    const ListMeta m = a.meta[plist[c.p]];
    const int tn = min(a.tile, m.len - c.i0);
    const int b0 = c.j * a.gb, b1 = min(b0 + a.gb, a.nb);
    const uint32_t bar = su32(&bars[slot]);
    mbar_expect_tx(bar, (uint32_t)((b1 - b0) * tn * 64));
    float *dst = stage + (size_t)slot * a.tile * a.gb * 16;
    for (int b = b0; b < b1; ++b)
        bulk_g2s(su32(dst + (size_t)(b - b0) * a.tile * 16),
                 a.data + m.base + (int64_t)b * m.np * 16 + (int64_t)c.i0 * 16, (uint32_t)(tn * 64), bar);
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
    size_t qv, stage, l0, l1, fl, fraw, fsort, top, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline SmemLayout layout(int dp, int tile, int gb, int ns, int k) {
    SmemLayout L;
    size_t o = 64;                                  // mbarriers (up to 8)
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

template <bool FD, bool STATS>
__global__ void __launch_bounds__(NT) k_scan(const ScanArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_cnt[2], s_cntF, s_ntop, s_cur;
    __shared__ float s_r2;
    __shared__ unsigned long long s_stats[4];

    const int tid = threadIdx.x, quad = tid >> 2, lq = tid & 3;
    const int64_t qi = blockIdx.x;
    const SmemLayout L = layout(a.dp, a.tile, a.gb, a.ns, a.k);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *qv = reinterpret_cast<float *>(smem + L.qv);
    float *stage = reinterpret_cast<float *>(smem + L.stage);
    Surv *lst[2] = {reinterpret_cast<Surv *>(smem + L.l0), reinterpret_cast<Surv *>(smem + L.l1)};
    Surv *fl = reinterpret_cast<Surv *>(smem + L.fl);
    unsigned long long *fraw = reinterpret_cast<unsigned long long *>(smem + L.fraw);
    unsigned long long *fsort = reinterpret_cast<unsigned long long *>(smem + L.fsort);
    unsigned long long *top[2] = {reinterpret_cast<unsigned long long *>(smem + L.top),
                                  reinterpret_cast<unsigned long long *>(smem + L.top) + a.k};

    for (int k = tid; k < a.dp; k += NT) qv[k] = k < a.d ? a.q_rot[qi * a.q_stride + k] : 0.f;
    if (tid == 0) {
        for (int s = 0; s < a.ns; ++s) mbar_init(su32(&bars[s]), 1);
        fence_mbar_init();
        s_ntop = 0;
        s_cur = 0;
        s_r2 = INFINITY;
    }
    if (STATS && tid < 4) s_stats[tid] = 0;
    __syncthreads();

    const int32_t *plist = a.probe + qi * a.nprobe;
    Cur cc{0, 0, 0};
    normalize(cc, a, plist);
    Cur ic = cc;          // issue cursor (thread 0 only)
    int issued = 0;       // units issued (thread 0 only)
    if (tid == 0)
        for (int s = 0; s < a.ns && ic.p < a.nprobe; ++s) {
            issue(a, plist, ic, s, stage, bars);
            advance<FD>(ic, a, plist);
            ++issued;
        }
    unsigned long long st_cand = 0, st_dims = 0, st_acc = 0, st_prn = 0;
    int unit = 0;
    bool aborted = false;

    while (cc.p < a.nprobe) {
        const ListMeta m = a.meta[plist[cc.p]];
        const int tn = min(a.tile, m.len - cc.i0);
        const int nit = (tn + NQUAD - 1) / NQUAD;
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
                const int b0 = j * a.gb, nbj = min(a.gb, a.nb - b0);
#pragma unroll
                for (int it = 0; it < MAXIT; ++it) {
                    const int c = quad + it * NQUAD;
                    if (it < nit && c < tn)
                        for (int b = 0; b < nbj; ++b) {
                            float4 o = *reinterpret_cast<const float4 *>(st + ((size_t)b * a.tile + c) * 16 + lq * 4);
                            float4 q = *reinterpret_cast<const float4 *>(qv + (b0 + b) * 16 + lq * 4);
                            acc[it] += sqd4(q, o);
                        }
                }
                __syncthreads();
                if (tid == 0 && ic.p < a.nprobe) {
                    issue(a, plist, ic, slot, stage, bars);
                    advance<FD>(ic, a, plist);
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
            // ---- DADE: first increment from the staged blocks ---------------------
            const int slot = unit % a.ns;
            const bool ok = wait_bounded(su32(&bars[slot]), (uint32_t)((unit / a.ns) & 1), WAIT_NS);
            if (__syncthreads_or(!ok)) { aborted = true; break; }
            r2 = s_r2;
            const float *st = stage + (size_t)slot * a.tile * a.gb * 16;
            const int nb0 = min(a.gb, a.nb);
            const bool last0 = a.n_inc == 1;
            const int d0 = min(a.delta_d, a.d);
            const float c0 = a.coef[0] * r2;
            for (int it = 0; it < nit; ++it) {
                const int c = quad + it * NQUAD;
                const bool act = c < tn;
                float p = 0.f;
                if (act)
                    for (int b = 0; b < nb0; ++b) {
                        float4 o = *reinterpret_cast<const float4 *>(st + ((size_t)b * a.tile + c) * 16 + lq * 4);
                        float4 q = *reinterpret_cast<const float4 *>(qv + b * 16 + lq * 4);
                        p += sqd4(q, o);
                    }
                p += __shfl_xor_sync(0xffffffffu, p, 1);
                p += __shfl_xor_sync(0xffffffffu, p, 2);
                const bool lead = act && lq == 0;
                const bool toF = lead && last0 && p <= r2;
                const bool toN = lead && !last0 && !(p > c0);
                push(toF, fl, &s_cntF, c, p);
                push(toN, lst[0], &s_cnt[0], c, p);
                if (STATS && lead) {
                    ++st_cand;
                    if (last0) { st_dims += a.d; st_acc += toF; }
                    else if (!toN) { st_dims += d0; ++st_prn; }
                }
            }
            __syncthreads();
            if (tid == 0 && ic.p < a.nprobe) {
                issue(a, plist, ic, slot, stage, bars);
                advance<FD>(ic, a, plist);
                ++issued;
            }
            ++unit;
            // ---- later increments: gather survivors' block rows ------------------
            int ns_cur = s_cnt[0];
            for (int j = 1; j < a.n_inc && ns_cur > 0; ++j) {
                const int src = (j - 1) & 1, dst = j & 1;
                if (tid == 0) s_cnt[dst] = 0;
                __syncthreads();
                const int b0 = j * a.gb, b1 = min(b0 + a.gb, a.nb);
                const bool last = j == a.n_inc - 1;
                const int dj = min((j + 1) * a.delta_d, a.d);
                const float cj = a.coef[j] * r2;
                const Surv *in = lst[src];
                const int nits = (ns_cur + NQUAD - 1) / NQUAD;
                for (int it = 0; it < nits; ++it) {
                    const int s = quad + it * NQUAD;
                    const bool act = s < ns_cur;
                    Surv sv = act ? in[s] : Surv{0, 0.f};
                    float part = 0.f;
                    if (act) {
                        const float *row = a.data + m.base + (int64_t)(cc.i0 + sv.idx) * 16 + lq * 4;
                        for (int b = b0; b < b1; ++b) {
                            float4 o = __ldg(reinterpret_cast<const float4 *>(row + (int64_t)b * m.np * 16));
                            float4 q = *reinterpret_cast<const float4 *>(qv + b * 16 + lq * 4);
                            part += sqd4(q, o);
                        }
                    }
                    part += __shfl_xor_sync(0xffffffffu, part, 1);
                    part += __shfl_xor_sync(0xffffffffu, part, 2);
                    const float p = sv.p + part;
                    const bool lead = act && lq == 0;
                    const bool toF = lead && last && p <= r2;
                    const bool toN = lead && !last && !(p > cj);
                    push(toF, fl, &s_cntF, sv.idx, p);
                    push(toN, lst[dst], &s_cnt[dst], sv.idx, p);
                    if (STATS && lead) {
                        if (last) { st_dims += a.d; st_acc += toF; }
                        else if (!toN) { st_dims += dj; ++st_prn; }
                    }
                }
                __syncthreads();
                ns_cur = last ? 0 : s_cnt[dst];
            }
        }

        // ---- merge accepted candidates into the K best ------------------------------
        const int nF = s_cntF;
        if (nF > 0) {
            for (int t = tid; t < nF; t += NT) {
                const Surv f = fl[t];
                const unsigned id = (unsigned)a.ids[m.slot + cc.i0 + f.idx];
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
            const unsigned long long *A = top[cur];
            unsigned long long *O = top[cur ^ 1];
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
        if (!FD) advance<FD>(cc, a, plist);
        else { cc.j = 0; cc.i0 += a.tile; normalize(cc, a, plist); }
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
    const unsigned long long *R = top[s_cur];
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

template <bool FD, bool STATS>
dade_status launch(const ScanArgs &a, int64_t nq, size_t smem, cudaStream_t s) {
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        DADE_TRY_CUDA(cudaFuncSetAttribute(k_scan<FD, STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        configured = smem;
    }
    k_scan<FD, STATS><<<(unsigned)nq, NT, smem, s>>>(a);
    return launch_check(FD ? "k_scan<FD>" : "k_scan<DADE>");
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
    const SmemLayout L = layout(a.dp, a.tile, a.gb, a.ns, a.k);
    if (L.total > 227 * 1024) {
        set_error("scan configuration needs more than 227 KB of shared memory (reduce tile or delta_d)");
        return DADE_EUNSUPPORTED;
    }
    if (fd) return p.stats ? launch<true, true>(a, nq, L.total, s) : launch<true, false>(a, nq, L.total, s);
    return p.stats ? launch<false, true>(a, nq, L.total, s) : launch<false, false>(a, nq, L.total, s);
}

} // namespace dade
