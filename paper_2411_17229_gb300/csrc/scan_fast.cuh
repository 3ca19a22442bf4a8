// scan_fast.cuh -- the tile-schedule scan kernels specialised at compile time
// for a dimension-blocked layout of NB = 8 blocks (D in 113..128) and an
// increment of GB blocks (delta_d = 16 GB), shared by scan_fast.cu (FP32 and
// FDScanning instantiations) and scan_lead.cu (low-precision leading blocks).
// Same algorithm and results as the generic kernel in scan.cu (Algorithm 1
// with the Section 3.3 test, threshold refreshed once per tile), with:
//   - the query's 4-dimension slice of every block held in registers by each
//     lane of a quad for the whole scan (no shared-memory loads of q);
//   - every loop over blocks and increments unrolled, so increment
//     boundaries and pruning coefficients are compile-time positions;
//   - phase A (increment 0 of the whole tile, bulk-copied) compacts the
//     survivors with one warp-aggregated append per pass;
//   - phase B loads all remaining blocks of a survivor at once into registers
//     and runs the remaining tests there.
// FDScanning gets the same treatment: q in registers, units of 4 blocks
// streamed through the bulk-copy ring, unrolled accumulation.
#pragma once

#include <algorithm>

#include "internal.cuh"
#include "scan_common.cuh"

namespace dade {
namespace {
using namespace scanning;

constexpr int FNB = 8;   // blocks of the specialised layout

template <int NB>
__device__ __forceinline__ void load_q(const ScanArgs &a, int64_t qi, int lq, float4 (&qr)[NB]) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        float v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int k = b * 16 + lq * 4 + t;
            v[t] = k < a.d ? a.q_rot[qi * a.q_stride + k] : 0.f;
        }
        qr[b] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

__device__ __forceinline__ float quad_sum(float p) {
    p += __shfl_xor_sync(0xffffffffu, p, 1);
    p += __shfl_xor_sync(0xffffffffu, p, 2);
    return p;
}

// Chunked staging: a tile of up to 256 candidates (one threshold epoch)
// streams its first increment in chunks of CH candidates through a ring of
// NSF bulk-copy slots, so the tile size does not dictate shared memory.
constexpr int CH = 64;

template <int GB, int LF = 0>
struct ChunkRing {
    static constexpr int NSF32 = GB >= 8 ? 2 : (GB >= 4 ? 2 : 8 / GB);   // FP32: slots of CH x GB x 64 B
    // floats per slot: FP32 slabs, or (LF) the codes plus the error norms, 128-B aligned
    static constexpr int SLOT = LF ? (GB * CH * 16 * LeadFmt<LF>::ES + CH * 4 + 127) / 128 * 32 : GB * CH * 16;
    // LF: as many of the smaller slots as fit in the FP32 ring (<= 8 mbarriers)
    static constexpr int NSF = LF ? (NSF32 * GB * CH * 16 / SLOT < 8 ? NSF32 * GB * CH * 16 / SLOT : 8) : NSF32;
};

struct FastLayout {
    size_t meta, stage, l0, fl, fraw, fsort, top, total;
};

__host__ __device__ inline FastLayout fast_layout(int tile, int slot_floats, int nsf, int k, int nprobe) {
    FastLayout L;
    size_t o = 64;                                  // mbarriers (up to 8)
    L.meta = o;  o = align_up(o + sizeof(int4) * (size_t)min(nprobe, PMETA), 128);
    L.stage = o; o = align_up(o + sizeof(float) * (size_t)nsf * slot_floats, 128);
    L.l0 = o;    o += sizeof(Surv) * (size_t)tile;
    L.fl = o;    o += sizeof(Surv) * (size_t)tile;
    L.fraw = o;  o += 8 * (size_t)pow2_at_least(tile);
    L.fsort = o; o += 8 * (size_t)pow2_at_least(tile);
    L.top = o;   o += 16 * (size_t)k;
    L.total = align_up(o, 128);
    return L;
}

// Chunk cursor: probe position p, tile start i0, chunk j within the tile.
__device__ __forceinline__ void chunk_advance(Cur &c, const ScanArgs &a, const int4 *sm, const int32_t *plist) {
    const int len = meta_of(a, sm, plist, c.p).z;
    const int tn = min(a.tile, len - c.i0);
    if ((++c.j) * CH < tn) return;
    c.j = 0;
    c.i0 += a.tile;
    normalize(c, a, sm, plist);
}

// One chunk of the first increment into ring slot `slot`: GB FP32 slabs, or
// (LF) the low-precision codes of the same dims plus their error norms.
template <int GB, int LF>
__device__ inline void issue_chunk(const ScanArgs &a, const int4 *sm, const int32_t *plist, const Cur &c, int slot,
                                   float *stage, uint64_t *bars) {
    const int4 m = meta_of(a, sm, plist, c.p);
    const int tn = min(a.tile, m.z - c.i0);
    const int c0 = c.i0 + c.j * CH;
    const int cn = min(CH, c.i0 + tn - c0);
    const uint32_t bar = su32(&bars[slot]);
    float *dst = stage + (size_t)slot * ChunkRing<GB, LF>::SLOT;
    if constexpr (LF != 0) {
        issue_lead<LF>(a, m, c0, cn, GB, CH, reinterpret_cast<unsigned char *>(dst), bar);
        return;
    }
    mbar_expect_tx(bar, (uint32_t)(GB * cn * 64));
    const float *src = list_base(a, m) + (int64_t)c0 * 16;
#pragma unroll
    for (int b = 0; b < GB; ++b)
        bulk_g2s(su32(dst + (size_t)b * CH * 16), src + (int64_t)b * m.w * 16, (uint32_t)(cn * 64), bar);
}

// LF = 0: FP32 throughout.  LF = 1 (BF16) / 2 (FP8): phase A runs the
// certified prefilter on the low-precision copy of the first increment
// (lead_prunes); phase B loads all NB FP32 blocks of every survivor and runs
// Algorithm 1 from the first increment, with the same arithmetic order as
// the FP32 kernel, so the two give identical results.
template <int NT, int NB, int GB, bool STATS, int LF>
__global__ void __launch_bounds__(NT, 640 / NT) k_dade_fast(const ScanArgs a) {
    constexpr int NQUAD = NT / 4;
    constexpr int CIT = (CH + NQUAD - 1) / NQUAD;   // passes over one chunk
    constexpr int NINC = (NB + GB - 1) / GB;
    constexpr int NSF = ChunkRing<GB, LF>::NSF;
    constexpr int SLOT = ChunkRing<GB, LF>::SLOT;
    constexpr int ES = LeadFmt<LF>::ES;
    constexpr int B0 = LF ? 0 : GB;                 // first FP32 block a survivor loads in phase B
    constexpr int NLOAD = NB - B0;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_cnt, s_cntF, s_ntop, s_cur;
    __shared__ float s_r2;
    __shared__ unsigned long long s_stats[4], s_lead;

    const int tid = threadIdx.x, quad = tid >> 2, lq = tid & 3;
    const int64_t qi = cta_query(a);
    // this query's K and nprobe, within the batch's largest (a.k, a.nprobe: buffer sizes and strides)
    const int kq = a.q_k ? min(max(a.q_k[qi], 1), a.k) : a.k;
    const int npq = a.q_np ? min(max(a.q_np[qi], 0), a.nprobe) : a.nprobe;
    const FastLayout L = fast_layout(a.tile, SLOT, NSF, a.k, a.nprobe);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int4 *smeta = reinterpret_cast<int4 *>(smem + L.meta);
    float *stage = reinterpret_cast<float *>(smem + L.stage);
    Surv *l0 = reinterpret_cast<Surv *>(smem + L.l0);
    Surv *fl = reinterpret_cast<Surv *>(smem + L.fl);
    unsigned long long *fraw = reinterpret_cast<unsigned long long *>(smem + L.fraw);
    unsigned long long *fsort = reinterpret_cast<unsigned long long *>(smem + L.fsort);
    unsigned long long *top0 = reinterpret_cast<unsigned long long *>(smem + L.top);
    unsigned long long *top1 = top0 + a.k;

    float4 qr[NB];
    load_q<NB>(a, qi, lq, qr);
    const int32_t *plist = a.probe + qi * a.pstride;
    for (int p = tid; p < min(a.nprobe, PMETA); p += NT) {
        const ListMeta m = a.meta[plist[p]];
        smeta[p] = make_int4((int)(m.base >> 6), (int)m.slot, m.len, m.np);
    }
    if (tid == 0) {
        for (int s = 0; s < NSF; ++s) mbar_init(su32(&bars[s]), 1);
        fence_mbar_init();
        s_ntop = 0;
        s_cur = 0;
        s_r2 = INFINITY;
    }
    if (STATS && tid < 4) s_stats[tid] = 0;
    if (tid == 0) s_lead = 0;
    __syncthreads();

    Cur cc{0, 0, 0, npq};
    normalize(cc, a, smeta, plist);
    Cur ic = cc;           // next chunk to issue (thread 0)
    int issued = 0;
    if (tid == 0)
        for (int s = 0; s < NSF && ic.p < npq; ++s) {
            issue_chunk<GB, LF>(a, smeta, plist, ic, s, stage, bars);
            chunk_advance(ic, a, smeta, plist);
            ++issued;
        }
    unsigned long long st_cand = 0, st_dims = 0, st_acc = 0, st_prn = 0, st_lead = 0;
    int unit = 0;
    bool aborted = false;

    while (cc.p < npq) {
        const int4 m = meta_of(a, smeta, plist, cc.p);
        const int tn = min(a.tile, m.z - cc.i0);
        const float *lbase = list_base(a, m);
        const int64_t bstride = (int64_t)m.w * 16;
        if (tid == 0) {
            s_cnt = 0;
            s_cntF = 0;
        }
        float r2 = 0.f;
        // LF: this lane's slice of q' - c' over the first increment, the FP8 block
        // scales and ||q' - c'|| (whole quad), fixed for the list
        float4 qc[LF ? GB : 1];
        float sc[LF ? GB : 1];
        float qcn = 0.f;
        if constexpr (LF != 0) {
            const int list = plist[cc.p];
            const float *cp = a.cent + (int64_t)list * a.dp + lq * 4;
            float qn = 0.f;
#pragma unroll
            for (int b = 0; b < GB; ++b) {
                const float4 c4 = __ldg(reinterpret_cast<const float4 *>(cp + b * 16));
                qc[b] = make_float4(__fsub_rn(qr[b].x, c4.x), __fsub_rn(qr[b].y, c4.y), __fsub_rn(qr[b].z, c4.z),
                                    __fsub_rn(qr[b].w, c4.w));
                qn = fmaf(qc[b].x, qc[b].x, fmaf(qc[b].y, qc[b].y, fmaf(qc[b].z, qc[b].z, fmaf(qc[b].w, qc[b].w, qn))));
                sc[b] = LF == 2 ? __ldg(a.lead_scale + (int64_t)list * a.lead_nb + b) : 1.f;
            }
            qcn = sqrtf(quad_sum(qn));
        }
        // ---- phase A: increment 0 of the tile, chunk by chunk ----------------------------
        const int nch = (tn + CH - 1) / CH;
        for (int j = 0; j < nch; ++j) {
            const int slot = unit % NSF;
            if (!wait_block(su32(&bars[slot]), (uint32_t)((unit / NSF) & 1), a.wait_ns, unit == 0 ? a.never : nullptr)) { aborted = true; break; }
            if (j == 0) r2 = s_r2;
            const int cbase = j * CH, cn = min(CH, tn - cbase);
            if constexpr (LF != 0) {
                const unsigned char *sl = reinterpret_cast<const unsigned char *>(stage + (size_t)slot * SLOT);
                const float *se = reinterpret_cast<const float *>(sl + (size_t)GB * CH * 16 * ES);
                const float thr = NINC == 1 ? r2 : a.coef[0] * r2;
#pragma unroll
                for (int it = 0; it < CIT; ++it) {
                    const int c = quad + it * NQUAD;
                    const bool act = c < cn;
                    float p = 0.f;
                    if (act) {
#pragma unroll
                        for (int b = 0; b < GB; ++b)
                            p += sqd4(qc[b], lead4<LF>(sl + ((size_t)(b * CH + c) * 16 + lq * 4) * ES, sc[b]));
                    }
                    p = quad_sum(p);
                    const bool lead = act && lq == 0;
                    const bool drop = lead && lead_prunes(p, se[c], qcn, thr);
                    push(lead && !drop, l0, &s_cnt, cbase + c, 0.f);
                    if (drop) {   // counted as the exact path counts it: pruned at d0, or rejected at D
                        ++st_lead;
                        if (STATS) { ++st_cand; st_dims += NINC == 1 ? a.d : min(GB * 16, a.d); st_prn += NINC != 1; }
                    } else if (STATS && lead) {
                        ++st_cand;
                    }
                }
                __syncthreads();
                if (tid == 0 && ic.p < npq) {
                    issue_chunk<GB, LF>(a, smeta, plist, ic, slot, stage, bars);
                    chunk_advance(ic, a, smeta, plist);
                    ++issued;
                }
                ++unit;
                continue;
            }
            const float *st = stage + (size_t)slot * SLOT + lq * 4;
            const float c0 = a.coef[0] * r2;
            Surv *dst = NINC == 1 ? fl : l0;
            int *cnt = NINC == 1 ? &s_cntF : &s_cnt;
#pragma unroll
            for (int it = 0; it < CIT; ++it) {
                const int c = quad + it * NQUAD;
                const bool act = c < cn;
                float p = 0.f;
                if (act) {
#pragma unroll
                    for (int b = 0; b < GB; ++b)
                        p += sqd4(qr[b], *reinterpret_cast<const float4 *>(st + ((size_t)b * CH + c) * 16));
                }
                p = quad_sum(p);
                const bool lead = act && lq == 0;
                const bool keep = lead && (NINC == 1 ? p <= r2 : !(p > c0));
                push(keep, dst, cnt, cbase + c, p);
                if (STATS && lead) {
                    ++st_cand;
                    if (NINC == 1) { st_dims += a.d; st_acc += keep; }
                    else if (!keep) { st_dims += min(GB * 16, a.d); ++st_prn; }
                }
            }
            __syncthreads();
            if (tid == 0 && ic.p < npq) {
                issue_chunk<GB, LF>(a, smeta, plist, ic, slot, stage, bars);
                chunk_advance(ic, a, smeta, plist);
                ++issued;
            }
            ++unit;
        }
        if (aborted) break;
        // ---- phase B: remaining increments of the survivors (LF: all of them, on FP32) --
        if (NINC > 1 || LF != 0) {
            const int nS = s_cnt;
            for (int r0 = 0; r0 < nS; r0 += NQUAD) {
                const int sidx = r0 + quad;
                const bool act = sidx < nS;
                const Surv sv = act ? l0[sidx] : Surv{0, 0.f};
                const float *row = lbase + (int64_t)(cc.i0 + sv.idx) * 16 + lq * 4;
                // blocks from tail_nb0 on: one contiguous row of the row-major copy
                const float *trow = a.tail ? a.tail + ((int64_t)(unsigned)m.y + cc.i0 + sv.idx) * a.tail_w +
                                                 lq * 4 - (int64_t)a.tail_nb0 * 16
                                           : nullptr;
                float4 o[NLOAD > 0 ? NLOAD : 1];
#pragma unroll
                for (int u = 0; u < NLOAD; ++u) {
                    const int b = B0 + u;
                    const float *src = (trow && b >= a.tail_nb0) ? trow + b * 16 : row + (int64_t)b * bstride;
                    o[u] = act ? __ldg(reinterpret_cast<const float4 *>(src)) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                float p = LF ? 0.f : sv.p;
                bool alive = act;
#pragma unroll
                for (int j = LF ? 0 : 1; j < NINC; ++j) {
                    float part = 0.f;
#pragma unroll
                    for (int b = j * GB; b < (j + 1) * GB && b < NB; ++b) part += sqd4(qr[b], o[b - B0]);
                    part = quad_sum(part);
                    p += part;
                    if (j < NINC - 1 && alive && p > a.coef[j] * r2) {
                        alive = false;
                        if (STATS && lq == 0) { st_dims += min((j + 1) * GB * 16, a.d); ++st_prn; }
                    }
                }
                const bool take = alive && lq == 0 && p <= r2;
                if (STATS && alive && lq == 0) { st_dims += a.d; st_acc += take; }
                push(take, fl, &s_cntF, sv.idx, p);
            }
            __syncthreads();
        }
        // ---- merge --------------------------------------------------------------------
        const int nF = s_cntF;
        if (nF > 0)
            merge_topk<NT>(a, kq, fl, nF, (int64_t)(unsigned)m.y + cc.i0, fraw, fsort, top0, top1, &s_ntop, &s_cur, &s_r2);
        cc.i0 += a.tile;
        normalize(cc, a, smeta, plist);
    }
    if (aborted) {
        if (tid == 0) {
            atomicExch(a.err, (int)DADE_ETIMEOUT);
            for (int u = unit; u < issued; ++u)
                wait_bounded(su32(&bars[u % NSF]), (uint32_t)((u / NSF) & 1), 10000000ull);
        }
        return;
    }
    write_results<NT>(a, qi, s_ntop, s_cur ? top1 : top0);
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
    if (LF != 0 && a.lead_stats) {
        if (st_lead) atomicAdd(&s_lead, st_lead);
        __syncthreads();
        if (tid == 0) a.lead_stats[qi] = (int64_t)s_lead;
    }
}

// FDScanning: units of UB = 4 blocks per tile, q in registers.
template <int NT, int NB, bool STATS>
__global__ void __launch_bounds__(NT, 768 / NT) k_fd_fast(const ScanArgs a) {
    constexpr int NQUAD = NT / 4;
    constexpr int MAXIT = MAX_TILE / NQUAD;
    constexpr int UB = 4;
    constexpr int NU = (NB + UB - 1) / UB;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_cntF, s_ntop, s_cur;
    __shared__ float s_r2;
    __shared__ unsigned long long s_stats[4];

    const int tid = threadIdx.x, quad = tid >> 2, lq = tid & 3;
    const int64_t qi = cta_query(a);
    // this query's K and nprobe, within the batch's largest (a.k, a.nprobe: buffer sizes and strides)
    const int kq = a.q_k ? min(max(a.q_k[qi], 1), a.k) : a.k;
    const int npq = a.q_np ? min(max(a.q_np[qi], 0), a.nprobe) : a.nprobe;
    const SmemLayout L = layout(a.dp, a.tile, UB, a.ns, a.k, a.nprobe);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int4 *smeta = reinterpret_cast<int4 *>(smem + L.meta);
    float *stage = reinterpret_cast<float *>(smem + L.stage);
    Surv *fl = reinterpret_cast<Surv *>(smem + L.fl);
    unsigned long long *fraw = reinterpret_cast<unsigned long long *>(smem + L.fraw);
    unsigned long long *fsort = reinterpret_cast<unsigned long long *>(smem + L.fsort);
    unsigned long long *top0 = reinterpret_cast<unsigned long long *>(smem + L.top);
    unsigned long long *top1 = top0 + a.k;

    float4 qr[NB];
    load_q<NB>(a, qi, lq, qr);
    const int32_t *plist = a.probe + qi * a.pstride;
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

    Cur cc{0, 0, 0, npq};
    normalize(cc, a, smeta, plist);
    Cur ic = cc;
    int issued = 0;
    if (tid == 0)
        for (int s = 0; s < a.ns && ic.p < npq; ++s) {
            issue(a, smeta, plist, ic, s, stage, bars);
            advance(ic, NU, a, smeta, plist);
            ++issued;
        }
    unsigned long long st_cand = 0, st_acc = 0;
    int unit = 0;
    bool aborted = false;

    while (cc.p < npq) {
        const int4 m = meta_of(a, smeta, plist, cc.p);
        const int tn = min(a.tile, m.z - cc.i0);
        const int nit = (tn + NQUAD - 1) / NQUAD;
        if (tid == 0) s_cntF = 0;
        float acc[MAXIT];
#pragma unroll
        for (int it = 0; it < MAXIT; ++it) acc[it] = 0.f;
        float r2 = 0.f;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
            const int slot = unit % a.ns;
            if (!wait_block(su32(&bars[slot]), (uint32_t)((unit / a.ns) & 1), a.wait_ns, unit == 0 ? a.never : nullptr)) { aborted = true; break; }
            if (u == 0) r2 = s_r2;
            const float *st = stage + (size_t)slot * a.tile * UB * 16 + lq * 4;
#pragma unroll
            for (int it = 0; it < MAXIT; ++it) {
                const int c = quad + it * NQUAD;
                if (it < nit && c < tn) {
#pragma unroll
                    for (int b = 0; b < UB && u * UB + b < NB; ++b)
                        acc[it] += sqd4(qr[u * UB + b], *reinterpret_cast<const float4 *>(st + ((size_t)b * a.tile + c) * 16));
                }
            }
            __syncthreads();
            if (tid == 0 && ic.p < npq) {
                issue(a, smeta, plist, ic, slot, stage, bars);
                advance(ic, NU, a, smeta, plist);
                ++issued;
            }
            ++unit;
        }
        if (aborted) break;
#pragma unroll
        for (int it = 0; it < MAXIT; ++it) {
            if (it >= nit) break;
            const int c = quad + it * NQUAD;
            const float p = quad_sum(acc[it]);
            const bool act = c < tn;
            const bool take = act && lq == 0 && p <= r2;
            push(take, fl, &s_cntF, c, p);
            if (STATS && act && lq == 0) { ++st_cand; st_acc += take; }
        }
        __syncthreads();
        const int nF = s_cntF;
        if (nF > 0)
            merge_topk<NT>(a, kq, fl, nF, (int64_t)(unsigned)m.y + cc.i0, fraw, fsort, top0, top1, &s_ntop, &s_cur, &s_r2);
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
    write_results<NT>(a, qi, s_ntop, s_cur ? top1 : top0);
    if (STATS) {
        if (lq == 0) {
            atomicAdd(&s_stats[0], st_cand);
            atomicAdd(&s_stats[1], st_cand * (unsigned long long)a.d);
            atomicAdd(&s_stats[2], st_acc);
        }
        __syncthreads();
        if (tid < 4) a.stats[qi * 4 + tid] = (int64_t)s_stats[tid];
    }
}

template <typename K>
dade_status launch_k(K kern, const char *name, int threads, const ScanArgs &a, int64_t nq, size_t smem,
                     cudaStream_t s) {
    if (smem > 48 * 1024)
        DADE_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)nq, threads, smem, s>>>(a);
    return launch_check(name);
}

template <int NT, int GB, bool STATS, int LF>
dade_status dade_gb(const ScanArgs &a, int64_t nq, cudaStream_t s) {
    const FastLayout L = fast_layout(a.tile, ChunkRing<GB, LF>::SLOT, ChunkRing<GB, LF>::NSF, a.k, a.nprobe);
    return launch_k(k_dade_fast<NT, FNB, GB, STATS, LF>, LF ? "k_dade_fast<lead>" : "k_dade_fast", NT, a, nq,
                    L.total, s);
}

template <int NT, bool STATS, int LF>
dade_status dade_by_gb(const ScanArgs &a, int64_t nq, cudaStream_t s) {
    switch (a.gb) {
    case 1: return dade_gb<NT, 1, STATS, LF>(a, nq, s);
    case 2: return dade_gb<NT, 2, STATS, LF>(a, nq, s);
    case 4: return dade_gb<NT, 4, STATS, LF>(a, nq, s);
    default: return dade_gb<NT, 8, STATS, LF>(a, nq, s);
    }
}

template <int LF>
dade_status dade_fast_by_threads(const ScanArgs &a, int64_t nq, int threads, cudaStream_t s) {
    const bool st = a.stats != nullptr;
    if (threads == 256) return st ? dade_by_gb<256, true, LF>(a, nq, s) : dade_by_gb<256, false, LF>(a, nq, s);
    return st ? dade_by_gb<128, true, LF>(a, nq, s) : dade_by_gb<128, false, LF>(a, nq, s);
}

} // namespace
} // namespace dade
