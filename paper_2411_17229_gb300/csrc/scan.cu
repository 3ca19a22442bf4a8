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
// With a low-precision copy of the leading dims (LF = 1 BF16, 2 FP8), step 1
// stages that copy and its error norms instead, step 2 drops a candidate only
// on the certified margin test (lead_prunes), and step 3 starts again at the
// first increment on FP32 rows, so results equal those of the FP32 path.
//
// Every mbarrier wait is bounded (2 s on %globaltimer); on expiry the CTA
// records DADE_ETIMEOUT in the index's error word, waits (bounded) for its
// own copies in flight and exits without writing results.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "scan_common.cuh"

namespace dade {

namespace {
using namespace scanning;

template <int NT, bool FD, bool STATS, int LF>
__global__ void __launch_bounds__(NT, FD ? 1024 / NT : 768 / NT) k_scan(const ScanArgs a) {
    constexpr int NQUAD = NT / 4;              // candidates per pass
    constexpr int MAXIT = MAX_TILE / NQUAD;    // passes over a full tile
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_cnt[2], s_cntF, s_ntop, s_cur;
    __shared__ float s_r2;
    __shared__ unsigned long long s_stats[4], s_lead;

    const int tid = threadIdx.x, quad = tid >> 2, lq = tid & 3;
    const int64_t qi = cta_query(a);
    // this query's K and nprobe, within the batch's largest (a.k, a.nprobe: buffer sizes and strides)
    const int kq = a.q_k ? min(max(a.q_k[qi], 1), a.k) : a.k;
    const int npq = a.q_np ? min(max(a.q_np[qi], 0), a.nprobe) : a.nprobe;
    const SmemLayout L = layout(a.dp, a.tile, a.ub, a.ns, a.k, a.nprobe, LF != 0);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int4 *smeta = reinterpret_cast<int4 *>(smem + L.meta);
    float *qv = reinterpret_cast<float *>(smem + L.qv);
    float *qc = reinterpret_cast<float *>(smem + L.qc);      // LF: q' - c' of the first increment, then scales
    float *stage = reinterpret_cast<float *>(smem + L.stage);
    Surv *l0 = reinterpret_cast<Surv *>(smem + L.l0);
    Surv *l1 = reinterpret_cast<Surv *>(smem + L.l1);
    Surv *fl = reinterpret_cast<Surv *>(smem + L.fl);
    unsigned long long *fraw = reinterpret_cast<unsigned long long *>(smem + L.fraw);
    unsigned long long *fsort = reinterpret_cast<unsigned long long *>(smem + L.fsort);
    unsigned long long *top0 = reinterpret_cast<unsigned long long *>(smem + L.top);
    unsigned long long *top1 = top0 + a.k;

    const int32_t *plist = a.probe + qi * a.pstride + a.c0;
    // split mode: this CTA's part of the probe positions
    const int part = a.parts > 0 ? (int)(blockIdx.x % (unsigned)a.parts) : 0;
    const int pbeg = a.parts > 0 ? (int)((int64_t)a.nprobe * part / a.parts) : 0;
    const int pend = a.parts > 0 ? (int)((int64_t)a.nprobe * (part + 1) / a.parts) : npq;
    for (int k = tid; k < a.dp; k += NT) qv[k] = k < a.d ? a.q_rot[qi * a.q_stride + k] : 0.f;
    for (int p = tid; p < min(a.nprobe, PMETA); p += NT) {
        const ListMeta m = a.meta[plist[p]];
        smeta[p] = make_int4((int)(m.base >> 6), (int)m.slot, list_end(a, m.len), m.np);
    }
    if (tid == 0) {
        for (int s = 0; s < a.ns; ++s) mbar_init(su32(&bars[s]), 1);
        fence_mbar_init();
        s_ntop = 0;
        s_cur = 0;
        s_r2 = a.r2src ? a.r2src[qi * a.k + a.k - 1] : INFINITY;
    }
    if (STATS && tid < 4) s_stats[tid] = 0;
    if (tid == 0) s_lead = 0;
    __syncthreads();

    const int units = FD ? a.n_inc : 1;   // staged units per tile
    constexpr int ES = LeadFmt<LF>::ES;
    auto issue_unit = [&](const Cur &c, int slot) {
        if constexpr (LF != 0) {
            const int4 m = meta_of(a, smeta, plist, c.p);
            issue_lead<LF>(a, m, c.i0, min(a.tile, m.z - c.i0), a.gb, a.tile,
                           reinterpret_cast<unsigned char *>(stage + (size_t)slot * a.tile * a.ub * 16),
                           su32(&bars[slot]));
        } else {
            issue(a, smeta, plist, c, slot, stage, bars);
        }
    };
    Cur cc{pbeg, a.row_lo, 0, pend};
    normalize(cc, a, smeta, plist);
    Cur ic = cc;          // issue cursor (thread 0 only)
    int issued = 0;       // units issued (thread 0 only)
    if (tid == 0)
        for (int s = 0; s < a.ns && ic.p < pend; ++s) {
            issue_unit(ic, s);
            advance(ic, units, a, smeta, plist);
            ++issued;
        }
    unsigned long long st_cand = 0, st_dims = 0, st_acc = 0, st_prn = 0, st_lead = 0;
    int unit = 0;
    bool aborted = false;

    while (cc.p < pend) {
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
        bool quiet = false;   // DADE: no survivor and nothing accepted in this tile

        if (FD) {
            // ---- FDScanning: every increment staged, partials kept per lane ------
            float acc[MAXIT];
#pragma unroll
            for (int it = 0; it < MAXIT; ++it) acc[it] = 0.f;
            for (int j = 0; j < a.n_inc; ++j) {
                const int slot = unit % a.ns;
                if (!wait_block(su32(&bars[slot]), (uint32_t)((unit / a.ns) & 1), a.wait_ns, unit == 0 ? a.never : nullptr)) { aborted = true; break; }
                if (j == 0) r2 = s_r2;
                const float *st = stage + (size_t)slot * a.tile * a.ub * 16;
                const int b0 = j * a.ub, b1 = min(b0 + a.ub, a.nb);
#pragma unroll
                for (int it = 0; it < MAXIT; ++it) {
                    const int c = quad + it * NQUAD;
                    if (it < nit && c < tn) acc[it] += row_part(st + c * 16 + lq * 4, (int64_t)a.tile * 16, qv, b0, b1, lq, false);
                }
                __syncthreads();
                if (tid == 0 && ic.p < pend) {
                    issue_unit(ic, slot);
                    advance(ic, units, a, smeta, plist);
                    ++issued;
                }
                ++unit;
            }
            if (aborted) break;
#pragma unroll
            for (int it = 0; it < MAXIT; ++it) {
                if (it >= nit) break;
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
            // ---- phase A: increment 0 of the whole tile, streamed (bulk copy) ----------
            const int slot = unit % a.ns;
            if constexpr (LF != 0) {   // q' - c' of the first increment and its scales
                const int list = plist[cc.p];
                for (int k = tid; k < a.gb * 16; k += NT) qc[k] = __fsub_rn(qv[k], a.cent[(int64_t)list * a.dp + k]);
                for (int b = tid; b < a.gb; b += NT)
                    qc[a.dp + b] = LF == 2 ? a.lead_scale[(int64_t)list * a.lead_nb + b] : 1.f;
            }
            if (!wait_block(su32(&bars[slot]), (uint32_t)((unit / a.ns) & 1), a.wait_ns, unit == 0 ? a.never : nullptr)) { aborted = true; break; }
            r2 = s_r2;
            if constexpr (LF != 0) {
                const unsigned char *st = reinterpret_cast<const unsigned char *>(stage + (size_t)slot * a.tile * a.ub * 16);
                const float *se = reinterpret_cast<const float *>(st + (size_t)a.gb * a.tile * 16 * ES);
                const bool last0 = a.n_inc == 1;
                const int d0 = min(a.delta_d, a.d);
                const float thr = last0 ? r2 : a.coef[0] * r2;
                float qn = 0.f;
                for (int b = 0; b < a.gb; ++b) {
                    const float4 v = *reinterpret_cast<const float4 *>(qc + b * 16 + lq * 4);
                    qn = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, qn))));
                }
                qn += __shfl_xor_sync(0xffffffffu, qn, 1);
                qn += __shfl_xor_sync(0xffffffffu, qn, 2);
                const float qcn = sqrtf(qn);
                for (int it = 0; it < nit; ++it) {
                    const int c = quad + it * NQUAD;
                    const bool act = c < tn;
                    float p = 0.f;
                    if (act)
                        for (int b = 0; b < a.gb; ++b)
                            p += sqd4(*reinterpret_cast<const float4 *>(qc + b * 16 + lq * 4),
                                      lead4<LF>(st + ((size_t)b * a.tile * 16 + c * 16 + lq * 4) * ES, qc[a.dp + b]));
                    p += __shfl_xor_sync(0xffffffffu, p, 1);
                    p += __shfl_xor_sync(0xffffffffu, p, 2);
                    const bool lead = act && lq == 0;
                    const bool drop = lead && lead_prunes(p, se[c], qcn, thr);
                    push(lead && !drop, l0, &s_cnt[0], c, 0.f);
                    if (drop) {   // counted as the exact path counts it: pruned at d0, or rejected at D
                        ++st_lead;
                        if (STATS) { ++st_cand; st_dims += last0 ? a.d : d0; st_prn += !last0; }
                    } else if (STATS && lead) {
                        ++st_cand;
                    }
                }
            } else {
                // the staged unit holds the first ub blocks (a whole number of increments):
                // run every increment inside it, testing at each boundary; a candidate
                // that survives them all goes to phase B, or, if the unit reaches D, to
                // the exact compare
                const float *st = stage + (size_t)slot * a.tile * a.ub * 16;
                const int ninc_a = (min(a.ub, a.nb) + a.gb - 1) / a.gb;
                const bool all_staged = a.ub >= a.nb;
                for (int it = 0; it < nit; ++it) {
                    const int c = quad + it * NQUAD;
                    const bool act = c < tn;
                    float p = 0.f;
                    bool alive = act;
                    int pruned_at = -1;
                    for (int j = 0; j < ninc_a; ++j) {
                        const int b0 = j * a.gb, b1 = min(b0 + a.gb, a.nb);
                        float part = act ? row_part(st + (size_t)b0 * a.tile * 16 + c * 16 + lq * 4,
                                                    (int64_t)a.tile * 16, qv, b0, b1, lq, false)
                                         : 0.f;
                        part += __shfl_xor_sync(0xffffffffu, part, 1);
                        part += __shfl_xor_sync(0xffffffffu, part, 2);
                        p += part;
                        if (alive && b1 < a.nb && p > a.coef[j] * r2) {
                            alive = false;
                            pruned_at = j;
                        }
                    }
                    const bool lead = act && lq == 0;
                    const bool toF = lead && alive && all_staged && p <= r2;
                    const bool toN = lead && alive && !all_staged;
                    push(toF, fl, &s_cntF, c, p);
                    push(toN, l0, &s_cnt[0], c, p);
                    if (STATS && lead) {
                        ++st_cand;
                        if (!alive) { st_dims += min((pruned_at + 1) * a.delta_d, a.d); ++st_prn; }
                        else if (all_staged) { st_dims += a.d; st_acc += toF; }
                    }
                }
            }
            __syncthreads();
            if (tid == 0 && ic.p < pend) {
                issue_unit(ic, slot);
                advance(ic, units, a, smeta, plist);
                ++issued;
            }
            ++unit;
            // ---- phase B: the survivors' remaining blocks, loaded ahead in registers -----
            // Each quad owns one survivor and loads up to SPECB blocks of it at once (one
            // round trip), then runs the increments in order on registers: partial sum
            // over the increment's blocks, quad reduction, test P_d > coef_j r^2.  A
            // pruned candidate stops loading; a warp whose candidates are all pruned
            // stops early.  Candidates alive at d = D are accepted iff P_D <= r^2.
            const int nS = s_cnt[0];
            // a tile that leaves no survivor and accepts nothing skips the barriers of
            // phase B and the merge (every thread sees the same two zero counts; the
            // next tile's first barrier orders the rest)
            quiet = nS == 0 && s_cntF == 0;
            for (int r0 = 0; r0 < nS; r0 += NQUAD) {
                const int sidx = r0 + quad;
                const bool act = sidx < nS;
                const Surv sv = act ? l0[sidx] : Surv{0, 0.f};
                // after the prefilter (LF) every increment, the first included, runs on FP32
                // rows; otherwise phase B starts after the staged unit (ub blocks)
                const int sb = LF ? 0 : a.ub;
                float p = LF ? 0.f : sv.p, part = 0.f;
                bool alive = act;
                const float *row = lbase + (int64_t)(cc.i0 + sv.idx) * 16 + lq * 4;
                int jj = sb / a.gb, bend = min(sb + a.gb, a.nb);
                for (int wb = sb; wb < a.nb; wb += a.spec) {
                    if (!__any_sync(0xffffffffu, alive)) break;
                    float4 o[SPECB];
#pragma unroll
                    for (int u = 0; u < SPECB; ++u) {
                        const int bb = wb + u;
                        o[u] = (u < a.spec && bb < a.nb && alive)
                                   ? __ldg(reinterpret_cast<const float4 *>(row + (int64_t)bb * bstride))
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < SPECB; ++u) {
                        const int bb = wb + u;
                        if (u < a.spec && bb < a.nb) {
                            part += sqd4(*reinterpret_cast<const float4 *>(qv + bb * 16 + lq * 4), o[u]);
                            if (bb + 1 == bend) {        // end of increment jj
                                part += __shfl_xor_sync(0xffffffffu, part, 1);
                                part += __shfl_xor_sync(0xffffffffu, part, 2);
                                if (alive) {
                                    p += part;
                                    if (jj < a.n_inc - 1 && p > a.coef[jj] * r2) {
                                        alive = false;
                                        if (STATS && lq == 0) { st_dims += min((jj + 1) * a.delta_d, a.d); ++st_prn; }
                                    }
                                }
                                part = 0.f;
                                ++jj;
                                bend = min(bend + a.gb, a.nb);
                            }
                        }
                    }
                }
                const bool take = alive && lq == 0 && p <= r2;
                if (STATS && alive && lq == 0) { st_dims += a.d; st_acc += take; }
                push(take, fl, &s_cntF, sv.idx, p);
            }
            if (!quiet) __syncthreads();
        }

        // ---- merge accepted candidates into the K best ------------------------------
        const int nF = s_cntF;
        if (a.parts > 0) {   // split mode: r stays frozen; accepted keys go to the query's buffer
            __shared__ int s_abase;
            if (nF > 0) {
                if (tid == 0) s_abase = atomicAdd(&a.acnt[qi], nF);
                __syncthreads();
                for (int t = tid; t < nF; t += NT) {
                    const Surv f = fl[t];
                    const unsigned id = (unsigned)a.ids[(int64_t)(unsigned)m.y + cc.i0 + f.idx];
                    if (s_abase + t < a.cap)
                        a.acc[qi * a.cap + s_abase + t] = ((unsigned long long)__float_as_uint(f.p) << 32) | id;
                    else
                        atomicExch(a.err, (int)DADE_ENOMEM);   // accept buffer full: the call reports it
                }
            }
        } else if (nF > 0) {
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
                if (pos < kq) O[pos] = A[t];
            }
            for (int t = tid; t < nF; t += NT) {
                const int pos = t + lower_bound_u64(A, nt, fsort[t]);
                if (pos < kq) O[pos] = fsort[t];
            }
            __syncthreads();
            if (tid == 0) {
                const int nn = min(kq, nt + nF);
                s_ntop = nn;
                s_cur = cur ^ 1;
                s_r2 = nn == kq ? __uint_as_float((unsigned)(O[kq - 1] >> 32)) : INFINITY;
            }
        }
        if (!quiet) __syncthreads();
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
    for (int t = tid; a.parts == 0 && t < a.k; t += NT) {
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
        if (tid < 4) {
            if (a.parts > 0)   // added to the seed lists' counts by every part
                atomicAdd(reinterpret_cast<unsigned long long *>(&a.stats[qi * 4 + tid]), s_stats[tid]);
            else
                a.stats[qi * 4 + tid] = (int64_t)s_stats[tid];
        }
    }
    if (LF != 0 && a.lead_stats) {
        if (st_lead) atomicAdd(&s_lead, st_lead);
        __syncthreads();
        if (tid == 0) {
            if (a.parts > 0) atomicAdd(reinterpret_cast<unsigned long long *>(&a.lead_stats[qi]), s_lead);
            else a.lead_stats[qi] = (int64_t)s_lead;
        }
    }
}

template <int NT, bool FD, bool STATS, int LF>
dade_status launch(const ScanArgs &a, int64_t nq, size_t smem, cudaStream_t s) {
    DADE_TRY(kernel_smem((const void *)k_scan<NT, FD, STATS, LF>, smem));
    k_scan<NT, FD, STATS, LF><<<(unsigned)nq, NT, smem, s>>>(a);
    return launch_check(FD ? "k_scan<FD>" : (LF ? "k_scan<DADE, lead>" : "k_scan<DADE>"));
}

template <int NT, int LF>
dade_status launch_dade(const ScanArgs &a, int64_t nq, size_t smem, bool stats, cudaStream_t s) {
    return stats ? launch<NT, false, true, LF>(a, nq, smem, s) : launch<NT, false, false, LF>(a, nq, smem, s);
}

template <int NT>
dade_status launch_nt(const ScanArgs &a, int64_t nq, size_t smem, bool fd, bool stats, int lf, cudaStream_t s) {
    if (fd) return stats ? launch<NT, true, true, 0>(a, nq, smem, s) : launch<NT, true, false, 0>(a, nq, smem, s);
    if (lf == DADE_LEAD_BF16) return launch_dade<NT, 1>(a, nq, smem, stats, s);
    if (lf == DADE_LEAD_FP8) return launch_dade<NT, 2>(a, nq, smem, stats, s);
    return launch_dade<NT, 0>(a, nq, smem, stats, s);
}

} // namespace

dade_status scan_pipelined(const scanning::ScanArgs &a, int64_t nq, int threads, cudaStream_t s);
int pipe_depth_limit();
bool scan_fast_applies(const scanning::ScanArgs &a, bool fd);
dade_status scan_fast(const scanning::ScanArgs &a, int64_t nq, bool fd, int threads, int lf, cudaStream_t s);

dade_status scan(const dade_index *ix, int64_t nq, const ScanParams &p, cudaStream_t s) {
    if (nq == 0) return DADE_OK;
    if ((p.q_k || p.q_np) && ((p.schedule != DADE_SCHED_TILE && p.schedule != DADE_SCHED_ROUNDS) || p.parts > 0)) {
        set_error("per-query K and nprobe need the tile schedule or the row rounds");
        return DADE_EUNSUPPORTED;
    }
    if (p.schedule == DADE_SCHED_SEEDED && p.seed_lists > 0 && p.seed_lists < p.nprobe)
        return scan_seeded(ix, nq, p, s);
    if (p.schedule == DADE_SCHED_ROUNDS && p.parts == 0) return scan_rounds(ix, nq, p, s);
    ScanArgs a{};
    a.data = ix->data.as<float>();
    a.ids = ix->ids.as<int32_t>();
    a.meta = ix->meta.as<ListMeta>();
    a.q_rot = p.q_rot;
    a.probe = p.probe;
    a.out_ids = p.ids;
    a.out_d = p.dists;
    a.stats = p.stats;
    a.order = p.order;
    if (p.use_tail && ix->tail_nb0 > 0) {
        a.tail = ix->tail.as<float>();
        a.tail_nb0 = ix->tail_nb0;
        a.tail_w = ix->tail_w;
    }
    a.err = ix->errflag.as<int>();
    a.wait_ns = p.wait_ns > 0 ? (uint64_t)p.wait_ns : WAIT_NS;
    a.never = p.check_timeout ? ix->errflag.as<int>() + 3 : nullptr;
    a.q_k = p.q_k;
    a.q_np = p.q_np;
    a.q_stride = p.q_stride;
    a.nprobe = p.nprobe;
    if (p.parts > 0) {
        a.parts = p.parts;
        a.c0 = p.c0;
        a.r2src = p.r2src;
        a.acc = p.acc;
        a.acnt = p.acnt;
        a.cap = p.cap;
        a.row_lo = p.row_lo;
        a.row_hi = p.row_hi;
    }
    a.pstride = p.pstride > 0 ? p.pstride : p.nprobe;
    a.d = ix->d;
    a.dp = ix->dp;
    a.nb = ix->nb;
    a.k = p.k;
    a.tile = p.tile;
    a.ns = 2;
    a.spec = std::min(std::max(p.spec, 1), SPECB);
    const bool fd = p.mode == DADE_MODE_FD;
    if (fd) {
        a.gb = std::min(4, ix->nb);
        a.delta_d = a.gb * 16;
    } else {
        a.gb = std::min(p.delta_d / 16, ix->nb);
        a.delta_d = p.delta_d;
    }
    a.n_inc = (ix->nb + a.gb - 1) / a.gb;
    // blocks per staged unit: FDScanning and the prefilter one increment; the FP32
    // DADE tile kernel p.stage_dims (a whole number of increments, default one)
    a.ub = a.gb;
    if (!fd && !p.use_lead && p.stage_dims > a.delta_d) a.ub = std::min((p.stage_dims / 16) / a.gb * a.gb, ix->nb);
    for (int j = 0; j < DADE_MAX_DIM / DADE_BLOCK; ++j) a.coef[j] = j < p.n_inc ? p.coef[j] : INFINITY;
    const int lf = (!fd && p.use_lead) ? ix->lead_format : 0;
    if (lf) {
        a.lead = ix->lead.as<unsigned char>();
        a.lead_err = ix->lead_err.as<float>();
        a.lead_scale = ix->lead_scale.as<float>();
        a.cent = ix->cent.as<float>();
        a.lead_stats = p.lead_stats;
        a.lead_slots = ix->slots;
        a.lead_nb = ix->lead_nb;
    }
    const bool plain = a.ub == a.gb && a.parts == 0;   // the specialised kernels run neither mode
    if (!fd && !lf && plain && p.schedule == DADE_SCHED_PIPELINED && a.n_inc <= pipe_depth_limit())
        return scan_pipelined(a, nq, p.threads, s);
    if (scan_fast_applies(a, fd) && !p.generic && plain) return scan_fast(a, nq, fd, p.threads, lf, s);
    if (p.stage_ring >= 2) a.ns = std::min(p.stage_ring, 8);   // the tile kernel's ring depth
    const SmemLayout L = layout(a.dp, a.tile, a.ub, a.ns, a.k, a.nprobe, lf != 0);
    if (L.total > 227 * 1024) {
        set_error("scan configuration needs more than 227 KB of shared memory (reduce tile or delta_d)");
        return DADE_EUNSUPPORTED;
    }
    const int64_t ctas = nq * std::max(a.parts, 1);
    if (p.threads == 256) return launch_nt<256>(a, ctas, L.total, fd, p.stats != nullptr, lf, s);
    return launch_nt<128>(a, ctas, L.total, fd, p.stats != nullptr, lf, s);
}

} // namespace dade
