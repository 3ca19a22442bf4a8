// scan_pipe.cu -- pipelined DADE scan (Algorithm 1 with the Section 3.3 test
// inside the IVF loop of Section 3.4), one CTA per query.
//
// The sequential kernel (scan.cu) finishes a tile through all its increments
// before the next tile starts, so every increment costs a dependent global
// round trip.  Here the CTA keeps P = number of increments tiles in flight:
// at step s, tile s enters at increment 0 (its blocks were bulk-copied into
// shared memory NS steps earlier), tile s-1 runs increment 1, ..., tile
// s-P+1 runs its last increment and is merged into the K best.  All
// survivors' block rows that the step needs, from every tile in flight, are
// fetched together with cp.async into one shared buffer, so one round trip
// advances P tiles.  Work items of all tiles form one flat list that the
// quads (4 lanes per candidate, float4 loads, two shuffles) walk uniformly.
//
// Threshold schedule: a tile takes r^2 when it enters, which reflects the
// tiles merged by then, i.e. all tiles up to P earlier.  This is the tile
// schedule with a lag of P - 1 tiles (a stale threshold can only prune
// less); the oracle runs the same schedule for parity.
#include <algorithm>

#include "internal.cuh"
#include "scan_common.cuh"

namespace dade {

namespace {
using namespace scanning;

constexpr int PMAX = 8;   // deepest pipeline (increments per tile)

struct TileHdr {
    int4 m;         // list descriptor (see meta_of)
    int i0, tn;     // first candidate and size of the tile
    float r2;       // threshold taken when the tile entered
    int cnt[2];     // survivors in the two ping-pong lists
    int cntF;       // accepted candidates
    int pad[2];
};

struct PipeLayout {
    size_t meta, qv, stage, gbuf, lists, fin, hdr, fraw, fsort, top, total;
};

__host__ __device__ inline PipeLayout pipe_layout(int dp, int tile, int gb, int ns, int k, int nprobe, int P) {
    PipeLayout L;
    size_t o = 64;                                  // mbarriers (up to 8)
    L.meta = o;  o = align_up(o + sizeof(int4) * (size_t)min(nprobe, PMETA), 16);
    L.qv = o;    o = align_up(o + sizeof(float) * dp, 128);
    L.stage = o; o = align_up(o + sizeof(float) * (size_t)ns * tile * gb * 16, 128);
    L.gbuf = o;  o = align_up(o + sizeof(float) * (size_t)(P > 1 ? P - 1 : 0) * tile * gb * 16, 128);
    L.lists = o; o += sizeof(Surv) * 2 * (size_t)P * tile;
    L.fin = o;   o += sizeof(Surv) * (size_t)P * tile;
    L.hdr = o;   o = align_up(o + sizeof(TileHdr) * P, 16);
    L.fraw = o;  o += 8 * (size_t)pow2_at_least(tile);
    L.fsort = o; o += 8 * (size_t)pow2_at_least(tile);
    L.top = o;   o += 16 * (size_t)k;
    L.total = align_up(o, 128);
    return L;
}

template <int NT, bool STATS>
__global__ void __launch_bounds__(NT, 1024 / NT) k_scan_pipe(const ScanArgs a) {
    constexpr int NQUAD = NT / 4;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_ntop, s_cur, s_off[PMAX + 1];
    __shared__ float s_r2;
    __shared__ unsigned long long s_stats[4];

    const int tid = threadIdx.x, quad = tid >> 2, lq = tid & 3;
    const int64_t qi = cta_query(a);
    const int P = a.n_inc, T = a.tile, gb = a.gb;
    const PipeLayout L = pipe_layout(a.dp, T, gb, a.ns, a.k, a.nprobe, P);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    int4 *smeta = reinterpret_cast<int4 *>(smem + L.meta);
    float *qv = reinterpret_cast<float *>(smem + L.qv);
    float *stage = reinterpret_cast<float *>(smem + L.stage);
    float *gbuf = reinterpret_cast<float *>(smem + L.gbuf);
    Surv *lists = reinterpret_cast<Surv *>(smem + L.lists);     // [slot][parity][T]
    Surv *fin = reinterpret_cast<Surv *>(smem + L.fin);         // [slot][T]
    TileHdr *hdr = reinterpret_cast<TileHdr *>(smem + L.hdr);   // [slot]
    unsigned long long *fraw = reinterpret_cast<unsigned long long *>(smem + L.fraw);
    unsigned long long *fsort = reinterpret_cast<unsigned long long *>(smem + L.fsort);
    unsigned long long *top0 = reinterpret_cast<unsigned long long *>(smem + L.top);
    unsigned long long *top1 = top0 + a.k;

    const int32_t *plist = a.probe + qi * a.pstride;
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

    Cur cc{0, 0, 0, a.nprobe};   // next tile to enter
    normalize(cc, a, smeta, plist);
    Cur ic = cc;              // next tile whose first increment to issue (thread 0)
    int issued = 0;
    if (tid == 0)
        for (int s = 0; s < a.ns && ic.p < a.nprobe; ++s) {
            issue(a, smeta, plist, ic, s, stage, bars);
            advance(ic, 1, a, smeta, plist);
            ++issued;
        }
    unsigned long long st_cand = 0, st_dims = 0, st_acc = 0, st_prn = 0;
    int ne = 0;               // tiles entered so far (= stage units consumed)
    bool aborted = false;

    for (int s = 0;; ++s) {
        const bool enter = cc.p < a.nprobe;
        if (!enter && (ne == 0 || s > ne + P - 2)) break;   // every tile has left the pipeline
        // ---- step set-up (thread 0): entering tile, job offsets per level ----------
        if (tid == 0) {
            int off = 0;
            s_off[0] = 0;
            if (enter) {
                TileHdr &h = hdr[s % P];
                h.m = meta_of(a, smeta, plist, cc.p);
                h.i0 = cc.i0;
                h.tn = min(T, h.m.z - cc.i0);
                h.r2 = s_r2;
                h.cnt[0] = h.cnt[1] = 0;
                h.cntF = 0;
                off = h.tn;
            }
            s_off[1] = off;
            for (int j = 1; j < P; ++j) {
                const int t = s - j;
                if (t >= 0 && t < ne) {
                    TileHdr &h = hdr[t % P];
                    off += h.cnt[j & 1];
                    h.cnt[(j + 1) & 1] = 0;   // the list this level fills
                }
                s_off[j + 1] = off;
            }
        }
        __syncthreads();
        // ---- gathers of every tile in flight (levels >= 1) -------------------------
        const int g0 = s_off[1], gtot = s_off[P] - g0;
        const int chunks = gtot * gb * 4;
        for (int c = tid; c < chunks; c += NT) {
            const int g = c / (gb * 4) + g0, w = c % (gb * 4), b = w >> 2, qq = w & 3;
            int j = 1;
            while (g >= s_off[j + 1]) ++j;
            const int slot = (s - j) % P;
            const TileHdr &h = hdr[slot];
            const Surv sv = lists[((size_t)slot * 2 + (j & 1)) * T + (g - s_off[j])];
            const int blk = j * gb + b;
            if (blk < a.nb) {
                const float *src = list_base(a, h.m) + (int64_t)(h.i0 + sv.idx) * 16 + (int64_t)blk * h.m.w * 16 + qq * 4;
                cp_async16(su32(gbuf + ((size_t)(g - g0) * gb + b) * 16 + qq * 4), src);
            }
        }
        bool ok = true;
        if (enter && tid == 0)
            ok = (ne != 0 || a.never == nullptr || wait_word(a.never, a.wait_ns)) &&
                 wait_bounded(su32(&bars[ne % a.ns]), (uint32_t)((ne / a.ns) & 1), a.wait_ns);
        cp_async_wait_all();
        if (__syncthreads_or(!ok)) { aborted = true; break; }
        // ---- one increment for every work item of the step ---------------------------
        const int total = s_off[P];
        const float *st = stage + (size_t)(ne % a.ns) * T * gb * 16;
        const int nit = (total + NQUAD - 1) / NQUAD;
        for (int it = 0; it < nit; ++it) {
            const int g = quad + it * NQUAD;
            const bool act = g < total;
            int j = 0, slot = 0, idx = 0;
            float prev = 0.f, part = 0.f;
            if (act) {
                while (g >= s_off[j + 1]) ++j;
                slot = (s - j) % P;
                const int b0 = j * gb, b1 = min(b0 + gb, a.nb);
                const float *row;
                int64_t bstride;
                if (j == 0) {
                    idx = g;
                    row = st + (size_t)idx * 16 + lq * 4;
                    bstride = (int64_t)T * 16;
                } else {
                    const Surv sv = lists[((size_t)slot * 2 + (j & 1)) * T + (g - s_off[j])];
                    idx = sv.idx;
                    prev = sv.p;
                    row = gbuf + (size_t)(g - g0) * gb * 16 + lq * 4;
                    bstride = 16;
                }
                part = row_part(row, bstride, qv, b0, b1, lq, false);
            }
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            if (act && lq == 0) {
                TileHdr &h = hdr[slot];
                const float p = prev + part;
                if (STATS && j == 0) ++st_cand;
                if (j == P - 1) {
                    if (p <= h.r2) {
                        fin[(size_t)slot * T + atomicAdd(&h.cntF, 1)] = Surv{idx, p};
                        if (STATS) ++st_acc;
                    }
                    if (STATS) st_dims += a.d;
                } else if (!(p > a.coef[j] * h.r2)) {
                    lists[((size_t)slot * 2 + ((j + 1) & 1)) * T + atomicAdd(&h.cnt[(j + 1) & 1], 1)] = Surv{idx, p};
                } else if (STATS) {
                    st_dims += min((j + 1) * a.delta_d, a.d);
                    ++st_prn;
                }
            }
        }
        __syncthreads();
        if (enter) {
            if (tid == 0 && ic.p < a.nprobe) {
                issue(a, smeta, plist, ic, ne % a.ns, stage, bars);
                advance(ic, 1, a, smeta, plist);
                ++issued;
            }
            ++ne;
            cc.i0 += T;
            normalize(cc, a, smeta, plist);
        }
        // ---- the tile at the last level leaves: merge its accepted candidates ----------
        const int tl = s - (P - 1);
        if (tl >= 0 && tl < ne) {
            const int slot = tl % P;
            const int nF = hdr[slot].cntF;
            if (nF > 0)
                merge_topk<NT>(a, a.k, fin + (size_t)slot * T, nF, (int64_t)(unsigned)hdr[slot].m.y + hdr[slot].i0, fraw,
                               fsort, top0, top1, &s_ntop, &s_cur, &s_r2);
        }
        __syncthreads();
    }

    if (aborted) {
        if (tid == 0) {
            atomicExch(a.err, (int)DADE_ETIMEOUT);
            for (int u = ne; u < issued; ++u)
                wait_bounded(su32(&bars[u % a.ns]), (uint32_t)((u / a.ns) & 1), 10000000ull);
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
}

template <int NT, bool STATS>
dade_status launch_pipe(const ScanArgs &a, int64_t nq, size_t smem, cudaStream_t s) {
    DADE_TRY(kernel_smem((const void *)k_scan_pipe<NT, STATS>, smem));
    k_scan_pipe<NT, STATS><<<(unsigned)nq, NT, smem, s>>>(a);
    return launch_check("k_scan_pipe");
}

} // namespace

int pipe_depth_limit() { return PMAX; }

dade_status scan_pipelined(const scanning::ScanArgs &a, int64_t nq, int threads, cudaStream_t s) {
    const PipeLayout L = pipe_layout(a.dp, a.tile, a.gb, a.ns, a.k, a.nprobe, a.n_inc);
    if (L.total > 227 * 1024) {
        set_error("pipelined scan needs more than 227 KB of shared memory (reduce tile)");
        return DADE_EUNSUPPORTED;
    }
    const bool st = a.stats != nullptr;
    if (threads == 256) return st ? launch_pipe<256, true>(a, nq, L.total, s) : launch_pipe<256, false>(a, nq, L.total, s);
    return st ? launch_pipe<128, true>(a, nq, L.total, s) : launch_pipe<128, false>(a, nq, L.total, s);
}

} // namespace dade
