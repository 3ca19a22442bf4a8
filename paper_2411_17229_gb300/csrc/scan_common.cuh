// scan_common.cuh -- device helpers shared by the scan kernels: PTX wrappers
// for mbarriers, bulk copies and cp.async, bounded waits, the per-probe list
// descriptors kept in shared memory, the tile cursor, and the shared-memory
// top-K merge.
#pragma once

#include <cmath>
#include <cstdint>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "internal.cuh"

namespace dade {
namespace scanning {

constexpr int MAX_TILE = 256;
constexpr int SPECB = 8;           // blocks of a surviving candidate loaded per round
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
    int q_stride, nprobe, pstride, d, dp, nb, k, tile, gb, n_inc, ns, delta_d, spec;   // pstride: probe row stride
    int ub;                      // blocks per staged unit (gb, or more for a deeper FP32 first stage)
    float coef[DADE_MAX_DIM / DADE_BLOCK];
    // low-precision leading blocks (prefilter of the first increment)
    const unsigned char *lead;   // residual codes, list region at slot * lead_nb * 16 * ES bytes
    const float *lead_err;       // [lead_nb][lead_slots] cumulative error norms, rounded up
    const float *lead_scale;     // [nc][lead_nb] FP8 scales
    const float *cent;           // [nc][dp] rotated centroids
    int64_t *lead_stats;         // [nq] candidates dropped by the prefilter, or null
    int64_t lead_slots;
    int lead_nb;
    const int32_t *order;        // CTA b runs query order[b] (null: query b)
    const float *tail;           // row-major copy of blocks >= tail_nb0 (null: none)
    int tail_nb0, tail_w;
    // split mode (parts > 0): r frozen at r2src[q][k - 1]; CTA b runs part b % parts of the
    // probe positions [c0, c0 + nprobe) of query b / parts and appends what it accepts
    // to acc[q][cap] (count acnt[q]) instead of keeping a K-best list
    const float *r2src;
    unsigned long long *acc;
    int *acnt;
    int64_t cap;
    int parts, c0;
    // row window of every list (split passes of the row-rounds schedule): rows
    // [row_lo, min(len, row_hi)) are scanned; row_hi = 0 means no upper limit
    int row_lo, row_hi;
    uint64_t wait_ns;            // limit of every bounded wait on a copy
    const int *never;            // failure-path check: a device word nothing sets (else NULL)
    // per-query K and nprobe (tile schedule, one CTA per query), or NULL for k and
    // nprobe; k and nprobe are then the batch's largest (output row stride, probe rows)
    const int32_t *q_k, *q_np;
};

// Rows of a list of `len` members that a pass scans end here.
__device__ __forceinline__ int list_end(const ScanArgs &a, int len) {
    return a.row_hi > 0 ? min(len, a.row_hi) : len;
}

// The query a CTA runs.
__device__ __forceinline__ int64_t cta_query(const ScanArgs &a) {
    const unsigned b = a.parts > 0 ? blockIdx.x / (unsigned)a.parts : blockIdx.x;
    return a.order ? (int64_t)a.order[b] : (int64_t)b;
}

// ---------------------------------------------------------- PTX helpers ----
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or ~0.1 ms pass, instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 100000;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
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
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// One thread of the block waits; the others park on the block barrier that
// follows (wait_block), which makes the bulk-copied data visible to them.
// Limits below 0.2 ms (a caller trying the timeout path) poll without the
// suspend hint, so that they can expire before a copy lands; below 1 us (the
// global timer's resolution) they poll exactly once.
__device__ inline bool wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (limit_ns < 1000ull) return mbar_test_wait(bar, parity);
    if (limit_ns < 200000ull) {
        const uint64_t t0 = gtimer();
        do {
            if (mbar_test_wait(bar, parity)) return true;
        } while (gtimer() - t0 <= limit_ns);
        return false;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try_wait(bar, parity))
        if (gtimer() - t0 > limit_ns) return false;
    return true;
}

// Failure-path check (DADE_FLAG_CHECK_TIMEOUT): a bounded wait on a device
// word that nothing sets.  It runs out after limit_ns, like a wait on a copy
// that never lands, and the caller takes its timeout path.
__device__ inline bool wait_word(const volatile int *w, uint64_t limit_ns) {
    const uint64_t t0 = gtimer();
    while (*w == 0)
        if (gtimer() - t0 > limit_ns) return false;
    return true;
}

// Block-wide wait for the mbarrier phase: thread 0 waits (bounded), then a
// barrier.  Returns false on every thread if the wait timed out.  With `never`
// set (a block's first wait under the failure-path check), thread 0 first
// waits on that word.
__device__ __forceinline__ bool wait_block(uint32_t bar, uint32_t parity, uint64_t limit_ns = WAIT_NS,
                                           const int *never = nullptr) {
    bool ok = true;
    if (threadIdx.x == 0) ok = (never == nullptr || wait_word(never, limit_ns)) && wait_bounded(bar, parity, limit_ns);
    return !__syncthreads_or(!ok);
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
    return make_int4((int)(m.base >> 6), (int)m.slot, list_end(a, m.len), m.np);
}

// Tile cursor: probe position p, first candidate i0, increment j; probe
// positions end at np (the query's nprobe, or the end of its part).
struct Cur {
    int p, i0, j, np;
};

__device__ __forceinline__ void normalize(Cur &c, const ScanArgs &a, const int4 *sm, const int32_t *plist) {
    while (c.p < c.np && c.i0 >= meta_of(a, sm, plist, c.p).z) {
        ++c.p;
        c.i0 = a.row_lo;
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
__device__ inline void issue(const ScanArgs &a, const int4 *sm, const int32_t *plist, const Cur &c, int slot, float *stage,
                      uint64_t *bars) {
    const int4 m = meta_of(a, sm, plist, c.p);
    const int tn = min(a.tile, m.z - c.i0);
    const int b0 = c.j * a.ub, b1 = min(b0 + a.ub, a.nb);
    const uint32_t bar = su32(&bars[slot]);
    mbar_expect_tx(bar, (uint32_t)((b1 - b0) * tn * 64));
    float *dst = stage + (size_t)slot * a.tile * a.ub * 16;
    const float *src = list_base(a, m) + (int64_t)c.i0 * 16;
    for (int b = b0; b < b1; ++b)
        bulk_g2s(su32(dst + (size_t)(b - b0) * a.tile * 16), src + (int64_t)b * m.w * 16, (uint32_t)(tn * 64), bar);
}

// ---------------------------------------------- low-precision leading blocks ----
// Bytes per code: BF16 (format 1) 2, FP8 e4m3 (format 2) 1.
template <int LF> struct LeadFmt { static constexpr int ES = LF == 1 ? 2 : 1; };

// Lane lq's four codes of one candidate block, dequantised to FP32.  BF16 is
// the high half of an FP32 word, so widening is exact; FP8 codes widen
// exactly to half, then to float, and the product with the block scale is
// rounded once (no fused multiply-add), as in the build's error norm.
template <int LF>
__device__ __forceinline__ float4 lead4(const unsigned char *p, float scale) {
    if constexpr (LF == 1) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    } else {
        const uint32_t u = *reinterpret_cast<const uint32_t *>(p);
        const float2 lo = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u & 0xffffu), __NV_E4M3)));
        const float2 hi = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u >> 16), __NV_E4M3)));
        return make_float4(__fmul_rn(scale, lo.x), __fmul_rn(scale, lo.y), __fmul_rn(scale, hi.x), __fmul_rn(scale, hi.y));
    }
}

// Certified test of the prefilter.  p_lead is the FP32 sum of squares of
// (q' - c') - dequant over the first increment's dims, e the stored error
// norm of those dims and qcn = ||q' - c'|| there.  The true distance of the
// candidate over the same dims is at least sqrt(p_lead) - e, less FP32
// rounding in forming q' - c', the differences and the sum, which the
// factors below cover (relative 2^-16 on the root, 2^-20 ||q' - c'||).  The
// candidate is dropped only when that lower bound squared exceeds thr by a
// further relative 2^-15, more than the rounding of the FP32 exact partial,
// so the exact test on FP32 data would drop it as well.
__device__ __forceinline__ bool lead_prunes(float p_lead, float e, float qcn, float thr) {
    const float L = sqrtf(p_lead) * (1.f - 0x1p-16f) - e - qcn * 0x1p-20f;
    const float lb = L > 0.f ? L * L : 0.f;
    return lb > thr * (1.f + 0x1p-15f);
}

// Queue the prefilter unit of a tile: gb blocks of tn codes (tn * 16 * ES
// bytes each) plus the tile's error norms (rounded up to a multiple of 4
// slots; the padded slots exist in every list).  dst layout: block b at
// b * cap * 16 * ES bytes, norms at gb * cap * 16 * ES.
template <int LF>
__device__ inline void issue_lead(const ScanArgs &a, int4 m, int c0, int cn, int gb, int cap, unsigned char *dst,
                                  uint32_t bar) {
    constexpr int ES = LeadFmt<LF>::ES;
    const int cn4 = (cn + 3) & ~3;
    mbar_expect_tx(bar, (uint32_t)(gb * cn * 16 * ES + cn4 * 4));
    const int64_t slot = (int64_t)(unsigned)m.y;
    const unsigned char *src = a.lead + (slot * a.lead_nb * 16 + (int64_t)c0 * 16) * ES;
    for (int b = 0; b < gb; ++b)
        bulk_g2s(su32(dst + (size_t)b * cap * 16 * ES), src + (int64_t)b * m.w * 16 * ES, (uint32_t)(cn * 16 * ES), bar);
    bulk_g2s(su32(dst + (size_t)gb * cap * 16 * ES), a.lead_err + (int64_t)(gb - 1) * a.lead_slots + slot + c0,
             (uint32_t)(cn4 * 4), bar);
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
    size_t meta, qv, qc, stage, l0, l1, fl, fraw, fsort, top, total;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
__host__ __device__ inline int pow2_at_least(int x) {
    int n = 1;
    while (n < x) n <<= 1;
    return n;
}

__host__ __device__ inline SmemLayout layout(int dp, int tile, int gb, int ns, int k, int nprobe, bool lead = false) {
    SmemLayout L;
    size_t o = 64;                                  // mbarriers (up to 8)
    L.meta = o;  o = align_up(o + sizeof(int4) * (size_t)min(nprobe, PMETA), 16);
    L.qv = o;    o = align_up(o + sizeof(float) * dp, 128);
    L.qc = o;    o = align_up(o + (lead ? sizeof(float) * (dp + 64) : 0), 128);   // q' - c', then <= 64 block scales
    L.stage = o; o = align_up(o + sizeof(float) * (size_t)ns * tile * gb * 16, 128);
    L.l0 = o;    o += sizeof(Surv) * tile;
    L.l1 = o;    o += sizeof(Surv) * tile;
    L.fl = o;    o += sizeof(Surv) * tile;
    L.fraw = o;  o += 8 * (size_t)pow2_at_least(tile);
    L.fsort = o; o += 8 * (size_t)pow2_at_least(tile);
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


__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Merge the nF accepted candidates fl[0..nF) of the tile whose ids start at
// slot `id0` into the query's kq-best list (rank sort, then merge by rank);
// refresh s_r2 from the kq-th entry.  Every thread of the block calls it; nF is
// uniform.  Ends with a barrier.
template <int NT>
__device__ inline void merge_topk(const ScanArgs &a, int kq, const Surv *fl, int nF, int64_t id0,
                                  unsigned long long *fraw, unsigned long long *fsort, unsigned long long *top0,
                                  unsigned long long *top1, int *s_ntop, int *s_cur, float *s_r2) {
    const int tid = threadIdx.x;
    const int N = nF > 64 ? pow2_at_least(nF) : nF;
    for (int t = tid; t < N; t += NT) {
        unsigned long long key = ~0ull;
        if (t < nF) {
            const Surv f = fl[t];
            key = ((unsigned long long)__float_as_uint(f.p) << 32) | (unsigned)a.ids[id0 + f.idx];
        }
        fraw[t] = key;
    }
    __syncthreads();
    if (nF > 64) {   // bitonic sort of the padded keys, in place
        for (int k = 2; k <= N; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = tid; t < N; t += NT) {
                    const int u = t ^ j;
                    if (u > t) {
                        const unsigned long long x = fraw[t], y = fraw[u];
                        if ((x > y) == ((t & k) == 0)) { fraw[t] = y; fraw[u] = x; }
                    }
                }
                __syncthreads();
            }
        fsort = fraw;
    } else {         // rank sort: keys are distinct (ids are unique)
        for (int t = tid; t < nF; t += NT) {
            const unsigned long long kk = fraw[t];
            int r = 0;
            for (int u = 0; u < nF; ++u) r += fraw[u] < kk;
            fsort[r] = kk;
        }
        __syncthreads();
    }
    const int nt = *s_ntop, cur = *s_cur;
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
        *s_ntop = nn;
        *s_cur = cur ^ 1;
        *s_r2 = nn == kq ? __uint_as_float((unsigned)(O[kq - 1] >> 32)) : INFINITY;
    }
    __syncthreads();
}

// Results of one query (ids, squared distances; -1 / +inf past the found ones).
template <int NT>
__device__ inline void write_results(const ScanArgs &a, int64_t qi, int nt, const unsigned long long *R) {
    for (int t = threadIdx.x; t < a.k; t += NT) {
        int64_t id = -1;
        float dv = INFINITY;
        if (t < nt) {
            id = (int64_t)(unsigned)(R[t] & 0xffffffffu);
            dv = __uint_as_float((unsigned)(R[t] >> 32));
        }
        a.out_ids[qi * a.k + t] = id;
        a.out_d[qi * a.k + t] = dv;
    }
}

} // namespace scanning
} // namespace dade
