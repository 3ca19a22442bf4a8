// tc_gemm.cu -- FP32-accurate GEMM on the fifth-generation tensor cores
// (tcgen05.mma, kind::tf32, accumulator in tensor memory) for the two dense
// contractions of the path: the PCA rotation x' = W^T (x - mu) of queries and
// base vectors (Section 3.2) and the query x centroid inner products of the
// coarse probe (Section 3.4).
//
// C[m][n] = sum_k a(m, k) b(n, k), a(m, k) = A[m * lda + k] - mu[k] (mu
// optional), b(n, k) = B[n * ldb + k]: both operands K-major.  3xTF32: every
// operand value x is split into hi = tf32(x) and lo = tf32(x - hi) (round to
// nearest), and C = Ahi Bhi + Ahi Blo + Alo Bhi is accumulated in FP32 in
// tensor memory; the dropped Alo Blo term is below 2^-22 of |a||b|.
//
// One CTA of 128 threads owns a 128 x 128 tile of C.  K advances in chunks of
// 32: the threads stage the chunk of A and of B, split, into shared memory in
// the canonical K-major layout without swizzle (core matrices of 8 rows x 16
// bytes, 16 B between the rows of a core matrix, 128 B between core matrices
// adjacent in K, 1 KB between 8-row groups), then one thread issues 4 k-steps
// x 3 MMAs of M = 128, N = 128, K = 8 and commits them to an mbarrier, which
// every thread waits on (bounded) before the buffers are rewritten.  The
// chunk's accumulator occupies 128 lanes x 128 FP32 columns of tensor memory;
// warp w reads lanes 32w .. 32w + 31 (its rows of C) 16 columns at a time
// with tcgen05.ld and adds them to FP32 registers.
#include <algorithm>

#include "internal.cuh"
#include "scan_common.cuh"

namespace dade {

namespace {
using namespace scanning;

constexpr int TM = 128, TN = 128, TK = 32;
constexpr uint32_t TMEM_COLS = 128;
constexpr uint32_t CORE_LBO = 128, CORE_SBO = 1024;   // bytes
constexpr int OP_WORDS = TM * TK;                     // 32-bit words per staged operand (16 KB)
constexpr size_t TC_SMEM = 4 * sizeof(uint32_t) * OP_WORDS;

// Instruction descriptor of kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N / 8 at bits 17-22,
// M / 16 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

// Shared-memory matrix descriptor: start address / 16 (bits 0-13), leading
// (K) byte offset / 16 (bits 16-29), stride (M/N) byte offset / 16 (bits
// 32-45), the fixed 0b001 at bits 46-48, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(CORE_LBO >> 4) << 16) |
           ((uint64_t)(CORE_SBO >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Rows [r0, r0 + 128) x dims [k0, k0 + 32) of a row-major FP32 matrix (minus
// mu), split into hi / lo TF32 words in the core-matrix layout.  Unit e
// (4 consecutive dims of one row) of 1024: row r0 + 8 (e / 64) + e % 8, dims
// k0 + 4 ((e / 8) % 8).  Out-of-range rows and dims read as 0.
__device__ __forceinline__ void stage(const float *__restrict__ X, int64_t nrows, int ld, int kdim, int64_t r0,
                                      int k0, const float *__restrict__ mu, uint32_t *hi, uint32_t *lo) {
#pragma unroll 2
    for (int i = 0; i < 8; ++i) {
        const int e = threadIdx.x + 128 * i;
        const int rr = e & 7, c = (e >> 3) & 7, g = e >> 6;
        const int64_t r = r0 + g * 8 + rr;
        const int k = k0 + c * 4;
        uint32_t h[4], l[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float v = 0.f;
            if (r < nrows && k + t < kdim) {
                v = X[r * ld + k + t];
                if (mu) v = __fsub_rn(v, mu[k + t]);
            }
            h[t] = tf32_rna(v);
            l[t] = tf32_rna(__fsub_rn(v, __uint_as_float(h[t])));
        }
        const int off = (g * (int)CORE_SBO + c * (int)CORE_LBO + rr * 16) / 4;
        *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// The accumulated tile (thread tid holds row m0 + tid in acc[]) leaves
// through shared memory in two halves of 64 columns, so that the global
// stores are row-contiguous.  EPI 1 turns inner products into distances.
template <int EPI>
__device__ __forceinline__ void store_tile(const float (&acc)[TN], float *tile, int64_t m0, int n0, int64_t M, float an,
                                           const float *__restrict__ bnorm, float *__restrict__ out, int64_t ldo,
                                           int ncols) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            const float c = acc[h * 64 + j];
            float v = c;
            if (EPI == 1) {
                const int n = n0 + h * 64 + j;
                v = fmaxf(fmaf(-2.f, c, an + (n < ncols ? bnorm[n] : 0.f)), 0.f);
            }
            tile[tid * 65 + j] = v;
        }
        __syncthreads();
        for (int idx = tid; idx < TM * 64; idx += 128) {
            const int r = idx >> 6, c = idx & 63;
            const int64_t orow = m0 + r;
            const int n = n0 + h * 64 + c;
            if (orow < M && n < ncols) out[orow * ldo + n] = tile[r * 65 + c];
        }
    }
}

// EPI 0: out[m][n] = C[m][n].  EPI 1 (probe distances):
// out[m][n] = max(0, ||a_m||^2 + bnorm[n] - 2 C[m][n]), ||a_m||^2 summed in
// FP32 in k_sqnorm_rows' order (see the epilogue).
template <int EPI>
__global__ void __launch_bounds__(128) k_tc_direct(const float *__restrict__ A, int64_t M, int lda,
                                                 const float *__restrict__ mu, const float *__restrict__ B, int nb_rows,
                                                 int ldb, int K, const float *__restrict__ bnorm,
                                                 float *__restrict__ out, int64_t ldo, int ncols, int *err) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    uint32_t *ahi = reinterpret_cast<uint32_t *>(tc_smem);
    uint32_t *alo = ahi + OP_WORDS, *bhi = alo + OP_WORDS, *blo = bhi + OP_WORDS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * TN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(su32(&bar), 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    // Per K-chunk: the two cross products (small) first, then the main
    // product, into a fresh accumulator; the chunk's result is added in FP32
    // registers (round to nearest).  Each output then carries the rounding of
    // 4 main MMAs, not of all 3 K / 8, so the result is FP32-accurate.
    float acc[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[j] = 0.f;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    uint32_t phase = 0;
    for (int k0 = 0; k0 < K; k0 += TK) {
        stage(A, M, lda, K, m0, k0, mu, ahi, alo);
        stage(B, nb_rows, ldb, K, n0, k0, nullptr, bhi, blo);
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < TK / 8; ++s) {
                const uint32_t koff = (uint32_t)s * 2 * CORE_LBO;   // K = 8 TF32 = two core matrices
                tc_mma(tmem, smem_desc(su32(ahi) + koff), smem_desc(su32(blo) + koff), s != 0);
                tc_mma(tmem, smem_desc(su32(alo) + koff), smem_desc(su32(bhi) + koff), 1u);
            }
#pragma unroll
            for (int s = 0; s < TK / 8; ++s) {
                const uint32_t koff = (uint32_t)s * 2 * CORE_LBO;
                tc_mma(tmem, smem_desc(su32(ahi) + koff), smem_desc(su32(bhi) + koff), 1u);
            }
            tc_commit(su32(&bar));
        }
        bool done = true;
        if (tid == 0) done = wait_bounded(su32(&bar), phase, WAIT_NS);
        if (__syncthreads_or(!done)) {
            ok = false;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            tc_ld16(trow + (uint32_t)c0, r);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(r[j]);
        }
    }
    if (!ok) {   // let the MMAs in flight finish (bounded) before the tensor memory is released
        if (tid == 0) {
            wait_bounded(su32(&bar), phase, 10000000ull);
            atomicExch(err, (int)DADE_ETIMEOUT);
        }
    } else {
        // thread tid owns row m0 + tid; the operand buffers are free (every
        // MMA has completed) and hold the outgoing tile.  ||a_m||^2 is summed
        // exactly as k_sqnorm_rows sums it for dade_probe (lane-strided FMAs
        // by one warp per row, then an xor-shuffle tree), so both probes
        // produce the same bits and order near-tied lists alike.
        float an = 0.f;
        if (EPI == 1)
            for (int i = 0; i < 32; ++i) {
                const int64_t r = m0 + warp * 32 + i;
                float s = 0.f;
                if (r < M)
                    for (int k = lane; k < K; k += 32) s = fmaf(A[r * lda + k], A[r * lda + k], s);
                for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == i) an = s;
            }
        store_tile<EPI>(acc, reinterpret_cast<float *>(tc_smem), m0, n0, M, an, bnorm, out, ldo, ncols);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

template <int EPI>
dade_status launch_direct(const float *A, int64_t M, int lda, const float *mu, const float *B, int nb_rows, int ldb, int K,
                      const float *bnorm, float *out, int64_t ldo, int ncols, int *err, cudaStream_t s) {
    DADE_TRY(kernel_smem((const void *)k_tc_direct<EPI>, TC_SMEM));
    dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)((ncols + TN - 1) / TN));
    k_tc_direct<EPI><<<grid, 128, TC_SMEM, s>>>(A, M, lda, mu, B, nb_rows, ldb, K, bnorm, out, ldo, ncols, err);
    return launch_check(EPI == 0 ? "k_tc_direct<rotate>" : "k_tc_direct<distances>");
}


// ---- pre-split operand images and the pipelined kernel ----------------------------
// Image of an operand (rows R, dims K): tiles of 128 rows x 32 dims, tile
// (rt, kc) at words ((rt * nkc + kc) * 2) * 4096: the hi words (16 KB) then
// the lo words, each in the core-matrix layout of stage().  One bulk copy of
// 32 KB moves a tile's operand into shared memory.
constexpr int IMG_WORDS = 2 * OP_WORDS;   // one tile: hi + lo

__global__ void __launch_bounds__(128) k_tc_image(const float *__restrict__ X, int64_t nrows, int ld, int K,
                                                  const float *__restrict__ mu, int nkc, uint32_t *__restrict__ img) {
    const int64_t rt = blockIdx.x;
    const int kc = blockIdx.y;
    uint32_t *hi = img + (rt * nkc + kc) * (int64_t)IMG_WORDS;
    stage(X, nrows, ld, K, rt * TM, kc * TK, mu, hi, hi + OP_WORDS);
}

constexpr size_t PIPE_STAGE = 2 * sizeof(uint32_t) * IMG_WORDS;   // A and B tile of one chunk: 64 KB
constexpr size_t PIPE_SMEM = 2 * PIPE_STAGE;                        // two stages
constexpr uint32_t PIPE_TMEM_COLS = 2 * TN;                         // two accumulator regions

// C tile (blockIdx.x, blockIdx.y) from operand images.  Thread 0 issues the
// bulk copies (two stages in flight) and the MMAs; chunk c accumulates into
// tensor-memory region c % 2 while every warp drains region (c - 1) % 2 into
// FP32 registers, so copies, MMAs and the register sums overlap.  mbarriers:
// full[s] (copies of stage s landed), done[s] (MMAs reading stage s and
// writing region s completed), tfree[s] (all 128 threads finished reading
// region s).  Every wait is bounded; on expiry the CTA records DADE_ETIMEOUT,
// waits (bounded) for the MMAs it issued, frees its tensor memory and exits.
template <int EPI>
__global__ void __launch_bounds__(128, 1) k_tc_pipe(const uint32_t *__restrict__ aimg, int64_t M,
                                                    const uint32_t *__restrict__ bimg, int nkc,
                                                    const float *__restrict__ anorm, const float *__restrict__ bnorm,
                                                    float *__restrict__ out, int64_t ldo, int ncols, int *err) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t full[2], done[2], tfree[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t mt = blockIdx.x;
    const int nt = blockIdx.y;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "r"(PIPE_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(su32(&full[i]), 1);
            mbar_init(su32(&done[i]), 1);
            mbar_init(su32(&tfree[i]), 128);
        }
        fence_mbar_init();
        s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t sbase = su32(tc_smem);

    auto copy_chunk = [&](int c) {   // thread 0
        const int st = c & 1;
        const uint32_t bar = su32(&full[st]);
        mbar_expect_tx(bar, (uint32_t)PIPE_STAGE);
        bulk_g2s(sbase + (uint32_t)(st * PIPE_STAGE), aimg + (mt * nkc + c) * (int64_t)IMG_WORDS,
                 (uint32_t)(PIPE_STAGE / 2), bar);
        bulk_g2s(sbase + (uint32_t)(st * PIPE_STAGE + PIPE_STAGE / 2), bimg + ((int64_t)nt * nkc + c) * IMG_WORDS,
                 (uint32_t)(PIPE_STAGE / 2), bar);
    };
    int issued = 0;                  // chunks whose MMAs thread 0 committed
    auto mma_chunk = [&](int c) {    // thread 0, after the copies of chunk c landed
        const int st = c & 1;
        const uint32_t a_hi = sbase + (uint32_t)(st * PIPE_STAGE), a_lo = a_hi + OP_WORDS * 4;
        const uint32_t b_hi = a_hi + IMG_WORDS * 4, b_lo = b_hi + OP_WORDS * 4;
        const uint32_t d = tmem + (uint32_t)(st * TN);
        tc_fence_after();
#pragma unroll
        for (int s = 0; s < TK / 8; ++s) {
            const uint32_t koff = (uint32_t)s * 2 * CORE_LBO;
            tc_mma(d, smem_desc(a_hi + koff), smem_desc(b_lo + koff), s != 0);
            tc_mma(d, smem_desc(a_lo + koff), smem_desc(b_hi + koff), 1u);
        }
#pragma unroll
        for (int s = 0; s < TK / 8; ++s) {
            const uint32_t koff = (uint32_t)s * 2 * CORE_LBO;
            tc_mma(d, smem_desc(a_hi + koff), smem_desc(b_hi + koff), 1u);
        }
        tc_commit(su32(&done[st]));
        issued = c + 1;
    };
    auto fail = [&]() { *(volatile int *)&s_abort = 1; };

    if (tid == 0) {
        for (int c = 0; c < 2 && c < nkc; ++c) copy_chunk(c);
        if (nkc > 0) {
            if (wait_bounded(su32(&full[0]), 0, WAIT_NS)) mma_chunk(0);
            else fail();
        }
    }
    float acc[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[j] = 0.f;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c = 0; c < nkc; ++c) {
        const int st = c & 1;
        if (tid == 0 && c + 1 < nkc && !*(volatile int *)&s_abort) {
            const int s1 = (c + 1) & 1;
            bool ok = wait_bounded(su32(&full[s1]), (uint32_t)(((c + 1) >> 1) & 1), WAIT_NS);
            if (ok && c + 1 >= 2) ok = wait_bounded(su32(&tfree[s1]), (uint32_t)(((c - 1) >> 1) & 1), WAIT_NS);
            if (ok) mma_chunk(c + 1);
            else fail();
        }
        if (*(volatile int *)&s_abort || !wait_bounded(su32(&done[st]), (uint32_t)((c >> 1) & 1), WAIT_NS)) {
            fail();
            break;
        }
        tc_fence_after();
#pragma unroll
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            tc_ld16(trow + (uint32_t)(st * TN + c0), r);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(r[j]);
        }
        tc_fence_before();
        mbar_arrive(su32(&tfree[st]));
        if (tid == 0 && c + 2 < nkc) copy_chunk(c + 2);   // the MMAs of chunk c are done: stage st is free
    }
    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            // MMAs committed for chunks [0, issued): let the unobserved ones finish
            for (int c = 0; c < issued; ++c) wait_bounded(su32(&done[c & 1]), (uint32_t)((c >> 1) & 1), 10000000ull);
            atomicExch(err, (int)DADE_ETIMEOUT);
        }
    } else {
        const int64_t row = mt * TM + tid;
        const float an = (EPI == 1 && row < M) ? anorm[row] : 0.f;
        store_tile<EPI>(acc, reinterpret_cast<float *>(tc_smem), mt * TM, nt * TN, M, an, bnorm, out, ldo, ncols);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PIPE_TMEM_COLS)
                     : "memory");
}

int chunks_of(int K) { return (K + TK - 1) / TK; }

dade_status build_image(const float *X, int64_t nrows, int ld, int K, const float *mu, DevBuf &img, cudaStream_t s) {
    const int64_t rt = (nrows + TM - 1) / TM;
    const int nkc = chunks_of(K);
    DADE_TRY(img.ensure(sizeof(uint32_t) * (size_t)(rt * nkc) * IMG_WORDS));
    if (rt == 0 || nkc == 0) return DADE_OK;
    k_tc_image<<<dim3((unsigned)rt, (unsigned)nkc), 128, 0, s>>>(X, nrows, ld, K, mu, nkc, img.as<uint32_t>());
    return launch_check("k_tc_image");
}

template <int EPI>
dade_status launch_pipe(const uint32_t *aimg, int64_t M, const uint32_t *bimg, int K, const float *anorm,
                        const float *bnorm, float *out, int64_t ldo, int ncols, int *err, cudaStream_t s) {
    DADE_TRY(kernel_smem((const void *)k_tc_pipe<EPI>, PIPE_SMEM));
    dim3 grid((unsigned)((M + TM - 1) / TM), (unsigned)((ncols + TN - 1) / TN));
    k_tc_pipe<EPI><<<grid, 128, PIPE_SMEM, s>>>(aimg, M, bimg, chunks_of(K), anorm, bnorm, out, ldo, ncols, err);
    return launch_check(EPI == 0 ? "k_tc_pipe<rotate>" : "k_tc_pipe<distances>");
}

__global__ void k_sqnorm_rows(const float *__restrict__ X, int64_t n, int ld, int kdim, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n) return;
    float s = 0.f;
    for (int k = lane; k < kdim; k += 32) s = fmaf(X[w * ld + k], X[w * ld + k], s);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[w] = s;
}

} // namespace

// Operand images of the index (rotated centroids, W^T), built once.
dade_status prepare_tensor_operands(dade_index *ix, cudaStream_t s) {
    DADE_TRY(build_image(ix->cent.as<float>(), ix->nc, ix->dp, ix->d, nullptr, ix->cent_img, s));
    return build_image(ix->WT32.as<float>(), ix->dp, ix->dp, ix->d, nullptr, ix->wt_img, s);
}

// Queries (a batch): image of x - mu, then the pipelined GEMM against W^T.
dade_status rotate(const dade_index *ix, const float *x, int64_t n, int32_t out_stride, float *out, cudaStream_t s) {
    if (n == 0) return DADE_OK;
    const int cols = std::min<int>(out_stride, ix->dp);
    DADE_TRY(build_image(x, n, ix->d, ix->d, ix->mu32.as<float>(), ws(ix).aimg, s));
    return launch_pipe<0>(ws(ix).aimg.as<uint32_t>(), n, ix->wt_img.as<uint32_t>(), ix->d, nullptr, nullptr, out,
                          out_stride, cols, ix->errflag.as<int>(), s);
}

// Base vectors at build time (no image: it would double the data in memory).
dade_status rotate_direct(const dade_index *ix, const float *x, int64_t n, int32_t out_stride, float *out,
                          cudaStream_t s) {
    if (n == 0) return DADE_OK;
    const int cols = std::min<int>(out_stride, ix->dp);
    return launch_direct<0>(x, n, ix->d, ix->mu32.as<float>(), ix->WT32.as<float>(), ix->dp, ix->dp, ix->d, nullptr,
                            out, out_stride, cols, ix->errflag.as<int>(), s);
}

dade_status probe_distances(const dade_index *ix, const float *q_rot, int64_t nq, int32_t q_stride, float *dist,
                            cudaStream_t s) {
    if (nq == 0) return DADE_OK;
    DADE_TRY(build_image(q_rot, nq, q_stride, ix->d, nullptr, ws(ix).aimg, s));
    DADE_TRY(ws(ix).anorm.ensure(sizeof(float) * (size_t)nq));
    k_sqnorm_rows<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, s>>>(q_rot, nq, q_stride, ix->d,
                                                                   ws(ix).anorm.as<float>());
    DADE_TRY(launch_check("k_sqnorm_rows"));
    return launch_pipe<1>(ws(ix).aimg.as<uint32_t>(), nq, ix->cent_img.as<uint32_t>(), ix->d,
                          ws(ix).anorm.as<float>(), ix->cnorm.as<float>(), dist, ix->nc, ix->nc,
                          ix->errflag.as<int>(), s);
}

// Without workspace (dade_probe_noalloc): operands staged by the threads.
dade_status probe_distances_direct(const dade_index *ix, const float *q_rot, int64_t nq, int32_t q_stride, float *dist,
                                   cudaStream_t s) {
    if (nq == 0) return DADE_OK;
    return launch_direct<1>(q_rot, nq, q_stride, nullptr, ix->cent.as<float>(), ix->nc, ix->dp, ix->d,
                            ix->cnorm.as<float>(), dist, ix->nc, ix->nc, ix->errflag.as<int>(), s);
}

} // namespace dade
