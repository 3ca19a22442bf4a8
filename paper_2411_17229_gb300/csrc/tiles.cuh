// tiles.cuh -- register-tiled squared-distance block used by the k-means
// assignment (points x centroids).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dade {

constexpr int L2T_ROWS = 64;   // rows of A per tile
constexpr int L2T_COLS = 64;   // rows of B per tile
constexpr int L2T_BK = 16;     // dimensions staged per step
constexpr int L2T_THREADS = 256;

struct L2TileSmem {
    float a[L2T_BK][L2T_ROWS];
    float b[L2T_BK][L2T_COLS];
};

// acc[i][j] = sum_k (A[r0 + 4 ty + i][k] - B[c0 + 4 tx + j][k])^2 over k < kdim,
// evaluated exactly as a sum of squared differences in FP32 (no expansion
// into norms and inner products, so no cancellation).  Rows beyond na / nb
// and dimensions beyond kdim read as zero.  256 threads, tx = tid % 16,
// ty = tid / 16.  Must be called by every thread of the block.
__device__ inline void l2_tile(const float *__restrict__ A, int64_t na, int lda,
                               const float *__restrict__ B, int64_t nb, int ldb, int kdim,
                               int64_t r0, int64_t c0, float acc[4][4], L2TileSmem &sm) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < kdim; k0 += L2T_BK) {
#pragma unroll
        for (int e = tid; e < L2T_ROWS * L2T_BK; e += L2T_THREADS) {
            int row = e / L2T_BK, kk = e % L2T_BK;
            int64_t ra = r0 + row, cb = c0 + row;
            int k = k0 + kk;
            sm.a[kk][row] = (ra < na && k < kdim) ? A[ra * lda + k] : 0.f;
            sm.b[kk][row] = (cb < nb && k < kdim) ? B[cb * ldb + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < L2T_BK; ++kk) {
            float4 a = *reinterpret_cast<const float4 *>(&sm.a[kk][ty * 4]);
            float4 b = *reinterpret_cast<const float4 *>(&sm.b[kk][tx * 4]);
            float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float t = av[i] - bv[j];
                    acc[i][j] = fmaf(t, t, acc[i][j]);
                }
        }
        __syncthreads();
    }
}

} // namespace dade
