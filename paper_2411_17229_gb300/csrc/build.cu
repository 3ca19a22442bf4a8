// build.cu -- index construction (offline steps of Section 3.2 and 3.4):
// FP64 mean and covariance on the GPU, FP64 eigendecomposition on the host,
// FP32 rotation of every base vector, inverted lists (given assignment or
// seeded k-means on the rotated vectors), the dimension-blocked packing, and
// the rho_d sample from which eps_d is read (Eq. 14).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "internal.cuh"
#include "tiles.cuh"

namespace dade {

namespace {

// ------------------------------------------------------------ SplitMix64 ----
// Counter-based draws: value i of stream `key` is mix(key + (i + 1) * gamma)
// with Steele, Lea and Flood's SplitMix64 finaliser.
inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
inline uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * 0x9E3779B97F4A7C15ULL); }
inline uint64_t uniform(uint64_t key, uint64_t i, uint64_t n) {   // in [0, n)
    return (uint64_t)(((unsigned __int128)draw(key, i) * n) >> 64);
}
// Standard normal draw i of stream `key` (Box-Muller on two 53-bit uniforms).
inline double gaussian(uint64_t key, uint64_t i) {
    const double u1 = ((double)(draw(key, 2 * i) >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
    const double u2 = (double)(draw(key, 2 * i + 1) >> 11) * 0x1.0p-53;        // [0, 1)
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

// ------------------------------------------------------------- kernels ------

// Column sums in FP64 (mean of Lemma 1's centring).
__global__ void k_colsum(const float *__restrict__ x, int64_t n, int d, int64_t rows_per_block,
                         double *__restrict__ sum) {
    int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    int64_t r1 = min(n, r0 + rows_per_block);
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int64_t r = r0; r < r1; ++r) s += (double)x[r * d + j];
        atomicAdd(&sum[j], s);
    }
}

// Covariance sum_i (x_i - mu)(x_i - mu)^T in FP64 (products of FP32 inputs are
// exact in FP64).  Block = one 32x32 tile (ti <= tj) of the upper triangle
// and one slice of rows; 256 threads each own a 2x2 patch.
constexpr int CT = 32;
__global__ void __launch_bounds__(256) k_cov(const float *__restrict__ x, int64_t n, int d,
                                             const double *__restrict__ mu, int64_t rows_per_slice,
                                             const int2 *__restrict__ tiles, double *__restrict__ C) {
    __shared__ double si[CT][CT + 1], sj[CT][CT + 1];
    const int2 t = tiles[blockIdx.x];
    const int ci0 = t.x * CT, cj0 = t.y * CT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    int64_t r0 = (int64_t)blockIdx.y * rows_per_slice, r1 = min(n, r0 + rows_per_slice);
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (int64_t rb = r0; rb < r1; rb += CT) {
        for (int e = tid; e < CT * CT; e += 256) {
            int rr = e / CT, cc = e % CT;
            int64_t r = rb + rr;
            int ci = ci0 + cc, cj = cj0 + cc;
            si[rr][cc] = (r < r1 && ci < d) ? (double)x[r * d + ci] - mu[ci] : 0.0;
            sj[rr][cc] = (r < r1 && cj < d) ? (double)x[r * d + cj] - mu[cj] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < CT; ++rr) {
            double a0 = si[rr][ty * 2], a1 = si[rr][ty * 2 + 1];
            double b0 = sj[rr][tx * 2], b1 = sj[rr][tx * 2 + 1];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            int i = ci0 + ty * 2 + a, j = cj0 + tx * 2 + b;
            if (i < d && j < d && (t.x != t.y || i <= j)) atomicAdd(&C[(int64_t)i * d + j], acc[a][b]);
        }
}

// Nearest centroid of every point (k-means assignment and list assignment),
// ties to the lower centroid index; adds the block's objective to *obj.
__global__ void __launch_bounds__(L2T_THREADS) k_nearest(const float *__restrict__ X, int64_t n, int ldx,
                                                         const float *__restrict__ cent, int nc, int ldc, int kdim,
                                                         int32_t *__restrict__ assign, double *__restrict__ obj) {
    __shared__ L2TileSmem sm;
    __shared__ double sobj[L2T_THREADS / 32];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * L2T_ROWS;
    float best[4];
    int bidx[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { best[i] = INFINITY; bidx[i] = 0x7fffffff; }
    for (int c0 = 0; c0 < nc; c0 += L2T_COLS) {
        float acc[4][4];
        l2_tile(X, n, ldx, cent, nc, ldc, kdim, r0, c0, acc, sm);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int c = c0 + tx * 4 + j;
                if (c < nc && (acc[i][j] < best[i] || (acc[i][j] == best[i] && c < bidx[i]))) {
                    best[i] = acc[i][j];
                    bidx[i] = c;
                }
            }
    }
    // reduce over the 16 threads (same ty, one half-warp) that share each row
    double part = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float b = best[i];
        int bi = bidx[i];
        for (int off = 8; off > 0; off >>= 1) {
            float ob = __shfl_xor_sync(0xffffffffu, b, off);
            int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (ob < b || (ob == b && oi < bi)) { b = ob; bi = oi; }
        }
        int64_t r = r0 + ty * 4 + i;
        if (tx == 0 && r < n) {
            assign[r] = bi;
            part += (double)b;
        }
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((tid & 31) == 0) sobj[tid >> 5] = part;
    __syncthreads();
    if (tid == 0 && obj) {
        double s = 0.0;
        for (int w = 0; w < L2T_THREADS / 32; ++w) s += sobj[w];
        atomicAdd(obj, s);
    }
}

// Per-list sums (FP64) and counts of member vectors.
__global__ void k_accum(const float *__restrict__ X, int64_t n, int dp, const int32_t *__restrict__ assign,
                        double *__restrict__ sum, int64_t *__restrict__ cnt) {
    int64_t total = n * (int64_t)dp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / dp;
        int k = (int)(e % dp);
        int c = assign[i];
        atomicAdd(&sum[(int64_t)c * dp + k], (double)X[e]);
        if (k == 0) atomicAdd((unsigned long long *)&cnt[c], 1ULL);
    }
}

// centroid = member mean; an empty list keeps its centroid (k-means) or gets
// zeros (member means of a given assignment).
__global__ void k_finalize(const double *__restrict__ sum, const int64_t *__restrict__ cnt, int nc, int dp,
                           int keep_empty, float *__restrict__ cent) {
    int64_t total = (int64_t)nc * dp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int c = (int)(e / dp);
        int64_t m = cnt[c];
        if (m > 0) cent[e] = (float)(sum[e] / (double)m);
        else if (!keep_empty) cent[e] = 0.f;
    }
}

__global__ void k_gather_rows(const float *__restrict__ X, int dp, const int64_t *__restrict__ rows, int nr,
                              float *__restrict__ out) {
    int64_t total = (int64_t)nr * dp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = X[rows[e / dp] * dp + e % dp];
}

// Dimension-blocked packing: vector i goes to slot pos[i] of list assign[i];
// its 16-dimension block b lands in that list's slab b.
__global__ void k_pack(const float *__restrict__ X, int64_t n, int dp, int nb, const int32_t *__restrict__ assign,
                       const int32_t *__restrict__ pos, const ListMeta *__restrict__ meta, float *__restrict__ data,
                       int32_t *__restrict__ ids) {
    int64_t total = n * (int64_t)nb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e / nb;
        int b = (int)(e % nb);
        ListMeta m = meta[assign[i]];
        const float4 *src = reinterpret_cast<const float4 *>(X + i * dp + b * 16);
        float4 *dst = reinterpret_cast<float4 *>(data + m.base + (int64_t)b * m.np * 16 + (int64_t)pos[i] * 16);
#pragma unroll
        for (int t = 0; t < 4; ++t) dst[t] = src[t];
        if (b == 0) ids[m.slot + pos[i]] = (int32_t)i;
    }
}

// ---- low-precision copy of the leading dims (prefilter codes) -----------------------
// FP8 only: per (list, lead block) maximum |o' - c'| over the list's members,
// as the bits of a nonnegative float (ordered like the values).
__global__ void k_lead_absmax(const float *__restrict__ X, int64_t n, int dp, int lead_nb,
                              const int32_t *__restrict__ assign, const float *__restrict__ cent,
                              unsigned *__restrict__ amax) {
    int64_t total = n * (int64_t)lead_nb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / lead_nb;
        const int b = (int)(e % lead_nb), c = assign[i];
        float m = 0.f;
        for (int k = 0; k < 16; ++k)
            m = fmaxf(m, fabsf(__fsub_rn(X[i * dp + b * 16 + k], cent[(int64_t)c * dp + b * 16 + k])));
        atomicMax(&amax[(int64_t)c * lead_nb + b], __float_as_uint(m));
    }
}

// FP8 scale of a (list, block): the largest residual maps to 448, the
// largest finite e4m3 value; an all-zero block gets scale 1.
__global__ void k_lead_scale(const unsigned *__restrict__ amax, int64_t cnt, float *__restrict__ scale) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        const float m = __uint_as_float(amax[e]);
        scale[e] = m > 0.f ? m / 448.f : 1.f;
    }
}

// Codes of vector i (list c, slot pos[i]): residual r = o' - c' per lead dim,
// BF16 round-to-nearest-even, or FP8 e4m3 of r / scale (saturating).  The
// list's codes start at byte slot(c) * lead_nb * 16 * ES; block b of it is a
// slab of np x 16 codes.  err[b][slot] is || r - dequant(code) || over the
// blocks 0..b, accumulated in FP64 from the exact differences and rounded up,
// where dequant is the scan's own widening (times the scale, rounded once).
__global__ void k_pack_lead(const float *__restrict__ X, int64_t n, int dp, int lead_nb, int lf,
                            const int32_t *__restrict__ assign, const int32_t *__restrict__ pos,
                            const ListMeta *__restrict__ meta, const float *__restrict__ cent,
                            const float *__restrict__ scale, unsigned char *__restrict__ lead, float *__restrict__ err,
                            int64_t slots) {
    const int es = lf == DADE_LEAD_BF16 ? 2 : 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = assign[i];
        const ListMeta m = meta[c];
        const int64_t slot = m.slot + pos[i];
        double acc = 0.0;
        for (int b = 0; b < lead_nb; ++b) {
            const float sc = lf == DADE_LEAD_FP8 ? scale[(int64_t)c * lead_nb + b] : 1.f;
            unsigned char *dst = lead + (m.slot * lead_nb * 16 + (int64_t)b * m.np * 16 + (int64_t)pos[i] * 16) * es;
            for (int k = 0; k < 16; k += 2) {
                const float o0 = X[i * dp + b * 16 + k], o1 = X[i * dp + b * 16 + k + 1];
                const float c0 = cent[(int64_t)c * dp + b * 16 + k], c1 = cent[(int64_t)c * dp + b * 16 + k + 1];
                const float r0 = __fsub_rn(o0, c0), r1 = __fsub_rn(o1, c1);
                float q0, q1;
                if (lf == DADE_LEAD_BF16) {
                    const __nv_bfloat16 h0 = __float2bfloat16_rn(r0), h1 = __float2bfloat16_rn(r1);
                    reinterpret_cast<unsigned short *>(dst)[k] = __bfloat16_as_ushort(h0);
                    reinterpret_cast<unsigned short *>(dst)[k + 1] = __bfloat16_as_ushort(h1);
                    q0 = __bfloat162float(h0);
                    q1 = __bfloat162float(h1);
                } else {
                    const __nv_fp8x2_storage_t v = __nv_cvt_float2_to_fp8x2(
                        make_float2(__fdiv_rn(r0, sc), __fdiv_rn(r1, sc)), __NV_SATFINITE, __NV_E4M3);
                    reinterpret_cast<unsigned short *>(dst)[k / 2] = v;
                    const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(v, __NV_E4M3)));
                    q0 = __fmul_rn(sc, f.x);
                    q1 = __fmul_rn(sc, f.y);
                }
                const double e0 = ((double)o0 - (double)c0) - (double)q0, e1 = ((double)o1 - (double)c1) - (double)q1;
                acc += e0 * e0 + e1 * e1;
            }
            err[(int64_t)b * slots + slot] = __double2float_ru(__dsqrt_ru(acc));
        }
    }
}

// Row-major copy of dims [16 nb0, dp) of vector i at slot(list) + pos[i].
__global__ void k_pack_tail(const float *__restrict__ X, int64_t n, int dp, int nb0, const int32_t *__restrict__ assign,
                            const int32_t *__restrict__ pos, const ListMeta *__restrict__ meta, float *__restrict__ tail) {
    const int tw = dp - 16 * nb0;
    const int64_t total = n * (int64_t)(tw / 4);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / (tw / 4);
        const int k4 = (int)(e % (tw / 4));
        const ListMeta m = meta[assign[i]];
        const float4 v = *reinterpret_cast<const float4 *>(X + i * dp + 16 * nb0 + 4 * k4);
        *reinterpret_cast<float4 *>(tail + (m.slot + pos[i]) * tw + 4 * k4) = v;
    }
}

// Prefix sums P_d (FP64) of one sampled pair's squared difference at every
// d = 16 (b + 1); one warp per pair, each half-warp one 16-dim block.
__global__ void k_pair_prefix(const float *__restrict__ X, int dp, int nb, const int64_t *__restrict__ pairs,
                              int64_t m, double *__restrict__ P) {
    const int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = w; s < m; s += nw) {
        const float *a = X + pairs[2 * s] * dp, *b = X + pairs[2 * s + 1] * dp;
        double run = 0.0;
        for (int b0 = 0; b0 < nb; b0 += 2) {
            int blk = b0 + (lane >> 4);
            double t = 0.0;
            if (blk < nb) {
                double df = (double)a[blk * 16 + (lane & 15)] - (double)b[blk * 16 + (lane & 15)];
                t = df * df;
            }
            for (int off = 8; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
            double lo = __shfl_sync(0xffffffffu, t, 0), hi = __shfl_sync(0xffffffffu, t, 16);
            run += lo;
            if (lane == 0) P[s * nb + b0] = run;
            if (b0 + 1 < nb) {
                run += hi;
                if (lane == 0) P[s * nb + b0 + 1] = run;
            }
        }
    }
}


int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

} // namespace

dade_status launch_nearest(const float *X, int64_t n, int ldx, const float *cent, int nc, int ldc, int kdim,
                           int32_t *assign, double *obj, cudaStream_t s) {
    k_nearest<<<(unsigned)((n + L2T_ROWS - 1) / L2T_ROWS), L2T_THREADS, 0, s>>>(X, n, ldx, cent, nc, ldc, kdim,
                                                                                 assign, obj);
    return launch_check("k_nearest");
}

// ------------------------------------------------------------ build ---------
dade_status build_index(const float *base, int64_t n, int32_t d, const dade_build_opts &o, dade_index *ix,
                        cudaStream_t s) {
    ix->n = n;
    ix->d = d;
    ix->dp = (d + 15) / 16 * 16;
    ix->nb = ix->dp / 16;
    ix->nc = o.n_clusters;
    const int dp = ix->dp, nb = ix->nb, nc = ix->nc;

    // base vectors on the device
    DevBuf xbuf;
    const float *x = base;
    cudaPointerAttributes attr{};
    bool host_in = cudaPointerGetAttributes(&attr, base) != cudaSuccess || attr.type == cudaMemoryTypeUnregistered ||
                   attr.type == cudaMemoryTypeHost;
    cudaGetLastError();
    if (host_in) {
        DADE_TRY(xbuf.alloc(sizeof(float) * (size_t)n * d));
        DADE_TRY_CUDA(cudaMemcpyAsync(xbuf.p, base, sizeof(float) * (size_t)n * d, cudaMemcpyHostToDevice, s));
        x = xbuf.as<float>();
    }

    // ---- mean and covariance (FP64) ------------------------------------------
    DevBuf musum, cov;
    DADE_TRY(musum.alloc(sizeof(double) * d));
    DADE_TRY(cov.alloc(sizeof(double) * (size_t)d * d));
    DADE_TRY_CUDA(cudaMemsetAsync(musum.p, 0, sizeof(double) * d, s));
    DADE_TRY_CUDA(cudaMemsetAsync(cov.p, 0, sizeof(double) * (size_t)d * d, s));
    {
        int64_t rpb = std::max<int64_t>(64, (n + 4095) / 4096);
        k_colsum<<<(unsigned)((n + rpb - 1) / rpb), 256, 0, s>>>(x, n, d, rpb, musum.as<double>());
        DADE_TRY(launch_check("k_colsum"));
    }
    std::vector<double> msum(d);
    DADE_TRY_CUDA(cudaMemcpyAsync(msum.data(), musum.p, sizeof(double) * d, cudaMemcpyDeviceToHost, s));
    DADE_TRY_CUDA(cudaStreamSynchronize(s));
    ix->mu.resize(d);
    for (int j = 0; j < d; ++j) ix->mu[j] = msum[j] / (double)n;
    DADE_TRY_CUDA(cudaMemcpyAsync(musum.p, ix->mu.data(), sizeof(double) * d, cudaMemcpyHostToDevice, s));
    {
        int nt = (d + CT - 1) / CT;
        std::vector<int2> tiles;
        for (int a = 0; a < nt; ++a)
            for (int b = a; b < nt; ++b) tiles.push_back(make_int2(a, b));
        DevBuf tb;
        DADE_TRY(tb.alloc(sizeof(int2) * tiles.size()));
        DADE_TRY_CUDA(cudaMemcpyAsync(tb.p, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, s));
        int64_t slices = std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, (152 * 8 + tiles.size() - 1) / tiles.size()));
        int64_t rps = (n + slices - 1) / slices;
        dim3 grid((unsigned)tiles.size(), (unsigned)((n + rps - 1) / rps));
        k_cov<<<grid, 256, 0, s>>>(x, n, d, musum.as<double>(), rps, tb.as<int2>(), cov.as<double>());
        DADE_TRY(launch_check("k_cov"));
        std::vector<double> C((size_t)d * d);
        DADE_TRY_CUDA(cudaMemcpyAsync(C.data(), cov.p, sizeof(double) * C.size(), cudaMemcpyDeviceToHost, s));
        DADE_TRY_CUDA(cudaStreamSynchronize(s));
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                if (j < i) C[(size_t)i * d + j] = C[(size_t)j * d + i];
            }
        for (auto &v : C) v /= (double)n;
        if (o.transform == DADE_TRANSFORM_PCA) {
            // ---- eigendecomposition (host FP64), descending --------------------------
            if (!sym_eig(d, C, ix->lam, ix->W)) {
                set_error("eigendecomposition did not converge");
                return DADE_ECUDA;
            }
        } else {
            // ---- a given or random orthogonal basis; lambda_k = w_k^T C w_k --------------
            ix->W.assign((size_t)d * d, 0.0);
            if (o.transform == DADE_TRANSFORM_GIVEN) {
                std::copy(o.basis, o.basis + (size_t)d * d, ix->W.begin());
            } else {
                uint64_t key = o.seed ^ 0x726f74617465ULL;
                for (size_t e = 0; e < ix->W.size(); ++e) ix->W[e] = gaussian(key, e);
            }
            // Gram-Schmidt over the columns, twice (a given basis is only re-orthonormalised
            // within rounding, a random one becomes Haar-distributed)
            for (int pass = 0; pass < 2; ++pass)
                for (int k = 0; k < d; ++k) {
                    for (int j = 0; j < k; ++j) {
                        double dot = 0.0;
                        for (int i = 0; i < d; ++i) dot += ix->W[(size_t)i * d + j] * ix->W[(size_t)i * d + k];
                        for (int i = 0; i < d; ++i) ix->W[(size_t)i * d + k] -= dot * ix->W[(size_t)i * d + j];
                    }
                    double nn = 0.0;
                    for (int i = 0; i < d; ++i) nn += ix->W[(size_t)i * d + k] * ix->W[(size_t)i * d + k];
                    if (!(nn > 0.0)) {
                        set_error("invalid argument: the basis is singular");
                        return DADE_EINVAL;
                    }
                    const double inv = 1.0 / std::sqrt(nn);
                    for (int i = 0; i < d; ++i) ix->W[(size_t)i * d + k] *= inv;
                }
            if (o.transform == DADE_TRANSFORM_GIVEN) {   // the given columns must already be orthonormal
                double worst = 0.0;
                for (size_t e = 0; e < ix->W.size(); ++e) worst = std::max(worst, std::fabs(ix->W[e] - o.basis[e]));
                if (worst > 1e-6) {
                    set_error("invalid argument: the given basis is not orthonormal (columns differ by " +
                              std::to_string(worst) + " after Gram-Schmidt)");
                    return DADE_EINVAL;
                }
            }
            ix->lam.assign(d, 0.0);
            std::vector<double> cw(d);
            for (int k = 0; k < d; ++k) {
                for (int i = 0; i < d; ++i) {
                    double t = 0.0;
                    for (int j = 0; j < d; ++j) t += C[(size_t)i * d + j] * ix->W[(size_t)j * d + k];
                    cw[i] = t;
                }
                double l = 0.0;
                for (int i = 0; i < d; ++i) l += ix->W[(size_t)i * d + k] * cw[i];
                ix->lam[k] = std::max(l, 0.0);
            }
        }
    }
    ix->Lam.assign(d + 1, 0.0);
    for (int k = 0; k < d; ++k) ix->Lam[k + 1] = ix->Lam[k] + ix->lam[k];

    // ---- rotation of every base vector (tensor-core GEMM) ---------------------------
    DADE_TRY(upload_basis(ix, s));
    DADE_TRY(ix->errflag.alloc(sizeof(int32_t) * 4));
    DADE_TRY_CUDA(cudaMemsetAsync(ix->errflag.p, 0, sizeof(int32_t) * 4, s));
    DevBuf rot;
    DADE_TRY(rot.alloc(sizeof(float) * (size_t)n * dp));
    DADE_TRY(rotate_direct(ix, x, n, dp, rot.as<float>(), s));
    xbuf.release();

    // ---- inverted lists ----------------------------------------------------------
    DevBuf asg, lsum, lcnt;
    DADE_TRY(asg.alloc(sizeof(int32_t) * n));
    DADE_TRY(ix->cent.alloc(sizeof(float) * (size_t)nc * dp));
    DADE_TRY(lsum.alloc(sizeof(double) * (size_t)nc * dp));
    DADE_TRY(lcnt.alloc(sizeof(int64_t) * nc));
    auto member_means = [&](int keep_empty) -> dade_status {
        DADE_TRY_CUDA(cudaMemsetAsync(lsum.p, 0, sizeof(double) * (size_t)nc * dp, s));
        DADE_TRY_CUDA(cudaMemsetAsync(lcnt.p, 0, sizeof(int64_t) * nc, s));
        k_accum<<<grid_for(n * dp, 256), 256, 0, s>>>(rot.as<float>(), n, dp, asg.as<int32_t>(), lsum.as<double>(),
                                                      lcnt.as<int64_t>());
        DADE_TRY(launch_check("k_accum"));
        k_finalize<<<grid_for((int64_t)nc * dp, 256), 256, 0, s>>>(lsum.as<double>(), lcnt.as<int64_t>(), nc, dp,
                                                                   keep_empty, ix->cent.as<float>());
        return launch_check("k_finalize");
    };
    if (o.assign) {
        for (int64_t i = 0; i < n; ++i)
            if (o.assign[i] < 0 || o.assign[i] >= nc) {
                set_error("invalid argument: assign[] outside 0..n_clusters-1");
                return DADE_EINVAL;
            }
        DADE_TRY_CUDA(cudaMemcpyAsync(asg.p, o.assign, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
        DADE_TRY(member_means(0));
    } else {
        std::vector<int64_t> init(nc);
        if (o.kmeans_init) {
            std::vector<char> seen(n, 0);
            for (int c = 0; c < nc; ++c) {
                int64_t v = o.kmeans_init[c];
                if (v < 0 || v >= n || seen[v]) {
                    set_error("invalid argument: kmeans_init must hold distinct ids in 0..n-1");
                    return DADE_EINVAL;
                }
                seen[v] = 1;
                init[c] = v;
            }
        } else {   // partial Fisher-Yates shuffle driven by SplitMix64
            std::vector<int64_t> perm(n);
            for (int64_t i = 0; i < n; ++i) perm[i] = i;
            uint64_t key = o.seed ^ 0x6b6d65616e73ULL;
            for (int c = 0; c < nc; ++c) {
                int64_t j = c + (int64_t)uniform(key, (uint64_t)c, (uint64_t)(n - c));
                std::swap(perm[c], perm[j]);
                init[c] = perm[c];
            }
        }
        DevBuf ib, objb;
        DADE_TRY(ib.alloc(sizeof(int64_t) * nc));
        DADE_TRY(objb.alloc(sizeof(double) * std::max(1, o.kmeans_iters)));
        DADE_TRY_CUDA(cudaMemsetAsync(objb.p, 0, sizeof(double) * std::max(1, o.kmeans_iters), s));
        DADE_TRY_CUDA(cudaMemcpyAsync(ib.p, init.data(), sizeof(int64_t) * nc, cudaMemcpyHostToDevice, s));
        k_gather_rows<<<grid_for((int64_t)nc * dp, 256), 256, 0, s>>>(rot.as<float>(), dp, ib.as<int64_t>(), nc,
                                                                      ix->cent.as<float>());
        DADE_TRY(launch_check("k_gather_rows"));
        for (int it = 0; it < o.kmeans_iters; ++it) {
            DADE_TRY(launch_nearest(rot.as<float>(), n, dp, ix->cent.as<float>(), nc, dp, dp, asg.as<int32_t>(),
                                    objb.as<double>() + it, s));
            DADE_TRY(member_means(1));
        }
        ix->kmeans_obj.resize(o.kmeans_iters);
        if (o.kmeans_iters > 0)
            DADE_TRY_CUDA(cudaMemcpyAsync(ix->kmeans_obj.data(), objb.p, sizeof(double) * o.kmeans_iters,
                                          cudaMemcpyDeviceToHost, s));
        // lists: every vector to its nearest final centroid
        DADE_TRY(launch_nearest(rot.as<float>(), n, dp, ix->cent.as<float>(), nc, dp, dp, asg.as<int32_t>(), nullptr, s));
    }
    lsum.release();
    lcnt.release();
    DADE_TRY(centroid_norms(ix, s));
    DADE_TRY(prepare_tensor_operands(ix, s));
    ix->assign.resize(n);
    DADE_TRY_CUDA(cudaMemcpyAsync(ix->assign.data(), asg.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    DADE_TRY_CUDA(cudaStreamSynchronize(s));

    // ---- dimension-blocked packing ----------------------------------------------
    {
        std::vector<int32_t> len(nc, 0), pos(n);
        for (int64_t i = 0; i < n; ++i) pos[i] = len[ix->assign[i]]++;   // ascending base id within a list
        ix->lists.resize(nc);
        int64_t base = 0, slot = 0;
        int32_t mx = 0;
        for (int c = 0; c < nc; ++c) {
            ListMeta m;
            m.len = len[c];
            m.np = (len[c] + 3) / 4 * 4;
            m.base = base;
            m.slot = slot;
            base += ((int64_t)m.np * dp + 63) / 64 * 64;
            slot += m.np;
            mx = std::max(mx, len[c]);
            ix->lists[c] = m;
        }
        ix->max_list = mx;
        ix->data_floats = std::max<int64_t>(base, 64);
        ix->slots = std::max<int64_t>(slot, 1);
        DADE_TRY(ix->data.alloc(sizeof(float) * (size_t)ix->data_floats));
        DADE_TRY(ix->ids.alloc(sizeof(int32_t) * (size_t)ix->slots));
        DADE_TRY(ix->meta.alloc(sizeof(ListMeta) * nc));
        DADE_TRY_CUDA(cudaMemsetAsync(ix->data.p, 0, sizeof(float) * (size_t)ix->data_floats, s));
        DADE_TRY_CUDA(cudaMemsetAsync(ix->ids.p, 0xff, sizeof(int32_t) * (size_t)ix->slots, s));
        DADE_TRY_CUDA(cudaMemcpyAsync(ix->meta.p, ix->lists.data(), sizeof(ListMeta) * nc, cudaMemcpyHostToDevice, s));
        DevBuf posb;
        DADE_TRY(posb.alloc(sizeof(int32_t) * n));
        DADE_TRY_CUDA(cudaMemcpyAsync(posb.p, pos.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
        k_pack<<<grid_for(n * nb, 256), 256, 0, s>>>(rot.as<float>(), n, dp, nb, asg.as<int32_t>(), posb.as<int32_t>(),
                                                    ix->meta.as<ListMeta>(), ix->data.as<float>(), ix->ids.as<int32_t>());
        DADE_TRY(launch_check("k_pack"));
        if (o.tail_from > 0) {
            ix->tail_nb0 = o.tail_from / 16;
            ix->tail_w = dp - o.tail_from;
            DADE_TRY(ix->tail.alloc(sizeof(float) * (size_t)ix->slots * ix->tail_w));
            DADE_TRY_CUDA(cudaMemsetAsync(ix->tail.p, 0, sizeof(float) * (size_t)ix->slots * ix->tail_w, s));
            k_pack_tail<<<grid_for(n * (ix->tail_w / 4), 256), 256, 0, s>>>(
                rot.as<float>(), n, dp, ix->tail_nb0, asg.as<int32_t>(), posb.as<int32_t>(), ix->meta.as<ListMeta>(),
                ix->tail.as<float>());
            DADE_TRY(launch_check("k_pack_tail"));
        }
        if (o.lead_format != DADE_LEAD_NONE) {
            const int lnb = o.lead_dims / 16, es = o.lead_format == DADE_LEAD_BF16 ? 2 : 1;
            ix->lead_format = o.lead_format;
            ix->lead_dims = o.lead_dims;
            ix->lead_nb = lnb;
            const size_t code_bytes = (size_t)ix->slots * lnb * 16 * es;
            DADE_TRY(ix->lead.alloc(code_bytes));
            DADE_TRY(ix->lead_err.alloc(sizeof(float) * (size_t)ix->slots * lnb));
            DADE_TRY(ix->lead_scale.alloc(sizeof(float) * (size_t)nc * lnb));
            DADE_TRY_CUDA(cudaMemsetAsync(ix->lead.p, 0, code_bytes, s));
            DADE_TRY_CUDA(cudaMemsetAsync(ix->lead_err.p, 0, sizeof(float) * (size_t)ix->slots * lnb, s));
            if (o.lead_format == DADE_LEAD_FP8) {
                DevBuf amax;
                DADE_TRY(amax.alloc(sizeof(unsigned) * (size_t)nc * lnb));
                DADE_TRY_CUDA(cudaMemsetAsync(amax.p, 0, sizeof(unsigned) * (size_t)nc * lnb, s));
                k_lead_absmax<<<grid_for(n * lnb, 256), 256, 0, s>>>(rot.as<float>(), n, dp, lnb, asg.as<int32_t>(),
                                                                     ix->cent.as<float>(), amax.as<unsigned>());
                DADE_TRY(launch_check("k_lead_absmax"));
                k_lead_scale<<<grid_for((int64_t)nc * lnb, 256), 256, 0, s>>>(amax.as<unsigned>(), (int64_t)nc * lnb,
                                                                              ix->lead_scale.as<float>());
                DADE_TRY(launch_check("k_lead_scale"));
                DADE_TRY_CUDA(cudaStreamSynchronize(s));
            } else {
                std::vector<float> ones((size_t)nc * lnb, 1.f);
                DADE_TRY_CUDA(cudaMemcpyAsync(ix->lead_scale.p, ones.data(), sizeof(float) * ones.size(),
                                              cudaMemcpyHostToDevice, s));
                DADE_TRY_CUDA(cudaStreamSynchronize(s));
            }
            k_pack_lead<<<grid_for(n, 256), 256, 0, s>>>(rot.as<float>(), n, dp, lnb, o.lead_format, asg.as<int32_t>(),
                                                         posb.as<int32_t>(), ix->meta.as<ListMeta>(), ix->cent.as<float>(),
                                                         ix->lead_scale.as<float>(), ix->lead.as<unsigned char>(),
                                                         ix->lead_err.as<float>(), ix->slots);
            DADE_TRY(launch_check("k_pack_lead"));
        }
        DADE_TRY(make_data_tmap(ix));
        DADE_TRY_CUDA(cudaStreamSynchronize(s));
    }

    // ---- rho_d sample for eps_d (Eq. 14) -------------------------------------------
    {
        int64_t m = o.eps_pairs;
        std::vector<int64_t> pairs(2 * m);
        if (o.pairs) {
            for (int64_t t = 0; t < m; ++t) {
                int64_t a = o.pairs[2 * t], b = o.pairs[2 * t + 1];
                if (a < 0 || a >= n || b < 0 || b >= n || a == b) {
                    set_error("invalid argument: pairs[] must hold ids in 0..n-1 with i != j");
                    return DADE_EINVAL;
                }
                pairs[2 * t] = a;
                pairs[2 * t + 1] = b;
            }
        } else {
            uint64_t key = o.seed ^ 0x6570735f70616972ULL;
            for (int64_t t = 0; t < m; ++t) {
                int64_t a = (int64_t)uniform(key, 2 * (uint64_t)t, (uint64_t)n);
                int64_t b = (int64_t)uniform(key, 2 * (uint64_t)t + 1, (uint64_t)(n - 1));
                if (b >= a) ++b;
                pairs[2 * t] = a;
                pairs[2 * t + 1] = b;
            }
        }
        DevBuf pb, Pb;
        DADE_TRY(pb.alloc(sizeof(int64_t) * 2 * m));
        DADE_TRY(Pb.alloc(sizeof(double) * (size_t)m * nb));
        DADE_TRY_CUDA(cudaMemcpyAsync(pb.p, pairs.data(), sizeof(int64_t) * 2 * m, cudaMemcpyHostToDevice, s));
        k_pair_prefix<<<grid_for(m * 32, 256), 256, 0, s>>>(rot.as<float>(), dp, nb, pb.as<int64_t>(), m,
                                                            Pb.as<double>());
        DADE_TRY(launch_check("k_pair_prefix"));
        std::vector<double> P((size_t)m * nb);
        DADE_TRY_CUDA(cudaMemcpyAsync(P.data(), Pb.p, sizeof(double) * P.size(), cudaMemcpyDeviceToHost, s));
        DADE_TRY_CUDA(cudaStreamSynchronize(s));
        int rows = std::max(0, nb - 1);   // d = 16, 32, ..., 16 (nb - 1) < D
        std::vector<int64_t> keep;
        for (int64_t t = 0; t < m; ++t)
            if (P[(size_t)t * nb + nb - 1] > 0.0) keep.push_back(t);
        ix->eps_kept = (int64_t)keep.size();
        ix->rho.assign((size_t)rows * keep.size(), 0.0);
        for (int r = 0; r < rows; ++r) {
            int dd = 16 * (r + 1);
            double ratio = ix->Lam[d] / ix->Lam[dd];
            double *row = ix->rho.data() + (size_t)r * keep.size();
            for (size_t u = 0; u < keep.size(); ++u) {
                int64_t t = keep[u];
                row[u] = std::sqrt(ratio * P[(size_t)t * nb + r] / P[(size_t)t * nb + nb - 1]);
            }
            std::sort(row, row + keep.size());
        }
    }
    DADE_TRY_CUDA(cudaStreamSynchronize(s));
    int32_t err = 0;
    DADE_TRY_CUDA(cudaMemcpy(&err, ix->errflag.p, sizeof(err), cudaMemcpyDeviceToHost));
    if (err != 0) {
        set_error("a bounded device-side wait gave up during the index build");
        return DADE_ETIMEOUT;
    }
    return DADE_OK;
}

// FP32 copies of the basis (as W^T, dp x dp, zero padded) and of the mean.
dade_status upload_basis(dade_index *ix, cudaStream_t s) {
    const int d = ix->d, dp = ix->dp;
    std::vector<float> wt((size_t)dp * dp, 0.f), m32(d);
    for (int j = 0; j < d; ++j) {
        m32[j] = (float)ix->mu[j];
        for (int k = 0; k < d; ++k) wt[(size_t)k * dp + j] = (float)ix->W[(size_t)j * d + k];
    }
    DADE_TRY(ix->WT32.alloc(sizeof(float) * wt.size()));
    DADE_TRY(ix->mu32.alloc(sizeof(float) * d));
    DADE_TRY_CUDA(cudaMemcpyAsync(ix->WT32.p, wt.data(), sizeof(float) * wt.size(), cudaMemcpyHostToDevice, s));
    DADE_TRY_CUDA(cudaMemcpyAsync(ix->mu32.p, m32.data(), sizeof(float) * d, cudaMemcpyHostToDevice, s));
    DADE_TRY_CUDA(cudaStreamSynchronize(s));
    return DADE_OK;
}

} // namespace dade
