// peak.cu -- measured FP32 fused multiply-add throughput of the current GPU,
// the denominator of the arithmetic roofline of the scan kernels whose
// staged rows are shared by many queries (the distance arithmetic is FP32
// FMA/FSUB on the CUDA cores there, not memory traffic).
//
// Every thread runs 8 independent FMA chains (enough to cover the FMA
// pipeline latency with 8 warps per SM partition), the grid fills every SM
// with 8 blocks of 256 threads, and the chains' results are combined and
// stored so that nothing is removed by the compiler.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace dade {
namespace {

constexpr int PK_THREADS = 256, PK_CHAINS = 8, PK_UNROLL = 16;

__global__ void __launch_bounds__(PK_THREADS) k_fma_peak(int iters, float seed, float *out) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = seed + (float)(threadIdx.x + c);
    const float a = 0.999999f, b = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = s;
}

} // namespace
} // namespace dade

extern "C" dade_status dade_fp32_fma_peak(int32_t iters, double *tflops, dade_stream stream) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(iters >= 1 && iters <= (1 << 20), "iters outside 1..2^20");
    DADE_CHECK_ARG(tflops != nullptr, "tflops is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    DADE_TRY_CUDA(cudaGetDevice(&dev));
    DADE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    DevBuf out;
    DADE_TRY(out.alloc(sizeof(float) * (size_t)blocks * PK_THREADS));
    cudaEvent_t e0, e1;
    DADE_TRY_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        set_error("cudaEventCreate failed");
        return DADE_ECUDA;
    }
    dade_status st = DADE_OK;
    float best_ms = -1.f;
    for (int rep = 0; rep < 4 && st == DADE_OK; ++rep) {   // the first launch warms the clocks up
        cudaEventRecord(e0, s);
        k_fma_peak<<<blocks, PK_THREADS, 0, s>>>(iters, 1.f + rep, out.as<float>());
        st = launch_check("k_fma_peak");
        cudaEventRecord(e1, s);
        if (st == DADE_OK && cudaEventSynchronize(e1) == cudaSuccess) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best_ms < 0.f || ms < best_ms)) best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != DADE_OK) return st;
    if (best_ms <= 0.f) {
        set_error("timing of the FMA probe failed");
        return DADE_ECUDA;
    }
    const double flops = 2.0 * PK_CHAINS * PK_UNROLL * (double)iters * blocks * PK_THREADS;
    *tflops = flops / (best_ms * 1e-3) / 1e12;
    return DADE_OK;
}
