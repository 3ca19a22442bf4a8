// scan_fast.cu -- FP32 and FDScanning instantiations of the kernels
// specialised for D in 113..128 (scan_fast.cuh), and their dispatch.
#include "scan_fast.cuh"

namespace dade {

dade_status scan_fast_lead(const scanning::ScanArgs &a, int64_t nq, int threads, int lf, cudaStream_t s);

// True when the specialised kernels cover this index and request.
bool scan_fast_applies(const ScanArgs &a, bool fd) {
    return a.nb == FNB && (fd || a.gb == 1 || a.gb == 2 || a.gb == 4 || a.gb == 8);
}

dade_status scan_fast(const ScanArgs &a, int64_t nq, bool fd, int threads, int lf, cudaStream_t s) {
    const bool st = a.stats != nullptr;
    if (fd) {
        const SmemLayout L = layout(a.dp, a.tile, 4, a.ns, a.k, a.nprobe);
        if (threads == 256)
            return st ? launch_k(k_fd_fast<256, FNB, true>, "k_fd_fast", 256, a, nq, L.total, s)
                      : launch_k(k_fd_fast<256, FNB, false>, "k_fd_fast", 256, a, nq, L.total, s);
        return st ? launch_k(k_fd_fast<128, FNB, true>, "k_fd_fast", 128, a, nq, L.total, s)
                  : launch_k(k_fd_fast<128, FNB, false>, "k_fd_fast", 128, a, nq, L.total, s);
    }
    if (lf) return scan_fast_lead(a, nq, threads, lf, s);
    return dade_fast_by_threads<0>(a, nq, threads, s);
}

} // namespace dade
