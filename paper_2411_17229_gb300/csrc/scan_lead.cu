// scan_lead.cu -- instantiations of the D <= 128 DADE kernel that prefilter
// the first increment on the index's BF16 or FP8 copy of the leading dims
// (certified margin, FP32 rerun of every survivor; see scan_fast.cuh).
#include "scan_fast.cuh"

namespace dade {

dade_status scan_fast_lead(const scanning::ScanArgs &a, int64_t nq, int threads, int lf, cudaStream_t s) {
    if (lf == DADE_LEAD_FP8) return dade_fast_by_threads<DADE_LEAD_FP8>(a, nq, threads, s);
    return dade_fast_by_threads<DADE_LEAD_BF16>(a, nq, threads, s);
}

} // namespace dade
