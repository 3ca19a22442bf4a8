// tune.cpp -- dade_tune: the execution options that leave a search's results
// unchanged (threads per block, query order, the row-major tail copy, the
// seeded schedule's later lists query-major or list-major), timed on the
// caller's batch; the fastest is written back and cached per index and
// search shape, so a repeated shape costs no timing.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "dade.h"

namespace {

using Shape = std::tuple<const dade_index *, int64_t, int32_t, int32_t, float, int32_t, int32_t, int32_t, int32_t,
                         int32_t, int32_t, int32_t, int32_t>;
struct Knobs {
    int32_t threads, flags;
};
std::mutex g_mu;
std::map<Shape, Knobs> g_cache;

constexpr int32_t KNOB_FLAGS = DADE_FLAG_QUERY_ORDER | DADE_FLAG_ROW_TAIL | DADE_FLAG_SEED_SPLIT;

bool on_device(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

Shape shape_of(const dade_index *ix, int64_t nq, int32_t k, int32_t nprobe, float alpha, int32_t delta_d,
               const dade_search_opts &o) {
    return Shape(ix, nq, k, nprobe, alpha, delta_d, o.mode, o.tile, o.schedule, o.seed_lists,
                 o.flags & ~KNOB_FLAGS, o.stage_dims, o.estimator);
}

}  // namespace

namespace dade {
void set_error(const std::string &msg);

// The index is gone: its cached choices go too (called by dade_free_index).
void tune_forget(const dade_index *ix) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end();)
        it = std::get<0>(it->first) == ix ? g_cache.erase(it) : std::next(it);
}
}  // namespace dade

extern "C" dade_status dade_tune(const dade_index *ix, const float *q_rot, const int32_t *probe, int64_t nq,
                                 int32_t k, int32_t nprobe, float alpha, int32_t delta_d, dade_search_opts *opts,
                                 int64_t *ids, float *dists, dade_stream stream) {
    dade::set_error("");
    if (!ix || !q_rot || !probe || !opts || !ids || !dists) {
        dade::set_error("dade_tune: NULL pointer");
        return DADE_EINVAL;
    }
    if (!on_device(q_rot) || !on_device(probe) || !on_device(ids) || !on_device(dists)) {
        dade::set_error("dade_tune times the scan on device buffers: q_rot, probe, ids and dists must be device memory");
        return DADE_EINVAL;
    }
    if (nq <= 0) return DADE_OK;
    const dade_search_opts base = *opts;
    const Shape key = shape_of(ix, nq, k, nprobe, alpha, delta_d, base);
    {
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            opts->threads = it->second.threads;
            opts->flags = (base.flags & ~KNOB_FLAGS) | it->second.flags;
            return DADE_OK;
        }
    }
    dade_info info{};
    dade_status st = dade_index_info(ix, &info);
    if (st != DADE_OK) return st;
    std::vector<int32_t> threads = {128, 256}, orders = {0, DADE_FLAG_QUERY_ORDER}, tails = {0}, splits = {0};
    if (info.tail_from > 0) tails.push_back(DADE_FLAG_ROW_TAIL);
    if ((base.schedule == DADE_SCHED_SEEDED && base.seed_lists < nprobe) || base.schedule == DADE_SCHED_ROUNDS)
        splits.push_back(DADE_FLAG_SEED_SPLIT);
    const int32_t keep = base.flags & ~KNOB_FLAGS;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return DADE_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return DADE_ECUDA;
    }
    float best_ms = -1.f;
    Knobs best{base.threads, base.flags & KNOB_FLAGS};
    for (int32_t nt : threads)
        for (int32_t ord : orders)
            for (int32_t tail : tails)
                for (int32_t split : splits) {
                    dade_search_opts o = base;
                    o.threads = nt;
                    o.flags = keep | ord | tail | split;
                    o.stats = nullptr;
                    o.lead_stats = nullptr;
                    st = dade_scan(ix, q_rot, probe, nq, k, nprobe, alpha, delta_d, &o, ids, dists, stream);
                    if (st == DADE_OK) st = dade_sync(ix, stream);
                    if (st != DADE_OK) continue;   // an option this shape refuses: not a candidate
                    cudaEventRecord(e0, s);
                    for (int r = 0; r < 3 && st == DADE_OK; ++r)
                        st = dade_scan(ix, q_rot, probe, nq, k, nprobe, alpha, delta_d, &o, ids, dists, stream);
                    cudaEventRecord(e1, s);
                    if (st == DADE_OK) st = dade_sync(ix, stream);
                    float ms = 0.f;
                    if (st != DADE_OK || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                        continue;
                    if (best_ms < 0.f || ms < best_ms) {
                        best_ms = ms;
                        best = Knobs{nt, ord | tail | split};
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms < 0.f) {   // every candidate refused: the library's own message stands
        return st != DADE_OK ? st : DADE_EUNSUPPORTED;
    }
    opts->threads = best.threads;
    opts->flags = keep | best.flags;
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = best;
    return DADE_OK;
}
