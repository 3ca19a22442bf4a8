// api.cu -- the extern "C" entry points declared in include/dade.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "internal.cuh"

namespace dade {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

// Kernels launched by this library in this process (every launch site calls
// launch_check right after its launch).
static std::atomic<unsigned long long> g_launches{0};

unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

dade_status launch_check(const char *what) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("launch of ") + what + " failed: " + cudaGetErrorString(e));
        return DADE_ECUDA;
    }
    return DADE_OK;
}

namespace {
thread_local Workspace *t_ws = nullptr;

std::mutex g_attr_mu;
std::map<std::pair<const void *, int>, size_t> g_smem_set;            // (kernel, device) -> bytes allowed
std::map<std::tuple<const void *, int, int, size_t>, int> g_resident; // (kernel, device, threads, smem)
} // namespace

dade_status kernel_smem(const void *func, size_t smem) {
    // set even below 48 KB: a kernel whose static shared memory brings the total
    // above 48 KB needs the attribute for its dynamic part as well
    int dev = 0;
    DADE_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_attr_mu);
    size_t &have = g_smem_set[{func, dev}];
    if (have >= smem) return DADE_OK;
    DADE_TRY_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // as much shared memory per SM as the carveout allows, so that several blocks fit
    DADE_TRY_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared));
    have = smem;
    return DADE_OK;
}

dade_status resident_blocks(const void *func, int threads, size_t smem, int *blocks) {
    int dev = 0;
    DADE_TRY_CUDA(cudaGetDevice(&dev));
    DADE_TRY(kernel_smem(func, smem));
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto key = std::make_tuple(func, dev, threads, smem);
    auto it = g_resident.find(key);
    if (it == g_resident.end()) {
        int sms = 0, per = 0;
        DADE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        DADE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, func, threads, smem));
        it = g_resident.emplace(key, std::max(1, sms * std::max(1, per))).first;
    }
    *blocks = it->second;
    return DADE_OK;
}

Workspace &ws(const dade_index *ix) { return t_ws ? *t_ws : ix->ws0; }
WorkspaceScope::WorkspaceScope(Workspace *w) : prev(t_ws) { t_ws = w; }
WorkspaceScope::~WorkspaceScope() { t_ws = prev; }

namespace {
std::atomic<dade_alloc_hook> g_alloc_hook{nullptr};
std::atomic<void *> g_alloc_user{nullptr};
} // namespace

dade_status DevBuf::alloc(size_t b) {
    release();
    if (b == 0) b = 16;
    if (dade_alloc_hook h = g_alloc_hook.load()) {
        if (h(b, g_alloc_user.load()) != 0) {
            set_error(std::string("device allocation of ") + std::to_string(b) + " bytes refused by the allocation hook");
            return DADE_ENOMEM;
        }
    }
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        set_error(std::string("cudaMalloc of ") + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
        return DADE_ENOMEM;
    }
    bytes = b;
    return DADE_OK;
}

dade_status DevBuf::ensure(size_t b) {
    if (p && bytes >= b) return DADE_OK;
    return alloc(b + b / 4);
}

dade_status build_index(const float *base, int64_t n, int32_t d, const dade_build_opts &o, dade_index *ix,
                        cudaStream_t s);

int coef_table(const dade_index *ix, float alpha, int32_t delta_d, double *eps, float *coef, float eps0) {
    const int D = ix->d;
    const int gb = std::min(delta_d / 16, ix->nb);
    const int n_inc = (ix->nb + gb - 1) / gb;
    const double a = (double)alpha;   // alpha is an FP32 value; both sides of a comparison use it as such
    for (int j = 0; j + 1 < n_inc; ++j) {
        const int dd = (j + 1) * gb * 16;          // tested d < D
        if (eps0 >= 0.f) {   // ADSampling: (D/d) P_d > (1 + eps0/sqrt(d))^2 r^2
            const double e = (double)eps0 / std::sqrt((double)dd);
            if (eps) eps[dd] = e;
            coef[j] = (float)((1.0 + e) * (1.0 + e) * (double)dd / (double)D);
            continue;
        }
        double e = std::numeric_limits<double>::infinity();
        const int64_t m = ix->eps_kept;
        if (m > 0) {
            int64_t idx = (int64_t)std::ceil((1.0 - a) * (double)m);
            idx = std::min<int64_t>(std::max<int64_t>(idx, 1), m);
            e = ix->rho[(size_t)(dd / 16 - 1) * m + (idx - 1)] - 1.0;
        }
        if (eps) eps[dd] = e;
        const double c = (1.0 + e) * (1.0 + e) * ix->Lam[dd] / ix->Lam[D];
        coef[j] = (float)c;
    }
    return n_inc;
}

} // namespace dade

using namespace dade;

namespace {

bool is_device_ptr(const void *p) {
    cudaPointerAttributes attr{};
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

dade_status check_device_errors(const dade_index *ix, cudaStream_t s) {
    int h = 0;
    DADE_TRY_CUDA(cudaMemcpyAsync(&h, ix->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DADE_TRY_CUDA(cudaStreamSynchronize(s));
    if (h != 0) {
        DADE_TRY_CUDA(cudaMemsetAsync(ix->errflag.p, 0, sizeof(int), s));
        set_error(h == DADE_ENOMEM ? "a query accepted more candidates than its accept buffer holds (65,536 per "
                                     "pass; lower nprobe or K, or use the tile schedule)"
                                   : "a bounded device-side wait gave up (status recorded by the scan kernel)");
        return (dade_status)h;
    }
    return DADE_OK;
}

dade_status validate_search(const dade_index *ix, int64_t nq, int32_t k, int32_t nprobe, float alpha,
                            int32_t delta_d, const dade_search_opts *opts) {
    DADE_CHECK_ARG(ix != nullptr, "index is NULL");
    DADE_CHECK_ARG(nq >= 0, "nq < 0");
    DADE_CHECK_ARG(k >= 1 && k <= DADE_MAX_K, "k outside 1..DADE_MAX_K");
    DADE_CHECK_ARG(nprobe >= 1 && nprobe <= ix->nc, "nprobe outside 1..n_clusters");
    DADE_CHECK_ARG(nprobe <= 8192, "nprobe > 8192");
    const int mode = opts ? opts->mode : DADE_MODE_DADE;
    DADE_CHECK_ARG(mode == DADE_MODE_DADE || mode == DADE_MODE_FD, "unknown mode");
    const bool ads = opts && opts->estimator == DADE_ESTIMATOR_ADSAMPLING;
    DADE_CHECK_ARG(!opts || opts->estimator == DADE_ESTIMATOR_DADE || ads, "unknown estimator");
    DADE_CHECK_ARG(!ads || (opts->eps0 > 0.f && std::isfinite(opts->eps0)), "ADSampling needs eps0 > 0");
    if (mode == DADE_MODE_DADE) {
        DADE_CHECK_ARG(ads || (alpha > 0.f && alpha < 1.f), "alpha outside (0, 1)");
        DADE_CHECK_ARG(delta_d >= 16 && delta_d <= DADE_MAX_DIM && delta_d % 16 == 0,
                       "delta_d must be a multiple of 16 in [16, 1024]");
    }
    const int tile = opts && opts->tile ? opts->tile : 128;
    // the seeded schedule also takes a tile that holds every list (one epoch per list)
    const bool whole_lists = opts && opts->schedule == DADE_SCHED_SEEDED && tile >= ix->max_list;
    const bool rounds = opts && opts->schedule == DADE_SCHED_ROUNDS;
    DADE_CHECK_ARG((tile >= 32 && tile <= 256 && tile % 32 == 0) || (whole_lists && tile >= 32) || (rounds && tile >= 1),
                   "tile must be a multiple of 32 in [32, 256] (seeded schedule: or at least the longest list; "
                   "row rounds: any first-round row count >= 1)");
    DADE_CHECK_ARG(!opts || (opts->spec >= 0 && opts->spec <= 8), "spec outside 0..8");
    DADE_CHECK_ARG(!opts || opts->threads == 0 || opts->threads == 128 || opts->threads == 256,
                   "threads must be 0 (default), 128 or 256");
    DADE_CHECK_ARG(!opts || opts->schedule == DADE_SCHED_PIPELINED || opts->schedule == DADE_SCHED_TILE ||
                       opts->schedule == DADE_SCHED_SEEDED || opts->schedule == DADE_SCHED_ROUNDS,
                   "unknown schedule");
    DADE_CHECK_ARG(!opts || opts->seed_lists >= 0, "seed_lists < 0");
    DADE_CHECK_ARG(!opts || opts->list_chunk == 0 || (opts->list_chunk >= 64 && opts->list_chunk % 64 == 0),
                   "list_chunk must be 0 or a positive multiple of 64");
    DADE_CHECK_ARG(!opts || opts->stage_ring == 0 || (opts->stage_ring >= 2 && opts->stage_ring <= 8),
                   "stage_ring must be 0 or 2..8");
    DADE_CHECK_ARG(!opts || opts->wait_ns >= 0, "wait_ns < 0");
    DADE_CHECK_ARG(!opts || opts->tc_min_rows >= 0, "tc_min_rows < 0");
    DADE_CHECK_ARG(!opts || opts->stage_dims == 0 ||
                       (opts->stage_dims >= delta_d && delta_d > 0 && opts->stage_dims % delta_d == 0 &&
                        opts->stage_dims <= DADE_MAX_DIM),
                   "stage_dims must be 0 or a multiple of delta_d up to 1024");
    DADE_CHECK_ARG(!opts || (opts->flags & ~(DADE_FLAG_GENERIC_KERNEL | DADE_FLAG_LEAD | DADE_FLAG_QUERY_ORDER |
                                             DADE_FLAG_ROW_TAIL | DADE_FLAG_SEED_SPLIT | DADE_FLAG_TC_PREFILTER |
                                             DADE_FLAG_CHECK_TIMEOUT)) == 0,
                   "unknown flag bits");
    DADE_CHECK_ARG(!opts || !(opts->flags & DADE_FLAG_ROW_TAIL) || ix->tail_nb0 > 0,
                   "DADE_FLAG_ROW_TAIL on an index built without tail_from");
    if (opts && (opts->flags & DADE_FLAG_LEAD)) {
        DADE_CHECK_ARG(mode == DADE_MODE_DADE, "DADE_FLAG_LEAD needs mode DADE_MODE_DADE");
        DADE_CHECK_ARG(ix->lead_format != DADE_LEAD_NONE, "DADE_FLAG_LEAD on an index built without a lead copy");
        DADE_CHECK_ARG(opts->schedule != DADE_SCHED_PIPELINED,
                       "DADE_FLAG_LEAD needs the tile, seeded or row-rounds schedule");
        DADE_CHECK_ARG(std::min(delta_d, ix->dp) <= ix->lead_dims,
                       "DADE_FLAG_LEAD needs min(delta_d, D rounded up to 16) <= the index's lead_dims");
    }
    DADE_CHECK_ARG(!opts || !opts->lead_stats || (opts->flags & (DADE_FLAG_LEAD | DADE_FLAG_TC_PREFILTER)),
                   "lead_stats needs DADE_FLAG_LEAD or DADE_FLAG_TC_PREFILTER");
    return DADE_OK;
}

// Device copies of host inputs / host destinations of device outputs.
struct Staged {
    const float *q = nullptr;
    int64_t *ids = nullptr;
    float *dists = nullptr;
    bool ids_host = false, dists_host = false;
};

dade_status run_scan(const dade_index *ix, const float *q_dev, const int32_t *probe_dev, int64_t nq, int32_t k,
                     int32_t nprobe, float alpha, int32_t delta_d, const dade_search_opts *opts, int64_t *ids,
                     float *dists, cudaStream_t s, const int32_t *qk_dev = nullptr, const int32_t *qnp_dev = nullptr);

dade_status run_search(const dade_index *ix, const float *q_dev, int64_t nq, int32_t k, int32_t nprobe, float alpha,
                       int32_t delta_d, const dade_search_opts *opts, int64_t *ids, float *dists, cudaStream_t s) {
    DADE_TRY(ws(ix).probe.ensure(sizeof(int32_t) * (size_t)nq * nprobe));
    DADE_TRY(dade::probe(ix, q_dev, nq, ix->d, nprobe, ws(ix).probe.as<int32_t>(), s));
    return run_scan(ix, q_dev, ws(ix).probe.as<int32_t>(), nq, k, nprobe, alpha, delta_d, opts, ids, dists, s);
}

dade_status run_scan(const dade_index *ix, const float *q_dev, const int32_t *probe_dev, int64_t nq, int32_t k,
                     int32_t nprobe, float alpha, int32_t delta_d, const dade_search_opts *opts, int64_t *ids,
                     float *dists, cudaStream_t s, const int32_t *qk_dev, const int32_t *qnp_dev) {
    const bool ids_host = !is_device_ptr(ids), dists_host = !is_device_ptr(dists);
    int64_t *ids_d = ids;
    float *dists_d = dists;
    if (ids_host) {
        DADE_TRY(ws(ix).ids.ensure(sizeof(int64_t) * (size_t)nq * k));
        ids_d = ws(ix).ids.as<int64_t>();
    }
    if (dists_host) {
        DADE_TRY(ws(ix).dists.ensure(sizeof(float) * (size_t)nq * k));
        dists_d = ws(ix).dists.as<float>();
    }
    ScanParams p{};
    p.q_rot = q_dev;
    p.q_stride = ix->d;
    p.probe = probe_dev;
    p.nprobe = nprobe;
    p.k = k;
    p.tile = opts && opts->tile ? opts->tile : 128;
    p.mode = opts ? opts->mode : DADE_MODE_DADE;
    p.spec = opts && opts->spec > 0 ? opts->spec : 8;
    p.threads = opts && opts->threads ? opts->threads : 128;
    p.schedule = opts ? opts->schedule : DADE_SCHED_TILE;
    p.seed_lists = opts && opts->seed_lists > 0 ? opts->seed_lists : 2;
    p.stage_dims = opts ? opts->stage_dims : 0;
    p.list_chunk = opts ? opts->list_chunk : 0;
    p.stage_ring = opts ? opts->stage_ring : 0;
    p.generic = opts ? (opts->flags & DADE_FLAG_GENERIC_KERNEL) != 0 : 0;
    p.use_lead = opts ? (opts->flags & DADE_FLAG_LEAD) != 0 : 0;
    p.use_tail = opts ? (opts->flags & DADE_FLAG_ROW_TAIL) != 0 : 0;
    p.seed_split = opts ? (opts->flags & DADE_FLAG_SEED_SPLIT) != 0 : 0;
    p.use_tc = opts ? (opts->flags & DADE_FLAG_TC_PREFILTER) != 0 : 0;
    p.wait_ns = opts ? opts->wait_ns : 0;
    p.tc_min_rows = opts ? opts->tc_min_rows : 0;
    p.check_timeout = opts ? (opts->flags & DADE_FLAG_CHECK_TIMEOUT) != 0 : 0;
    p.q_k = qk_dev;
    p.q_np = qnp_dev;
    p.lead_stats = opts ? opts->lead_stats : nullptr;
    p.delta_d = delta_d;
    const bool ads = opts && opts->estimator == DADE_ESTIMATOR_ADSAMPLING;
    if (p.mode == DADE_MODE_DADE) p.n_inc = coef_table(ix, alpha, delta_d, nullptr, p.coef, ads ? opts->eps0 : -1.f);
    else p.n_inc = 0;
    p.ids = ids_d;
    p.dists = dists_d;
    p.stats = opts ? opts->stats : nullptr;
    if (opts && (opts->flags & DADE_FLAG_QUERY_ORDER)) {
        DADE_TRY(ws(ix).order.ensure(sizeof(int32_t) * (size_t)nq));
        DADE_TRY(dade::order_queries(ix, probe_dev, nq, nprobe, ws(ix).order.as<int32_t>(), s));
        p.order = ws(ix).order.as<int32_t>();
    }
    // counts of the tensor-core prefilter are added up by its passes; without the
    // low-precision prefilter (which writes them) they start from zero
    if (p.lead_stats && !p.use_lead) DADE_TRY_CUDA(cudaMemsetAsync(p.lead_stats, 0, sizeof(int64_t) * (size_t)nq, s));
    DADE_TRY(dade::scan(ix, nq, p, s));
    if (ids_host)
        DADE_TRY_CUDA(cudaMemcpyAsync(ids, ids_d, sizeof(int64_t) * (size_t)nq * k, cudaMemcpyDeviceToHost, s));
    if (dists_host)
        DADE_TRY_CUDA(cudaMemcpyAsync(dists, dists_d, sizeof(float) * (size_t)nq * k, cudaMemcpyDeviceToHost, s));
    if (ids_host || dists_host) return check_device_errors(ix, s);
    return DADE_OK;
}

const float *stage_in(const dade_index *ix, const float *src, size_t count, DevBuf &buf, cudaStream_t s,
                      dade_status *st) {
    *st = DADE_OK;
    if (is_device_ptr(src)) return src;
    if ((*st = buf.ensure(sizeof(float) * count)) != DADE_OK) return nullptr;
    cudaError_t e = cudaMemcpyAsync(buf.p, src, sizeof(float) * count, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
        *st = DADE_ECUDA;
        return nullptr;
    }
    (void)ix;
    return buf.as<float>();
}

} // namespace

extern "C" {

const char *dade_last_error(void) { return g_err.c_str(); }

const char *dade_version(void) { return "dade-gb300 0.1 (sm_103a)"; }

void dade_build_opts_default(dade_build_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->n_clusters = 1;
    o->kmeans_iters = 10;
    o->seed = 0;
    o->eps_pairs = 100000;
}

dade_status dade_build_index(const float *base, int64_t n, int32_t d, const dade_build_opts *opts, dade_index **out,
                             dade_stream stream) {
    g_err.clear();
    DADE_CHECK_ARG(base != nullptr && out != nullptr && opts != nullptr, "NULL pointer");
    DADE_CHECK_ARG(n >= 2, "n < 2");
    DADE_CHECK_ARG(d >= 1 && d <= DADE_MAX_DIM, "d outside 1..DADE_MAX_DIM");
    DADE_CHECK_ARG(n <= 0x7fffffffLL, "n must fit in 31 bits (ids are stored as int32)");
    DADE_CHECK_ARG(opts->n_clusters >= 1 && opts->n_clusters <= n, "n_clusters outside 1..n");
    DADE_CHECK_ARG(opts->kmeans_iters >= 0 && opts->kmeans_iters <= 1000, "kmeans_iters outside 0..1000");
    DADE_CHECK_ARG(opts->eps_pairs >= 1, "eps_pairs < 1");
    DADE_CHECK_ARG(opts->lead_format == DADE_LEAD_NONE || opts->lead_format == DADE_LEAD_BF16 ||
                       opts->lead_format == DADE_LEAD_FP8,
                   "unknown lead_format");
    if (opts->lead_format == DADE_LEAD_NONE)
        DADE_CHECK_ARG(opts->lead_dims == 0, "lead_dims given without a lead_format");
    else
        DADE_CHECK_ARG(opts->lead_dims >= 16 && opts->lead_dims % 16 == 0 && opts->lead_dims <= (d + 15) / 16 * 16,
                       "lead_dims must be a multiple of 16 in [16, D rounded up to 16]");
    DADE_CHECK_ARG(opts->transform == DADE_TRANSFORM_PCA || opts->transform == DADE_TRANSFORM_RANDOM ||
                       (opts->transform == DADE_TRANSFORM_GIVEN && opts->basis != nullptr),
                   "unknown transform, or DADE_TRANSFORM_GIVEN without a basis");
    DADE_CHECK_ARG(opts->tail_from == 0 || (opts->tail_from >= 16 && opts->tail_from % 16 == 0 &&
                                            opts->tail_from < (d + 15) / 16 * 16),
                   "tail_from must be 0 or a multiple of 16 in [16, D rounded up to 16)");
    *out = nullptr;
    dade_index *ix = new (std::nothrow) dade_index();
    if (!ix) {
        set_error("host allocation of the index failed");
        return DADE_ENOMEM;
    }
    dade_status st = build_index(base, n, d, *opts, ix, (cudaStream_t)stream);
    if (st != DADE_OK) {
        delete ix;
        return st;
    }
    *out = ix;
    return DADE_OK;
}

unsigned long long dade_launch_count(void) { return dade::launch_count(); }

void dade_free_index(dade_index *ix) {
    dade::tune_forget(ix);
    delete ix;
}

dade_status dade_save_index(const dade_index *ix, const char *path) {
    g_err.clear();
    DADE_CHECK_ARG(ix != nullptr && path != nullptr, "NULL pointer");
    return dade::save_index(ix, path);
}

dade_status dade_load_index(const char *path, dade_index **out) {
    g_err.clear();
    DADE_CHECK_ARG(path != nullptr && out != nullptr, "NULL pointer");
    *out = nullptr;
    dade_index *ix = new (std::nothrow) dade_index();
    if (!ix) {
        set_error("host allocation of the index failed");
        return DADE_ENOMEM;
    }
    dade_status st;
    try {
        st = dade::load_index(path, ix);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed while loading the index");
        st = DADE_ENOMEM;
    }
    if (st != DADE_OK) {
        delete ix;
        return st;
    }
    *out = ix;
    return DADE_OK;
}

dade_status dade_rotate_queries(const dade_index *ix, const float *q, int64_t nq, float *q_rot, dade_stream stream) {
    g_err.clear();
    DADE_CHECK_ARG(ix != nullptr, "index is NULL");
    DADE_CHECK_ARG(nq >= 0, "nq < 0");
    if (nq == 0) return DADE_OK;
    DADE_CHECK_ARG(q != nullptr && q_rot != nullptr, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    dade_status st;
    const float *qd = stage_in(ix, q, (size_t)nq * ix->d, ws(ix).qin, s, &st);
    if (!qd) return st;
    const bool out_host = !is_device_ptr(q_rot);
    float *od = q_rot;
    if (out_host) {
        DADE_TRY(ws(ix).qrot.ensure(sizeof(float) * (size_t)nq * ix->d));
        od = ws(ix).qrot.as<float>();
    }
    DADE_TRY(dade::rotate(ix, qd, nq, ix->d, od, s));
    if (out_host) {
        DADE_TRY_CUDA(cudaMemcpyAsync(q_rot, od, sizeof(float) * (size_t)nq * ix->d, cudaMemcpyDeviceToHost, s));
        DADE_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return DADE_OK;
}

dade_status dade_probe(const dade_index *ix, const float *q_rot, int64_t nq, int32_t nprobe, int32_t *probe,
                       dade_stream stream) {
    g_err.clear();
    DADE_CHECK_ARG(ix != nullptr, "index is NULL");
    DADE_CHECK_ARG(nq >= 0, "nq < 0");
    DADE_CHECK_ARG(nprobe >= 1 && nprobe <= ix->nc && nprobe <= 8192, "nprobe outside 1..min(n_clusters, 8192)");
    if (nq == 0) return DADE_OK;
    DADE_CHECK_ARG(q_rot != nullptr && probe != nullptr, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    dade_status st;
    const float *qd = stage_in(ix, q_rot, (size_t)nq * ix->d, ws(ix).qrot, s, &st);
    if (!qd) return st;
    const bool out_host = !is_device_ptr(probe);
    int32_t *pd = probe;
    if (out_host) {
        DADE_TRY(ws(ix).probe.ensure(sizeof(int32_t) * (size_t)nq * nprobe));
        pd = ws(ix).probe.as<int32_t>();
    }
    DADE_TRY(dade::probe(ix, qd, nq, ix->d, nprobe, pd, s));
    if (out_host) {
        DADE_TRY_CUDA(cudaMemcpyAsync(probe, pd, sizeof(int32_t) * (size_t)nq * nprobe, cudaMemcpyDeviceToHost, s));
        DADE_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return DADE_OK;
}

dade_status dade_search(const dade_index *ix, const float *q_rot, int64_t nq, int32_t k, int32_t nprobe, float alpha,
                        int32_t delta_d, const dade_search_opts *opts, int64_t *ids, float *dists,
                        dade_stream stream) {
    g_err.clear();
    DADE_TRY(validate_search(ix, nq, k, nprobe, alpha, delta_d, opts));
    if (nq == 0) return DADE_OK;
    DADE_CHECK_ARG(q_rot != nullptr && ids != nullptr && dists != nullptr, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    dade_status st;
    const float *qd = stage_in(ix, q_rot, (size_t)nq * ix->d, ws(ix).qrot, s, &st);
    if (!qd) return st;
    return run_search(ix, qd, nq, k, nprobe, alpha, delta_d, opts, ids, dists, s);
}

dade_status dade_scan(const dade_index *ix, const float *q_rot, const int32_t *probe, int64_t nq, int32_t k,
                      int32_t nprobe, float alpha, int32_t delta_d, const dade_search_opts *opts, int64_t *ids,
                      float *dists, dade_stream stream) {
    g_err.clear();
    DADE_TRY(validate_search(ix, nq, k, nprobe, alpha, delta_d, opts));
    if (nq == 0) return DADE_OK;
    DADE_CHECK_ARG(q_rot != nullptr && probe != nullptr && ids != nullptr && dists != nullptr, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    dade_status st;
    const float *qd = stage_in(ix, q_rot, (size_t)nq * ix->d, ws(ix).qrot, s, &st);
    if (!qd) return st;
    const int32_t *pd = probe;
    if (!is_device_ptr(probe)) {
        for (int64_t t = 0; t < nq * (int64_t)nprobe; ++t)
            DADE_CHECK_ARG(probe[t] >= 0 && probe[t] < ix->nc, "probe[] holds a list id outside 0..n_clusters-1");
        DADE_TRY(ws(ix).probe.ensure(sizeof(int32_t) * (size_t)nq * nprobe));
        DADE_TRY_CUDA(cudaMemcpyAsync(ws(ix).probe.p, probe, sizeof(int32_t) * (size_t)nq * nprobe,
                                      cudaMemcpyHostToDevice, s));
        pd = ws(ix).probe.as<int32_t>();
    }
    return run_scan(ix, qd, pd, nq, k, nprobe, alpha, delta_d, opts, ids, dists, s);
}

dade_status dade_query(const dade_index *ix, const float *q, int64_t nq, int32_t k, int32_t nprobe, float alpha,
                       int32_t delta_d, const dade_search_opts *opts, int64_t *ids, float *dists, dade_stream stream) {
    g_err.clear();
    DADE_TRY(validate_search(ix, nq, k, nprobe, alpha, delta_d, opts));
    if (nq == 0) return DADE_OK;
    DADE_CHECK_ARG(q != nullptr && ids != nullptr && dists != nullptr, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    dade_status st;
    const float *qd = stage_in(ix, q, (size_t)nq * ix->d, ws(ix).qin, s, &st);
    if (!qd) return st;
    DADE_TRY(ws(ix).qrot.ensure(sizeof(float) * (size_t)nq * ix->d));
    DADE_TRY(dade::rotate(ix, qd, nq, ix->d, ws(ix).qrot.as<float>(), s));
    return run_search(ix, ws(ix).qrot.as<float>(), nq, k, nprobe, alpha, delta_d, opts, ids, dists, s);
}

dade_status dade_query_mixed(const dade_index *ix, const float *q, int64_t nq, const int32_t *k, const int32_t *nprobe,
                             int32_t k_max, int32_t nprobe_max, float alpha, int32_t delta_d,
                             const dade_search_opts *opts, int64_t *ids, float *dists, dade_stream stream) {
    g_err.clear();
    DADE_TRY(validate_search(ix, nq, k_max, nprobe_max, alpha, delta_d, opts));
    DADE_CHECK_ARG(!opts || opts->schedule == DADE_SCHED_TILE || opts->schedule == DADE_SCHED_ROUNDS,
                   "per-query K and nprobe need the tile schedule or the row rounds");
    if (nq == 0) return DADE_OK;
    DADE_CHECK_ARG(q != nullptr && k != nullptr && nprobe != nullptr && ids != nullptr && dists != nullptr,
                   "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t *kd = k, *npd = nprobe;
    if (!is_device_ptr(k)) {
        for (int64_t i = 0; i < nq; ++i) DADE_CHECK_ARG(k[i] >= 1 && k[i] <= k_max, "k[i] outside 1..k_max");
        DADE_TRY(ws(ix).qk.ensure(sizeof(int32_t) * (size_t)nq));
        DADE_TRY_CUDA(cudaMemcpyAsync(ws(ix).qk.p, k, sizeof(int32_t) * (size_t)nq, cudaMemcpyHostToDevice, s));
        kd = ws(ix).qk.as<int32_t>();
    }
    if (!is_device_ptr(nprobe)) {
        for (int64_t i = 0; i < nq; ++i)
            DADE_CHECK_ARG(nprobe[i] >= 1 && nprobe[i] <= nprobe_max, "nprobe[i] outside 1..nprobe_max");
        DADE_TRY(ws(ix).qnp.ensure(sizeof(int32_t) * (size_t)nq));
        DADE_TRY_CUDA(cudaMemcpyAsync(ws(ix).qnp.p, nprobe, sizeof(int32_t) * (size_t)nq, cudaMemcpyHostToDevice, s));
        npd = ws(ix).qnp.as<int32_t>();
    }
    dade_status st;
    const float *qd = stage_in(ix, q, (size_t)nq * ix->d, ws(ix).qin, s, &st);
    if (!qd) return st;
    DADE_TRY(ws(ix).qrot.ensure(sizeof(float) * (size_t)nq * ix->d));
    DADE_TRY(dade::rotate(ix, qd, nq, ix->d, ws(ix).qrot.as<float>(), s));
    // the nprobe_max nearest lists in (distance, id) order: a query's first nprobe[i]
    // of them are its own nprobe[i] nearest
    DADE_TRY(ws(ix).probe.ensure(sizeof(int32_t) * (size_t)nq * nprobe_max));
    DADE_TRY(dade::probe(ix, ws(ix).qrot.as<float>(), nq, ix->d, nprobe_max, ws(ix).probe.as<int32_t>(), s));
    return run_scan(ix, ws(ix).qrot.as<float>(), ws(ix).probe.as<int32_t>(), nq, k_max, nprobe_max, alpha, delta_d,
                    opts, ids, dists, s, kd, npd);
}

dade_status dade_reserve(dade_index *ix, int64_t max_nq, int32_t max_nprobe) {
    g_err.clear();
    DADE_CHECK_ARG(ix != nullptr, "index is NULL");
    DADE_CHECK_ARG(max_nq >= 0 && max_nprobe >= 1 && max_nprobe <= ix->nc, "bad limits");
    DADE_TRY(ws(ix).dist.ensure(sizeof(float) * (size_t)max_nq * ix->nc));
    DADE_TRY(ws(ix).probe.ensure(sizeof(int32_t) * (size_t)max_nq * max_nprobe));
    DADE_TRY(ws(ix).qrot.ensure(sizeof(float) * (size_t)max_nq * ix->d));
    DADE_TRY(ws(ix).qin.ensure(sizeof(float) * (size_t)max_nq * ix->d));
    DADE_TRY(ws(ix).order.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(max_nq, 1)));
    DADE_TRY(ws(ix).ordcnt.ensure(sizeof(int) * (size_t)ix->nc));
    // tensor-core operand image of a query batch: 128-row tiles x 32-dim chunks x 32 KB
    DADE_TRY(ws(ix).aimg.ensure((size_t)((max_nq + 127) / 128) * ((ix->d + 31) / 32) * 32768));
    DADE_TRY(ws(ix).anorm.ensure(sizeof(float) * (size_t)std::max<int64_t>(max_nq, 1)));
    return DADE_OK;
}

dade_status dade_eps_table(const dade_index *ix, float alpha, int32_t delta_d, double *eps, float *coef) {
    g_err.clear();
    DADE_CHECK_ARG(ix != nullptr && eps != nullptr, "NULL pointer");
    DADE_CHECK_ARG(alpha > 0.f && alpha < 1.f, "alpha outside (0, 1)");
    DADE_CHECK_ARG(delta_d >= 16 && delta_d % 16 == 0 && delta_d <= DADE_MAX_DIM, "bad delta_d");
    for (int i = 0; i <= ix->d; ++i) eps[i] = std::numeric_limits<double>::quiet_NaN();
    float c[DADE_MAX_DIM / DADE_BLOCK];
    int n_inc = coef_table(ix, alpha, delta_d, eps, c);
    if (coef) {
        for (int i = 0; i <= ix->d; ++i) coef[i] = std::numeric_limits<float>::quiet_NaN();
        const int gb = std::min(delta_d / 16, ix->nb);
        for (int j = 0; j + 1 < n_inc; ++j) coef[(j + 1) * gb * 16] = c[j];
    }
    return DADE_OK;
}

dade_status dade_sync(const dade_index *ix, dade_stream stream) {
    g_err.clear();
    DADE_CHECK_ARG(ix != nullptr, "index is NULL");
    return check_device_errors(ix, (cudaStream_t)stream);
}

dade_status dade_index_info(const dade_index *ix, dade_info *info) {
    g_err.clear();
    DADE_CHECK_ARG(ix != nullptr && info != nullptr, "NULL pointer");
    info->n = ix->n;
    info->d = ix->d;
    info->d_pad = ix->dp;
    info->n_clusters = ix->nc;
    info->max_list = ix->max_list;
    info->eps_kept = ix->eps_kept;
    info->data_bytes = (int64_t)ix->data.bytes;
    info->device_bytes = (int64_t)(ix->data.bytes + ix->ids.bytes + ix->meta.bytes + ix->cent.bytes + ix->cnorm.bytes +
                                   ix->WT32.bytes + ix->cent_img.bytes + ix->wt_img.bytes + ix->mu32.bytes + ix->errflag.bytes + ix->lead.bytes +
                                   ix->lead_err.bytes + ix->lead_scale.bytes + ix->tail.bytes);
    info->kmeans_iters = (int32_t)ix->kmeans_obj.size();
    info->lead_format = ix->lead_format;
    info->lead_dims = ix->lead_dims;
    info->tail_from = ix->tail_nb0 * 16;
    return DADE_OK;
}

dade_status dade_index_export(const dade_index *ix, int32_t field, void *dst, size_t bytes) {
    g_err.clear();
    DADE_CHECK_ARG(ix != nullptr && dst != nullptr, "NULL pointer");
    const int d = ix->d;
    auto need = [&](size_t b) -> dade_status {
        if (bytes != b) {
            set_error("invalid argument: export size mismatch (expected " + std::to_string(b) + " bytes)");
            return DADE_EINVAL;
        }
        return DADE_OK;
    };
    switch (field) {
    case DADE_FIELD_MEAN:
        DADE_TRY(need(sizeof(double) * d));
        std::memcpy(dst, ix->mu.data(), bytes);
        return DADE_OK;
    case DADE_FIELD_BASIS:
        DADE_TRY(need(sizeof(double) * (size_t)d * d));
        std::memcpy(dst, ix->W.data(), bytes);
        return DADE_OK;
    case DADE_FIELD_EIGVAL:
        DADE_TRY(need(sizeof(double) * d));
        std::memcpy(dst, ix->lam.data(), bytes);
        return DADE_OK;
    case DADE_FIELD_ASSIGN:
        DADE_TRY(need(sizeof(int32_t) * (size_t)ix->n));
        std::memcpy(dst, ix->assign.data(), bytes);
        return DADE_OK;
    case DADE_FIELD_RHO:
        DADE_TRY(need(sizeof(double) * ix->rho.size()));
        if (bytes) std::memcpy(dst, ix->rho.data(), bytes);
        return DADE_OK;
    case DADE_FIELD_KMEANS_OBJ:
        DADE_TRY(need(sizeof(double) * ix->kmeans_obj.size()));
        if (bytes) std::memcpy(dst, ix->kmeans_obj.data(), bytes);
        return DADE_OK;
    case DADE_FIELD_CENTROIDS: {
        DADE_TRY(need(sizeof(float) * (size_t)ix->nc * d));
        std::vector<float> c((size_t)ix->nc * ix->dp);
        DADE_TRY_CUDA(cudaMemcpy(c.data(), ix->cent.p, sizeof(float) * c.size(), cudaMemcpyDeviceToHost));
        float *o = static_cast<float *>(dst);
        for (int r = 0; r < ix->nc; ++r) std::memcpy(o + (size_t)r * d, c.data() + (size_t)r * ix->dp, sizeof(float) * d);
        return DADE_OK;
    }
    case DADE_FIELD_ROTATED: {
        DADE_TRY(need(sizeof(float) * (size_t)ix->n * d));
        if (ix->shard >= 0) std::memset(dst, 0, bytes);   // rows of lists the shard does not hold
        std::vector<float> packed((size_t)ix->data_floats);
        std::vector<int32_t> ids((size_t)ix->slots);
        DADE_TRY_CUDA(cudaMemcpy(packed.data(), ix->data.p, sizeof(float) * packed.size(), cudaMemcpyDeviceToHost));
        DADE_TRY_CUDA(cudaMemcpy(ids.data(), ix->ids.p, sizeof(int32_t) * ids.size(), cudaMemcpyDeviceToHost));
        float *o = static_cast<float *>(dst);
        for (int c = 0; c < ix->nc; ++c) {
            const ListMeta &m = ix->lists[c];
            for (int i = 0; i < m.len; ++i) {
                int64_t id = ids[m.slot + i];
                for (int k = 0; k < d; ++k)
                    o[id * d + k] = packed[m.base + (int64_t)(k / 16) * m.np * 16 + (int64_t)i * 16 + k % 16];
            }
        }
        return DADE_OK;
    }
    case DADE_FIELD_LEAD_DEQ:
    case DADE_FIELD_LEAD_ERR:
    case DADE_FIELD_LEAD_SCALE: {
        DADE_CHECK_ARG(ix->lead_format != DADE_LEAD_NONE, "the index has no lead copy");
        const int lnb = ix->lead_nb, es = ix->lead_format == DADE_LEAD_BF16 ? 2 : 1;
        std::vector<float> scale((size_t)ix->nc * lnb);
        DADE_TRY_CUDA(cudaMemcpy(scale.data(), ix->lead_scale.p, sizeof(float) * scale.size(), cudaMemcpyDeviceToHost));
        if (field == DADE_FIELD_LEAD_SCALE) {
            DADE_TRY(need(sizeof(float) * scale.size()));
            std::memcpy(dst, scale.data(), bytes);
            return DADE_OK;
        }
        std::vector<int32_t> ids((size_t)ix->slots);
        DADE_TRY_CUDA(cudaMemcpy(ids.data(), ix->ids.p, sizeof(int32_t) * ids.size(), cudaMemcpyDeviceToHost));
        float *o = static_cast<float *>(dst);
        if (field == DADE_FIELD_LEAD_ERR) {
            DADE_TRY(need(sizeof(float) * (size_t)lnb * ix->n));
            if (ix->shard >= 0) std::memset(dst, 0, bytes);
            std::vector<float> err((size_t)ix->slots * lnb);
            DADE_TRY_CUDA(cudaMemcpy(err.data(), ix->lead_err.p, sizeof(float) * err.size(), cudaMemcpyDeviceToHost));
            for (int c = 0; c < ix->nc; ++c) {
                const ListMeta &m = ix->lists[c];
                for (int i = 0; i < m.len; ++i)
                    for (int b = 0; b < lnb; ++b) o[(size_t)b * ix->n + ids[m.slot + i]] = err[(size_t)b * ix->slots + m.slot + i];
            }
            return DADE_OK;
        }
        DADE_TRY(need(sizeof(float) * (size_t)ix->n * ix->lead_dims));
        if (ix->shard >= 0) std::memset(dst, 0, bytes);
        std::vector<unsigned char> codes(ix->lead.bytes);
        DADE_TRY_CUDA(cudaMemcpy(codes.data(), ix->lead.p, codes.size(), cudaMemcpyDeviceToHost));
        for (int c = 0; c < ix->nc; ++c) {
            const ListMeta &m = ix->lists[c];
            for (int i = 0; i < m.len; ++i) {
                const int64_t id = ids[m.slot + i];
                for (int b = 0; b < lnb; ++b) {
                    const unsigned char *src = codes.data() + (m.slot * lnb * 16 + (int64_t)b * m.np * 16 + (int64_t)i * 16) * es;
                    for (int k = 0; k < 16; ++k) {
                        float v;
                        if (es == 2) {
                            uint32_t bits = (uint32_t)(src[2 * k] | (src[2 * k + 1] << 8)) << 16;
                            std::memcpy(&v, &bits, 4);
                        } else {
                            const __half h(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)src[k], __NV_E4M3));
                            v = scale[(size_t)c * lnb + b] * __half2float(h);
                        }
                        o[(size_t)id * ix->lead_dims + b * 16 + k] = v;
                    }
                }
            }
        }
        return DADE_OK;
    }
    default:
        set_error("invalid argument: unknown field");
        return DADE_EINVAL;
    }
}

dade_status dade_host_sym_eig(double *a, int32_t n, double *w, double *v) {
    g_err.clear();
    DADE_CHECK_ARG(a != nullptr && w != nullptr && v != nullptr, "NULL pointer");
    DADE_CHECK_ARG(n >= 1 && n <= 4096, "n outside 1..4096");
    std::vector<double> A(a, a + (size_t)n * n), W, V;
    if (!dade::sym_eig(n, A, W, V)) {
        set_error("symmetric QR did not converge");
        return DADE_EUNSUPPORTED;
    }
    std::memcpy(w, W.data(), sizeof(double) * n);
    std::memcpy(v, V.data(), sizeof(double) * (size_t)n * n);
    std::memcpy(a, A.data(), sizeof(double) * (size_t)n * n);
    return DADE_OK;
}

} // extern "C"

extern "C" void dade_set_alloc_hook(dade_alloc_hook hook, void *user) {
    g_alloc_user.store(user);
    g_alloc_hook.store(hook);
}
