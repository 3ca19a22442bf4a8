// autotune.cu -- dade_autotune: the operating point of a search (nprobe,
// delta_d, alpha and the execution schedule) for a recall target, measured
// against the caller's exact neighbours on a sample of queries, and cached.
//
// The paper fixes P_s (alpha) and delta_d by hand (Section 4.1) and sweeps
// nprobe for its recall-QPS curves; a user of the library needs the fastest
// point that still reaches a recall.  The sweep: the smallest nprobe of a
// ladder at which FDScanning (the exact distances of the probed lists, the
// best any DCO can return there) reaches the target, and the next two
// rungs; at each, every delta_d in {16, 32, 64} and every execution variant
// the index serves (tile schedule, with the low-precision prefilter when the
// index has the copy; the seeded schedule with 2 or 3 seed lists, its later
// lists list-major or split over thread blocks; the row
// rounds from 16 or 32 rows with work items of the default size or of 1,024
// rows, and for D > 112 with the tensor-core prefilter too), alpha from the
// most pruning (0.98) down until the
// recall is reached; every passing point is timed and the fastest kept.
// dade_tune then adds the result-neutral options (threads, query order,
// row-major tail, list-major or split passes).  The choice is cached in the
// process, and in a JSON-lines file when the caller names one, keyed by a
// fingerprint of the index (sizes, eigenvalues, list sizes), K, the recall
// target, the query sample size (power-of-two bucket) and the GPU.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace dade {
namespace {

std::mutex g_at_mu;
std::map<std::string, dade_autotune_result> g_at_cache;

uint64_t fnv(uint64_t h, const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

// The identity of an index for the cache: its sizes, spectrum and list sizes.
uint64_t index_fingerprint(const dade_index *ix) {
    uint64_t h = 14695981039346656037ull;
    h = fnv(h, &ix->n, sizeof ix->n);
    h = fnv(h, &ix->d, sizeof ix->d);
    h = fnv(h, &ix->nc, sizeof ix->nc);
    h = fnv(h, ix->lam.data(), sizeof(double) * ix->lam.size());
    for (const ListMeta &m : ix->lists) h = fnv(h, &m.len, sizeof m.len);
    h = fnv(h, &ix->lead_format, sizeof ix->lead_format);
    h = fnv(h, &ix->tail_nb0, sizeof ix->tail_nb0);
    return h;
}

std::string cache_key(const dade_index *ix, int32_t k, float target, int64_t nq) {
    int dev = 0;
    cudaDeviceProp prop{};
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    int bucket = 0;
    while ((1ll << (bucket + 1)) <= nq) ++bucket;
    char buf[512];
    std::snprintf(buf, sizeof buf, "%016llx/k%d/r%.4f/q%d/%s/%d", (unsigned long long)index_fingerprint(ix), k,
                  (double)target, bucket, prop.name, prop.multiProcessorCount);
    return buf;
}

// ---- the cache file: one flat JSON object per line --------------------------------
bool json_string(const std::string &line, const char *field, std::string *out) {
    const std::string tag = std::string("\"") + field + "\": \"";
    const size_t p = line.find(tag);
    if (p == std::string::npos) return false;
    const size_t b = p + tag.size(), e = line.find('"', b);
    if (e == std::string::npos) return false;
    *out = line.substr(b, e - b);
    return true;
}

bool json_number(const std::string &line, const char *field, double *out) {
    const std::string tag = std::string("\"") + field + "\": ";
    const size_t p = line.find(tag);
    if (p == std::string::npos) return false;
    char *end = nullptr;
    const double v = std::strtod(line.c_str() + p + tag.size(), &end);
    if (end == line.c_str() + p + tag.size()) return false;
    *out = v;
    return true;
}

bool cache_file_lookup(const char *path, const std::string &key, dade_autotune_result *r) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    bool found = false;
    std::vector<char> buf(1 << 14);
    while (std::fgets(buf.data(), (int)buf.size(), f)) {
        const std::string line(buf.data());
        std::string kv;
        if (!json_string(line, "key", &kv) || kv != key) continue;
        double v[13];
        const char *names[13] = {"nprobe", "delta_d", "alpha", "schedule", "tile", "seed_lists",
                                 "list_chunk", "threads", "flags", "recall", "ms", "mode", "tc_min_rows"};
        bool ok = true;
        for (int i = 0; i < 13 && ok; ++i) ok = json_number(line, names[i], &v[i]);
        if (!ok) continue;   // a damaged line: not a hit
        dade_autotune_result t{};
        t.nprobe = (int32_t)v[0];
        t.delta_d = (int32_t)v[1];
        t.alpha = (float)v[2];
        t.opts.schedule = (int32_t)v[3];
        t.opts.tile = (int32_t)v[4];
        t.opts.seed_lists = (int32_t)v[5];
        t.opts.list_chunk = (int32_t)v[6];
        t.opts.threads = (int32_t)v[7];
        t.opts.flags = (int32_t)v[8];
        t.recall = (float)v[9];
        t.ms = (float)v[10];
        t.opts.mode = (int32_t)v[11];
        t.opts.tc_min_rows = (int32_t)v[12];
        *r = t;   // the last matching line wins
        found = true;
    }
    std::fclose(f);
    return found;
}

void cache_file_append(const char *path, const std::string &key, const dade_autotune_result &r) {
    FILE *f = std::fopen(path, "a");
    if (!f) return;   // the cache is an optimisation: a read-only path only costs a re-tune
    std::fprintf(f,
                 "{\"key\": \"%s\", \"nprobe\": %d, \"delta_d\": %d, \"alpha\": %.9g, \"schedule\": %d, "
                 "\"tile\": %d, \"seed_lists\": %d, \"list_chunk\": %d, \"threads\": %d, \"flags\": %d, "
                 "\"recall\": %.6f, \"ms\": %.6f, \"mode\": %d, \"tc_min_rows\": %d}\n",
                 key.c_str(), r.nprobe, r.delta_d, (double)r.alpha, r.opts.schedule, r.opts.tile, r.opts.seed_lists,
                 r.opts.list_chunk, r.opts.threads, r.opts.flags, (double)r.recall, (double)r.ms, r.opts.mode,
                 r.opts.tc_min_rows);
    std::fclose(f);
}

} // namespace
} // namespace dade

namespace dade {
namespace {

bool host_buffer(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return true;
    }
    return a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged;
}

struct Variant {
    int32_t schedule, tile, seed_lists, flags, list_chunk, tc_min_rows;
};

// The sweep's state: rotated queries, one probe at a time, scratch results.
struct Tuner {
    const dade_index *ix = nullptr;
    int64_t nq = 0;
    int32_t k = 0;
    int reps = 3;
    cudaStream_t s = nullptr;
    DevBuf qr, probe, ids, dists;
    std::vector<int64_t> gt, host_ids;   // gt: each row sorted
    int cur_np = -1;
    int tried = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;

    ~Tuner() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }

    dade_status probe_for(int np) {
        if (np == cur_np) return DADE_OK;
        DADE_TRY(dade_probe(ix, qr.as<float>(), nq, np, probe.as<int32_t>(), s));
        cur_np = np;
        return DADE_OK;
    }

    // One search at the point; DADE_OK and the recall, or the status the point gave.
    dade_status recall_of(int np, int dd, float alpha, const dade_search_opts &o, double *rc) {
        ++tried;
        DADE_TRY(probe_for(np));
        dade_status st = dade_scan(ix, qr.as<float>(), probe.as<int32_t>(), nq, k, np, alpha, dd, &o,
                                   ids.as<int64_t>(), dists.as<float>(), s);
        if (st == DADE_OK) st = dade_sync(ix, s);
        if (st != DADE_OK) return st;
        DADE_TRY_CUDA(cudaMemcpyAsync(host_ids.data(), ids.p, sizeof(int64_t) * host_ids.size(),
                                      cudaMemcpyDeviceToHost, s));
        DADE_TRY_CUDA(cudaStreamSynchronize(s));
        int64_t hit = 0;
        std::vector<int64_t> row(k);
        for (int64_t q = 0; q < nq; ++q) {
            std::copy(host_ids.begin() + q * k, host_ids.begin() + (q + 1) * k, row.begin());
            std::sort(row.begin(), row.end());
            const int64_t *g = gt.data() + q * k;
            int i = 0, j = 0;
            while (i < k && j < k) {
                if (row[i] < 0 || row[i] < g[j]) ++i;
                else if (g[j] < row[i]) ++j;
                else {
                    ++hit;
                    ++i;
                    ++j;
                }
            }
        }
        *rc = (double)hit / ((double)nq * k);
        return DADE_OK;
    }

    // Mean time of probe + scan at the point over `reps` runs (after one warm-up).
    dade_status time_of(int np, int dd, float alpha, const dade_search_opts &o, float *ms) {
        cur_np = -1;   // the probe is part of what is timed
        DADE_TRY(probe_for(np));
        DADE_TRY(dade_scan(ix, qr.as<float>(), probe.as<int32_t>(), nq, k, np, alpha, dd, &o, ids.as<int64_t>(),
                           dists.as<float>(), s));
        DADE_TRY_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < reps; ++r) {
            DADE_TRY(dade_probe(ix, qr.as<float>(), nq, np, probe.as<int32_t>(), s));
            DADE_TRY(dade_scan(ix, qr.as<float>(), probe.as<int32_t>(), nq, k, np, alpha, dd, &o,
                               ids.as<int64_t>(), dists.as<float>(), s));
        }
        DADE_TRY_CUDA(cudaEventRecord(e1, s));
        DADE_TRY(dade_sync(ix, s));
        DADE_TRY_CUDA(cudaEventSynchronize(e1));
        float t = 0.f;
        DADE_TRY_CUDA(cudaEventElapsedTime(&t, e0, e1));
        *ms = t / (float)reps;
        return DADE_OK;
    }
};

dade_status autotune(const dade_index *ix, const float *q, int64_t nq, int32_t k, const int64_t *gt_ids,
                     const dade_autotune_opts &o, dade_autotune_result *out, cudaStream_t s) {
    Tuner t;
    t.ix = ix;
    t.nq = nq;
    t.k = k;
    t.reps = o.reps > 0 ? o.reps : 3;
    t.s = s;
    DADE_TRY_CUDA(cudaEventCreate(&t.e0));
    DADE_TRY_CUDA(cudaEventCreate(&t.e1));
    std::vector<int32_t> ladder;
    if (o.n_nprobe > 0) {
        ladder.assign(o.nprobe_ladder, o.nprobe_ladder + o.n_nprobe);
    } else {
        for (int32_t v : {4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 64, 96, 128, 192, 256, 384, 512})
            if (v <= ix->nc) ladder.push_back(v);
        if (ladder.empty() || ladder.back() < std::min(ix->nc, 512)) ladder.push_back(std::min(ix->nc, 512));
    }
    const int32_t np_max = *std::max_element(ladder.begin(), ladder.end());
    DADE_TRY(t.qr.alloc(sizeof(float) * (size_t)nq * ix->d));
    DADE_TRY(t.probe.alloc(sizeof(int32_t) * (size_t)nq * np_max));
    DADE_TRY(t.ids.alloc(sizeof(int64_t) * (size_t)nq * k));
    DADE_TRY(t.dists.alloc(sizeof(float) * (size_t)nq * k));
    t.host_ids.resize((size_t)nq * k);
    t.gt.assign(gt_ids, gt_ids + (size_t)nq * k);
    for (int64_t r = 0; r < nq; ++r) std::sort(t.gt.begin() + r * k, t.gt.begin() + (r + 1) * k);
    DADE_TRY(dade_rotate_queries(ix, q, nq, t.qr.as<float>(), s));

    const double target = o.recall_target;
    const bool wide = ix->nb >= 8;   // the list-major kernels and the tensor-core prefilter serve D > 112
    const int32_t tail = ix->tail_nb0 > 0 ? DADE_FLAG_ROW_TAIL : 0;
    // 1. the smallest rung at which the exact scan of the probed lists reaches the target
    size_t r0 = ladder.size();
    for (size_t i = 0; i < ladder.size() && r0 == ladder.size(); ++i) {
        dade_search_opts fd{};
        fd.mode = DADE_MODE_FD;
        fd.schedule = wide ? DADE_SCHED_ROUNDS : DADE_SCHED_TILE;
        fd.tile = wide ? 64 : 128;
        fd.flags = DADE_FLAG_QUERY_ORDER | tail;
        double rc = 0.0;
        DADE_TRY(t.recall_of(ladder[i], 16, 0.5f, fd, &rc));
        if (rc >= target) r0 = i;
    }
    if (r0 == ladder.size()) {
        set_error("dade_autotune: the exact scan of nprobe = " + std::to_string(np_max) +
                  " lists does not reach the recall target on these queries");
        return DADE_EUNSUPPORTED;
    }
    // 2. at that rung and the next two: every delta_d and variant, alpha from the most pruning down
    const int32_t qo = DADE_FLAG_QUERY_ORDER | tail;
    std::vector<Variant> vars = {{DADE_SCHED_TILE, 128, 0, qo, 0, 0}};
    if (ix->lead_format != DADE_LEAD_NONE) vars.push_back({DADE_SCHED_TILE, 128, 0, qo | DADE_FLAG_LEAD, 0, 0});
    for (int32_t S : {2, 3}) {   // later lists list-major, or query-major split over thread blocks
        vars.push_back({DADE_SCHED_SEEDED, 128, S, qo, 0, 0});
        if (wide) vars.push_back({DADE_SCHED_SEEDED, 128, S, qo | DADE_FLAG_SEED_SPLIT, 0, 0});
    }
    for (int32_t r1 : {16, 32})
        for (int32_t chunk : {0, 1024}) {
            vars.push_back({DADE_SCHED_ROUNDS, r1, 0, qo, chunk, 0});
            if (wide)   // the tensor-core prefilter in every round, or only in windows of 16,384 rows on
                for (int32_t tcr : {0, 16384})
                    vars.push_back({DADE_SCHED_ROUNDS, r1, 0, qo | DADE_FLAG_TC_PREFILTER, chunk, tcr});
        }
    const float alphas[] = {0.98f, 0.95f, 0.9f, 0.8f, 0.6f, 0.4f, 0.2f, 0.1f, 0.05f};
    bool have = false;
    dade_autotune_result best{};
    for (size_t i = r0; i < std::min(ladder.size(), r0 + 3); ++i) {
        const int32_t np = ladder[i];
        for (int32_t dd : {16, 32, 64}) {
            if (dd > ix->dp) continue;
            for (const Variant &v : vars) {
                if (v.schedule == DADE_SCHED_SEEDED && v.seed_lists >= np) continue;
                if ((v.flags & DADE_FLAG_TC_PREFILTER) && dd > 64) continue;
                if ((v.flags & DADE_FLAG_LEAD) && dd > ix->lead_dims) continue;
                dade_search_opts so{};
                so.schedule = v.schedule;
                so.tile = v.tile;
                so.seed_lists = v.seed_lists;
                so.flags = v.flags;
                so.list_chunk = v.list_chunk;
                so.tc_min_rows = v.tc_min_rows;
                for (float a : alphas) {
                    double rc = 0.0;
                    if (t.recall_of(np, dd, a, so, &rc) != DADE_OK) break;   // a variant this shape refuses
                    if (rc < target) continue;
                    float ms = 0.f;
                    if (t.time_of(np, dd, a, so, &ms) != DADE_OK) break;
                    if (!have || ms < best.ms) {
                        have = true;
                        best = dade_autotune_result{};
                        best.nprobe = np;
                        best.delta_d = dd;
                        best.alpha = a;
                        best.opts = so;
                        best.recall = (float)rc;
                        best.ms = ms;
                    }
                    break;   // the most pruning alpha that reaches the target
                }
            }
        }
    }
    if (!have) {
        set_error("dade_autotune: no DADE point reached the recall target (the exact scan does at nprobe = " +
                  std::to_string(ladder[r0]) + ")");
        return DADE_EUNSUPPORTED;
    }
    // 3. the result-neutral options of the winner
    set_error("");
    DADE_TRY(t.probe_for(best.nprobe));
    DADE_TRY(dade_tune(ix, t.qr.as<float>(), t.probe.as<int32_t>(), nq, k, best.nprobe, best.alpha, best.delta_d,
                       &best.opts, t.ids.as<int64_t>(), t.dists.as<float>(), s));
    float ms = 0.f;
    DADE_TRY(t.time_of(best.nprobe, best.delta_d, best.alpha, best.opts, &ms));
    best.ms = std::min(best.ms, ms);
    best.points_tried = t.tried;
    *out = best;
    return DADE_OK;
}

} // namespace
} // namespace dade

using namespace dade;

extern "C" void dade_autotune_opts_default(dade_autotune_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->recall_target = 0.95f;
    o->reps = 3;
}

extern "C" dade_status dade_autotune(const dade_index *ix, const float *q, int64_t nq, int32_t k,
                                     const int64_t *gt_ids, const dade_autotune_opts *opts,
                                     dade_autotune_result *out, dade_stream stream) {
    set_error("");
    DADE_CHECK_ARG(ix && q && gt_ids && opts && out, "NULL pointer");
    DADE_CHECK_ARG(nq >= 1 && nq <= 0x7fffffffLL, "nq must be in 1 .. 2^31 - 1");
    DADE_CHECK_ARG(k >= 1 && k <= DADE_MAX_K, "k must be in 1 .. DADE_MAX_K");
    DADE_CHECK_ARG(opts->recall_target > 0.f && opts->recall_target <= 1.f, "recall_target must be in (0, 1]");
    DADE_CHECK_ARG(opts->n_nprobe >= 0 && (opts->n_nprobe == 0 || opts->nprobe_ladder != nullptr),
                   "nprobe_ladder is NULL");
    for (int i = 0; i < opts->n_nprobe; ++i)
        DADE_CHECK_ARG(opts->nprobe_ladder[i] >= 1 && opts->nprobe_ladder[i] <= ix->nc &&
                           (i == 0 || opts->nprobe_ladder[i] > opts->nprobe_ladder[i - 1]),
                       "nprobe_ladder must ascend within 1 .. n_clusters");
    DADE_CHECK_ARG(host_buffer(gt_ids), "gt_ids must be host memory");
    const std::string key = cache_key(ix, k, opts->recall_target, nq);
    {
        std::lock_guard<std::mutex> lock(g_at_mu);
        auto it = g_at_cache.find(key);
        dade_autotune_result r{};
        bool hit = it != g_at_cache.end();
        if (hit) r = it->second;
        else if (opts->cache_path && cache_file_lookup(opts->cache_path, key, &r)) hit = true;
        if (hit && !(opts->flags & DADE_AUTOTUNE_FORCE)) {
            r.from_cache = 1;
            r.points_tried = 0;
            *out = r;
            g_at_cache[key] = r;
            return DADE_OK;
        }
    }
    dade_autotune_result r{};
    dade_status st;
    try {
        st = autotune(ix, q, nq, k, gt_ids, *opts, &r, (cudaStream_t)stream);
    } catch (const std::bad_alloc &) {
        set_error("dade_autotune: host allocation failed");
        st = DADE_ENOMEM;
    }
    if (st != DADE_OK) return st;
    r.from_cache = 0;
    *out = r;
    std::lock_guard<std::mutex> lock(g_at_mu);
    g_at_cache[key] = r;
    if (opts->cache_path) cache_file_append(opts->cache_path, key, r);
    return DADE_OK;
}
