// server.cpp -- continuous-batching request loop over one resident index.
//
// Requests (host queries, per-request K, nprobe, alpha, delta_d) are queued
// by dade_server_submit.  One dispatcher thread admits them into slots: a
// slot is a CUDA stream with its own device workspace, pinned staging
// buffers and a completion event, so batches in different slots overlap on
// the GPU.  When a slot is free the dispatcher forms a batch from the oldest
// pending request and every later pending request it can run with, up to
// max_batch queries: under the tile schedule, and the row rounds where they
// run list-major, any request with the same alpha and delta_d (one launch
// serves a K and an nprobe per query, dade_query_mixed), otherwise the same
// (K, nprobe, alpha, delta_d).  It copies the queries in, runs the query step (rotation, probe,
// scan) on the slot's stream, copies the results out and records the event.
// A finished slot's results are scattered to the requests' host buffers and
// their tickets complete; requests that arrived meanwhile are admitted as
// slots free up.  Admission is by device bytes when a budget is set: a batch
// starts only if the slots' fixed buffers and the workspace every slot has
// grown to, plus what this batch adds, stay within the budget.  Every query's
// result depends only on that query (the step has no cross-query arithmetic),
// so a request gets the same result alone and in any mix.  A cancelled
// request leaves the queue, or, in flight, completes without its results
// being written to the caller's buffers.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    const float *q;
    int64_t nq;
    int32_t k, nprobe, delta_d;
    float alpha;
    int64_t *ids;
    float *dists;
    Clock::time_point t0;
};

struct Ticket {
    bool done = false;
    bool cancelled = false;
    dade_status status = DADE_OK;
    double latency = 0.0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    dade::Workspace ws;
    dade::DevBuf q_dev, ids_dev, dists_dev;
    float *q_host = nullptr;
    int64_t *ids_host = nullptr;
    float *dists_host = nullptr;
    int32_t *k_host = nullptr, *np_host = nullptr;   // per-query K and nprobe of a mixed batch
    bool busy = false;
    int32_t k = 0;                                   // the batch's result row stride (largest K)
    int64_t ws_bytes = 0;                            // workspace this slot's batches grew to (estimate)
    std::vector<Request> reqs;
};

} // namespace

struct dade_server {
    const dade_index *ix = nullptr;
    dade_server_opts o{};
    std::vector<std::unique_ptr<Slot>> slots;
    std::mutex mu;
    std::condition_variable cv_submit, cv_done;
    std::deque<Request> pending;
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    dade_server_stats st{};
    int device = 0;

    ~dade_server() {
        {
            std::lock_guard<std::mutex> g(mu);
            stop = true;
        }
        cv_submit.notify_all();
        if (worker.joinable()) worker.join();
        for (auto &sp : slots) {
            Slot &s = *sp;
            if (s.stream) cudaStreamSynchronize(s.stream);
            if (s.done) cudaEventDestroy(s.done);
            if (s.stream) cudaStreamDestroy(s.stream);
            if (s.q_host) cudaFreeHost(s.q_host);
            if (s.ids_host) cudaFreeHost(s.ids_host);
            if (s.dists_host) cudaFreeHost(s.dists_host);
            if (s.k_host) cudaFreeHost(s.k_host);
            if (s.np_host) cudaFreeHost(s.np_host);
        }
    }

    // Whether one launch serves a K and an nprobe per query at this delta_d: the tile
    // schedule, or the row rounds where they run list-major (D > 112, delta_d of 16, 32,
    // 64 or 128 dims, neither the split passes nor the low-precision prefilter).
    bool mixes(int32_t delta_d) const {
        if (o.schedule == DADE_SCHED_TILE) return true;
        if (o.schedule != DADE_SCHED_ROUNDS || ix->nb < 8 || (o.flags & (DADE_FLAG_SEED_SPLIT | DADE_FLAG_LEAD)))
            return false;
        const int gb = o.mode == DADE_MODE_FD ? 8 : std::min(delta_d / 16, ix->nb);
        return gb == 1 || gb == 2 || gb == 4 || gb == 8;
    }

    // Workspace bytes of a batch of nq queries (estimate of what the query step grows it to):
    // raw and rotated queries, probe distances and lists, results, the tensor-core operand
    // image, query order and per-query arrays; with r frozen over whole lists, the accept buffer.
    int64_t batch_bytes(int64_t nq, int32_t kmax, int32_t npmax) const {
        const int64_t d = ix->d;
        int64_t per = d * 4 * 2 + (int64_t)ix->nc * 4 + (int64_t)npmax * 4 + (int64_t)kmax * 12 + d * 8 + 72;
        if (o.schedule == DADE_SCHED_SEEDED || o.schedule == DADE_SCHED_ROUNDS)
            per += std::min<int64_t>((int64_t)npmax * std::max(ix->max_list, 1), 1 << 16) * 8;
        return nq * per;
    }
    int64_t fixed_bytes() const { return (int64_t)o.max_batch * ((int64_t)ix->d * 4 + (int64_t)o.max_k * 12); }
    int64_t used_bytes() const {
        int64_t u = 0;
        for (const auto &sp : slots) u += fixed_bytes() + sp->ws_bytes;
        return u;
    }
    // Whether slot s may run a batch of `need` workspace bytes within the budget.
    bool fits(const Slot &s, int64_t need) const {
        return o.device_budget <= 0 || used_bytes() + std::max<int64_t>(0, need - s.ws_bytes) <= o.device_budget;
    }

    // Runs one batch on slot s (dispatcher thread).  Returns the status of the launches.
    dade_status launch(Slot &s) {
        dade::WorkspaceScope scope(&s.ws);
        const int d = ix->d;
        int64_t nq = 0;
        for (const Request &r : s.reqs) {
            std::memcpy(s.q_host + nq * d, r.q, sizeof(float) * (size_t)r.nq * d);
            nq += r.nq;
        }
        const Request &r0 = s.reqs.front();
        int32_t kmax = 0, npmax = 0;
        int64_t qi = 0;
        for (const Request &r : s.reqs) {
            kmax = std::max(kmax, r.k);
            npmax = std::max(npmax, r.nprobe);
            for (int64_t i = 0; i < r.nq; ++i, ++qi) {
                s.k_host[qi] = r.k;
                s.np_host[qi] = r.nprobe;
            }
        }
        s.k = kmax;
        DADE_TRY_CUDA(cudaMemcpyAsync(s.q_dev.p, s.q_host, sizeof(float) * (size_t)nq * d, cudaMemcpyHostToDevice,
                                      s.stream));
        dade_search_opts so{};
        so.mode = o.mode;
        so.tile = o.tile;
        so.threads = o.threads;
        so.schedule = o.schedule;
        so.seed_lists = o.seed_lists;
        so.flags = o.flags;
        so.stage_dims = o.stage_dims;
        so.list_chunk = o.list_chunk;
        so.tc_min_rows = o.tc_min_rows;
        if (mixes(r0.delta_d))
            DADE_TRY(dade_query_mixed(ix, s.q_dev.as<float>(), nq, s.k_host, s.np_host, kmax, npmax, r0.alpha,
                                      r0.delta_d, &so, s.ids_dev.as<int64_t>(), s.dists_dev.as<float>(),
                                      (dade_stream)s.stream));
        else
            DADE_TRY(dade_query(ix, s.q_dev.as<float>(), nq, r0.k, r0.nprobe, r0.alpha, r0.delta_d, &so,
                                s.ids_dev.as<int64_t>(), s.dists_dev.as<float>(), (dade_stream)s.stream));
        DADE_TRY_CUDA(cudaMemcpyAsync(s.ids_host, s.ids_dev.p, sizeof(int64_t) * (size_t)nq * kmax,
                                      cudaMemcpyDeviceToHost, s.stream));
        DADE_TRY_CUDA(cudaMemcpyAsync(s.dists_host, s.dists_dev.p, sizeof(float) * (size_t)nq * kmax,
                                      cudaMemcpyDeviceToHost, s.stream));
        DADE_TRY_CUDA(cudaEventRecord(s.done, s.stream));
        return DADE_OK;
    }

    // Scatters a finished slot's results and completes its tickets (called with mu held).
    void finish(Slot &s, dade_status status) {
        const auto now = Clock::now();
        int64_t off = 0;
        for (const Request &r : s.reqs) {
            Ticket &t = tickets[r.ticket];
            if (status == DADE_OK && !t.cancelled)   // the request's own K columns of its rows
                for (int64_t i = 0; i < r.nq; ++i) {
                    std::memcpy(r.ids + i * r.k, s.ids_host + (off + i) * s.k, sizeof(int64_t) * (size_t)r.k);
                    std::memcpy(r.dists + i * r.k, s.dists_host + (off + i) * s.k, sizeof(float) * (size_t)r.k);
                }
            off += r.nq;
            t.done = true;
            t.status = t.cancelled ? DADE_ECANCELLED : status;
            t.latency = std::chrono::duration<double>(now - r.t0).count();
        }
        st.requests_done += (int64_t)s.reqs.size();
        s.reqs.clear();
        s.busy = false;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            // completions
            int busy = 0;
            for (auto &sp : slots) {
                Slot &s = *sp;
                if (!s.busy) continue;
                const cudaError_t e = cudaEventQuery(s.done);
                if (e == cudaSuccess) {
                    finish(s, DADE_OK);
                } else if (e != cudaErrorNotReady) {
                    cudaGetLastError();
                    finish(s, DADE_ECUDA);
                } else {
                    ++busy;
                }
            }
            cv_done.notify_all();
            // admissions
            bool admitted = false;
            for (auto &sp : slots) {
                Slot &s = *sp;
                if (s.busy || pending.empty()) continue;
                const Request first = pending.front();
                int64_t nq = first.nq;
                int32_t kmax = first.k, npmax = first.nprobe;
                if (!fits(s, batch_bytes(nq, kmax, npmax))) {
                    if (busy > 0) break;   // wait for a batch to finish and give its bytes back
                    pending.pop_front();   // nothing runs and it still does not fit: it never will
                    s.reqs.assign(1, first);
                    finish(s, DADE_ENOMEM);
                    continue;
                }
                pending.pop_front();
                s.reqs.assign(1, first);
                for (auto it = pending.begin(); it != pending.end();) {
                    const bool same = it->alpha == first.alpha && it->delta_d == first.delta_d &&
                                      (mixes(first.delta_d) || (it->k == first.k && it->nprobe == first.nprobe));
                    const int32_t k2 = std::max(kmax, it->k), np2 = std::max(npmax, it->nprobe);
                    if (same && nq + it->nq <= o.max_batch && fits(s, batch_bytes(nq + it->nq, k2, np2))) {
                        nq += it->nq;
                        kmax = k2;
                        npmax = np2;
                        s.reqs.push_back(*it);
                        it = pending.erase(it);
                    } else {
                        ++it;
                    }
                }
                s.ws_bytes = std::max(s.ws_bytes, batch_bytes(nq, kmax, npmax));
                s.busy = true;
                ++busy;
                admitted = true;
                st.batches += 1;
                st.queries += nq;
                lk.unlock();
                const dade_status rc = launch(s);
                lk.lock();
                if (rc != DADE_OK) {
                    finish(s, rc);
                    --busy;
                }
                st.max_inflight = std::max<int64_t>(st.max_inflight, busy);
            }
            if (stop && pending.empty() && busy == 0) break;
            if (admitted) continue;
            if (busy > 0) {   // poll the running slots without holding the lock
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                cv_submit.wait(lk, [&] { return stop || !pending.empty(); });
            }
        }
    }
};

namespace {

bool valid_opts(const dade_server_opts &o, std::string *why) {
    if (o.slots < 1 || o.slots > 64) return *why = "slots outside 1..64", false;
    if (o.max_batch < 1 || o.max_batch > (1 << 20)) return *why = "max_batch outside 1..2^20", false;
    if (o.max_k < 1 || o.max_k > DADE_MAX_K) return *why = "max_k outside 1..DADE_MAX_K", false;
    if (o.max_nprobe < 1) return *why = "max_nprobe < 1", false;
    if (o.device_budget < 0) return *why = "device_budget < 0", false;
    if (o.list_chunk != 0 && (o.list_chunk < 64 || o.list_chunk % 64 != 0))
        return *why = "list_chunk must be 0 or a positive multiple of 64", false;
    if (o.tc_min_rows < 0) return *why = "tc_min_rows < 0", false;
    return true;
}

} // namespace

extern "C" {

void dade_server_opts_default(dade_server_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->slots = 4;
    o->max_batch = 1024;
    o->max_k = 100;
    o->max_nprobe = 128;
    o->tile = 256;
    o->schedule = DADE_SCHED_TILE;
}

dade_status dade_server_create(const dade_index *ix, const dade_server_opts *opts, dade_server **out) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(ix != nullptr && opts != nullptr && out != nullptr, "NULL pointer");
    *out = nullptr;
    std::string why;
    if (!valid_opts(*opts, &why)) {
        set_error("invalid argument: " + why);
        return DADE_EINVAL;
    }
    DADE_CHECK_ARG(opts->max_nprobe <= ix->nc, "max_nprobe > n_clusters");
    dade_server *sv = new (std::nothrow) dade_server();
    if (!sv) {
        set_error("host allocation failed");
        return DADE_ENOMEM;
    }
    sv->ix = ix;
    sv->o = *opts;
    cudaGetDevice(&sv->device);
    // device memory per slot: queries in and rotated, probe distances, probe
    // lists, results, tensor-core operand image, and (seeded schedule) the
    // accept buffer of the list-major phase
    // every slot holds its fixed staging buffers (max_batch queries and results); the
    // workspace a slot's batches grow is admitted batch by batch against the budget
    const int64_t B = opts->max_batch, d = ix->d;
    const int64_t fixed = sv->fixed_bytes(), one = sv->batch_bytes(1, opts->max_k, opts->max_nprobe);
    int n = opts->slots;
    if (opts->device_budget > 0)
        n = (int)std::min<int64_t>(n, (opts->device_budget - one) / std::max<int64_t>(fixed, 1));
    if (n < 1) {
        delete sv;
        set_error("device_budget holds no slot (" + std::to_string(fixed + one) + " bytes for one request)");
        return DADE_ENOMEM;
    }
    sv->st.slots = n;
    sv->st.slot_bytes = fixed + sv->batch_bytes(B, opts->max_k, opts->max_nprobe);
    for (int i = 0; i < n; ++i) sv->slots.emplace_back(new (std::nothrow) Slot());
    for (auto &sp : sv->slots) {
        if (!sp) {
            delete sv;
            set_error("host allocation failed");
            return DADE_ENOMEM;
        }
        Slot &s = *sp;
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&s.q_host, sizeof(float) * (size_t)(B * d)) != cudaSuccess ||
            cudaMallocHost(&s.ids_host, sizeof(int64_t) * (size_t)(B * opts->max_k)) != cudaSuccess ||
            cudaMallocHost(&s.dists_host, sizeof(float) * (size_t)(B * opts->max_k)) != cudaSuccess ||
            cudaMallocHost(&s.k_host, sizeof(int32_t) * (size_t)B) != cudaSuccess ||
            cudaMallocHost(&s.np_host, sizeof(int32_t) * (size_t)B) != cudaSuccess) {
            cudaGetLastError();
            delete sv;
            set_error("stream, event or pinned host allocation failed");
            return DADE_ENOMEM;
        }
        dade_status st = s.q_dev.alloc(sizeof(float) * (size_t)(B * d));
        if (st == DADE_OK) st = s.ids_dev.alloc(sizeof(int64_t) * (size_t)(B * opts->max_k));
        if (st == DADE_OK) st = s.dists_dev.alloc(sizeof(float) * (size_t)(B * opts->max_k));
        if (st != DADE_OK) {
            delete sv;
            return st;
        }
    }
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return DADE_OK;
}

dade_status dade_server_submit(dade_server *sv, const float *q, int64_t nq, int32_t k, int32_t nprobe, float alpha,
                               int32_t delta_d, int64_t *ids, float *dists, uint64_t *ticket) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(sv != nullptr && q != nullptr && ids != nullptr && dists != nullptr && ticket != nullptr,
                   "NULL pointer");
    DADE_CHECK_ARG(nq >= 1 && nq <= sv->o.max_batch, "nq outside 1..max_batch");
    DADE_CHECK_ARG(k >= 1 && k <= sv->o.max_k, "k outside 1..max_k");
    DADE_CHECK_ARG(nprobe >= 1 && nprobe <= sv->o.max_nprobe, "nprobe outside 1..max_nprobe");
    dade_search_opts so{};
    so.mode = sv->o.mode;
    so.tile = sv->o.tile;
    so.threads = sv->o.threads;
    so.schedule = sv->o.schedule;
    so.seed_lists = sv->o.seed_lists;
    so.flags = sv->o.flags;
    so.stage_dims = sv->o.stage_dims;
    so.list_chunk = sv->o.list_chunk;
    so.tc_min_rows = sv->o.tc_min_rows;
    // the same checks dade_search makes, before the request is queued
    dade_status vs = dade_scan(sv->ix, nullptr, nullptr, 0, k, nprobe, alpha, delta_d, &so, nullptr, nullptr,
                               nullptr);
    if (vs != DADE_OK) return vs;
    std::lock_guard<std::mutex> g(sv->mu);
    Request r{sv->next_ticket++, q, nq, k, nprobe, delta_d, alpha, ids, dists, Clock::now()};
    sv->tickets.emplace(r.ticket, Ticket{});
    sv->pending.push_back(r);
    *ticket = r.ticket;
    sv->st.requests += 1;
    sv->cv_submit.notify_one();
    return DADE_OK;
}

dade_status dade_server_wait(dade_server *sv, uint64_t ticket, int64_t timeout_ms, double *latency_s) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(sv != nullptr, "NULL pointer");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    DADE_CHECK_ARG(it != sv->tickets.end(), "unknown ticket");
    auto ready = [&] { return sv->tickets[ticket].done; };
    if (timeout_ms < 0) {
        sv->cv_done.wait(lk, ready);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        set_error("the request has not completed yet");
        return DADE_ETIMEOUT;
    }
    const Ticket t = sv->tickets[ticket];
    sv->tickets.erase(ticket);
    if (latency_s) *latency_s = t.latency;
    if (t.status == DADE_ECANCELLED) set_error("the request was cancelled");
    else if (t.status != DADE_OK) set_error("the batch of this request failed on the device");
    return t.status;
}

dade_status dade_server_replay(dade_server *sv, const float *q, int64_t n, const int32_t *k, const int32_t *nprobe,
                               float alpha, int32_t delta_d, const double *arrival_s, int32_t k_stride, int64_t *ids,
                               float *dists, double *latency_s, double *submit_s) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(sv && q && k && nprobe && arrival_s && ids && dists && latency_s, "NULL pointer");
    DADE_CHECK_ARG(n >= 1, "n < 1");
    for (int64_t i = 0; i < n; ++i) {
        DADE_CHECK_ARG(k[i] >= 1 && k[i] <= k_stride, "k[i] outside 1..k_stride");
        DADE_CHECK_ARG(i == 0 || arrival_s[i] >= arrival_s[i - 1], "arrival times must not decrease");
    }
    std::vector<uint64_t> tickets((size_t)n, 0);
    const int64_t d = sv->ix->d;
    const auto t0 = Clock::now();
    dade_status first = DADE_OK;
    for (int64_t i = 0; i < n; ++i) {
        const auto due = t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {
        }
        const dade_status st = dade_server_submit(sv, q + i * d, 1, k[i], nprobe[i], alpha, delta_d,
                                                  ids + i * k_stride, dists + i * k_stride, &tickets[(size_t)i]);
        if (st != DADE_OK && first == DADE_OK) first = st;
    }
    if (submit_s) *submit_s = std::chrono::duration<double>(Clock::now() - t0).count();
    for (int64_t i = 0; i < n; ++i) {
        latency_s[i] = -1.0;
        if (tickets[(size_t)i] == 0) continue;   // refused at submission
        const dade_status st = dade_server_wait(sv, tickets[(size_t)i], -1, &latency_s[i]);
        if (st != DADE_OK && first == DADE_OK) first = st;
    }
    return first;
}

dade_status dade_server_cancel(dade_server *sv, uint64_t ticket) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(sv != nullptr, "NULL pointer");
    std::lock_guard<std::mutex> g(sv->mu);
    auto it = sv->tickets.find(ticket);
    DADE_CHECK_ARG(it != sv->tickets.end() && !it->second.done, "unknown or completed ticket");
    it->second.cancelled = true;
    for (auto p = sv->pending.begin(); p != sv->pending.end(); ++p)
        if (p->ticket == ticket) {   // not admitted yet: it leaves the queue now
            const Clock::time_point t0 = p->t0;
            sv->pending.erase(p);
            it->second.done = true;
            it->second.status = DADE_ECANCELLED;
            it->second.latency = std::chrono::duration<double>(Clock::now() - t0).count();
            sv->st.requests_done += 1;
            sv->cv_done.notify_all();
            break;
        }
    return DADE_OK;
}

dade_status dade_server_stats_get(dade_server *sv, dade_server_stats *out) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(sv != nullptr && out != nullptr, "NULL pointer");
    std::lock_guard<std::mutex> g(sv->mu);
    *out = sv->st;
    return DADE_OK;
}

void dade_server_free(dade_server *sv) { delete sv; }

} // extern "C"
