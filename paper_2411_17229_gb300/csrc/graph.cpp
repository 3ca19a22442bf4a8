// graph.cpp -- a query step captured once into a CUDA graph and replayed.
//
// dade_graph_create runs the step (dade_query on device buffers) once
// uncaptured, so that every workspace, kernel attribute and occupancy figure
// it needs exists, then captures the same step on a private stream and
// instantiates the graph.  dade_graph_launch replays it: the rotation, the
// probe (tensor-core GEMM and selection), the query ordering and the scan
// kernels, with the shapes and pointers fixed at capture, in one submission.
#include <new>
#include <string>

#include "internal.cuh"

struct dade_graph {
    const dade_index *ix = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~dade_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

bool on_device(const void *p) {
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

} // namespace

extern "C" {

dade_status dade_graph_create(const dade_index *ix, const float *q, int64_t nq, int32_t k, int32_t nprobe, float alpha,
                              int32_t delta_d, const dade_search_opts *opts, int64_t *ids, float *dists,
                              dade_graph **out) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(out != nullptr, "NULL pointer");
    *out = nullptr;
    DADE_CHECK_ARG(ix != nullptr && q != nullptr && ids != nullptr && dists != nullptr, "NULL pointer");
    DADE_CHECK_ARG(nq >= 1, "nq < 1");
    DADE_CHECK_ARG(on_device(q) && on_device(ids) && on_device(dists),
                   "a graph step takes device buffers only (host copies are not captured)");
    DADE_CHECK_ARG(!opts || !opts->stats || on_device(opts->stats), "stats must be a device buffer");
    dade_graph *g = new (std::nothrow) dade_graph();
    if (!g) {
        set_error("host allocation failed");
        return DADE_ENOMEM;
    }
    g->ix = ix;
    auto fail = [&](dade_status st) {
        delete g;
        return st;
    };
    if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess) {
        set_error("cudaStreamCreateWithFlags failed");
        return fail(DADE_ECUDA);
    }
    // uncaptured run: workspaces, attributes, occupancy
    dade_status st = dade_query(ix, q, nq, k, nprobe, alpha, delta_d, opts, ids, dists, (dade_stream)g->cap);
    if (st != DADE_OK) return fail(st);
    if (cudaStreamSynchronize(g->cap) != cudaSuccess) {
        set_error("the warm-up step failed");
        return fail(DADE_ECUDA);
    }
    if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        set_error("cudaStreamBeginCapture failed");
        return fail(DADE_ECUDA);
    }
    st = dade_query(ix, q, nq, k, nprobe, alpha, delta_d, opts, ids, dists, (dade_stream)g->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(g->cap, &graph);
    g->graph = graph;
    if (st != DADE_OK) return fail(st);
    if (ce != cudaSuccess || !graph) {
        set_error(std::string("stream capture failed: ") + cudaGetErrorString(ce));
        cudaGetLastError();
        return fail(DADE_ECUDA);
    }
    if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
        set_error("cudaGraphInstantiate failed");
        cudaGetLastError();
        return fail(DADE_ECUDA);
    }
    *out = g;
    return DADE_OK;
}

dade_status dade_graph_launch(dade_graph *g, dade_stream stream) {
    using namespace dade;
    set_error("");
    DADE_CHECK_ARG(g != nullptr && g->exec != nullptr, "graph is NULL");
    DADE_TRY_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return DADE_OK;
}

void dade_graph_free(dade_graph *g) { delete g; }

} // extern "C"
