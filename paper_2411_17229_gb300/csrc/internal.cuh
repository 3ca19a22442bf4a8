// internal.cuh -- shared declarations of libdade (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dade.h"

namespace dade {

// ---------------------------------------------------------------- errors ----
void set_error(const std::string &msg);

#define DADE_TRY_CUDA(expr)                                                              \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess) {                                                         \
            ::dade::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));       \
            return DADE_ECUDA;                                                           \
        }                                                                                \
    } while (0)

#define DADE_TRY(expr)                                                                   \
    do {                                                                                 \
        dade_status _s = (expr);                                                         \
        if (_s != DADE_OK) return _s;                                                    \
    } while (0)

#define DADE_CHECK_ARG(cond, msg)                                                        \
    do {                                                                                 \
        if (!(cond)) {                                                                   \
            ::dade::set_error(std::string("invalid argument: ") + (msg));                \
            return DADE_EINVAL;                                                          \
        }                                                                                \
    } while (0)

dade_status launch_check(const char *what);   // after every kernel launch: error check and launch count
unsigned long long launch_count();

// Let kernel `func` use `smem` bytes of dynamic shared memory on the current
// device.  The attribute is set once per (kernel, device) and size, under a
// lock, so any host thread may launch on any device.
dade_status kernel_smem(const void *func, size_t smem);
// Thread blocks of `func` (threads, smem) resident on the whole current
// device at once (SMs x blocks per SM, at least 1), cached per (kernel, device).
dade_status resident_blocks(const void *func, int threads, size_t smem, int *blocks);

// ----------------------------------------------------------- list layout ----
// Per inverted list: offset of its region in the packed data (in floats,
// 256-byte aligned), offset of its first slot in the id array, member count
// and padded count (a multiple of 4).  Block b of the list is the slab
// data[base + b * np * 16 ... + np * 16), candidate i at + i * 16.
struct ListMeta {
    int64_t base;
    int64_t slot;
    int32_t len;
    int32_t np;
};

// Device allocation that frees itself.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    dade_status alloc(size_t b);          // exact size, contents undefined
    dade_status ensure(size_t b);         // grow-only
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Device workspace of a query call (grown on demand, reused across calls).
// An index owns one; a server slot owns its own so that calls on different
// streams never share scratch memory.
struct Workspace {
    DevBuf dist, probe, qrot, qin, ids, dists, order, ordcnt, aimg, anorm, selflag;
    DevBuf lm_cnt, lm_items, lm_acc, lm_acnt;   // seeded schedule (lm.cu)
    DevBuf qk, qnp;                              // per-query K and nprobe (dade_query_mixed)
};

} // namespace dade

struct dade_index {
    int64_t n = 0;
    int32_t d = 0, dp = 0, nb = 0, nc = 0, max_list = 0;
    // host copies (FP64 from the offline steps)
    std::vector<double> mu, W, lam, Lam;    // Lam[d] = lambda_1 + ... + lambda_d, Lam[0] = 0
    std::vector<double> rho;                // [(nb - 1) rows][eps_kept], each row sorted
    int64_t eps_kept = 0;
    std::vector<int32_t> assign;            // [n]
    std::vector<dade::ListMeta> lists;      // [nc]
    std::vector<double> kmeans_obj;
    // device
    dade::DevBuf WT32;      // float [dp][dp]: W^T, row k = w_k (zero padded); x'_k = <w_k, x - mu>
    dade::DevBuf cent_img, wt_img;   // centroids and W^T split into TF32 hi/lo tiles (tc_gemm.cu)
    dade::DevBuf mu32;      // float [d]
    dade::DevBuf cent;      // float [nc][dp] rotated centroids (zero padded)
    dade::DevBuf cnorm;     // float [nc] squared norms of the centroids
    dade::DevBuf data;      // packed rotated vectors
    dade::DevBuf ids;       // int32 per slot (padding slots -1)
    dade::DevBuf meta;      // ListMeta [nc]
    dade::DevBuf errflag;   // int32 [4]: [0] device error word (bounded waits); [3] stays 0
                            // (the word the failure-path check waits on)
    // low-precision copy of the leading dims (prefilter), see dade_lead_format
    int32_t lead_format = 0, lead_dims = 0, lead_nb = 0;
    dade::DevBuf lead;      // codes; list c at slot_c * lead_nb * 16 * ES bytes, block b at + b * np * 16 * ES
    dade::DevBuf lead_scale;// float [nc][lead_nb] (FP8 only)
    dade::DevBuf lead_err;  // float [lead_nb][slots]: error norm over blocks 0..b (rounded up)
    // TMA view of the packed FP32 data as rows of 16 floats (64 B): row base_c / 16 + b np_c + i holds
    // block b of member i of list c; boxes of 4 floats x 128 rows (the tensor-core prefilter, lm.cu)
    CUtensorMap data_tmap{};
    bool data_tmap_ok = false;
    // row-major copy of dims [16 tail_nb0, dp) of every slot: tail[(slot) * tail_w + k - 16 tail_nb0]
    int32_t tail_nb0 = 0, tail_w = 0;
    dade::DevBuf tail;
    int64_t data_floats = 0, slots = 0;
    int32_t shard = -1;     // dade_index_subset: the shard this index holds (-1: every list)
    // workspace (grown on demand, reused across calls)
    mutable dade::Workspace ws0;   // used unless a WorkspaceScope is active on the calling thread
};

namespace dade {

// The workspace of the calling thread's current call: the one a
// WorkspaceScope installed, else the index's own.
Workspace &ws(const dade_index *ix);
struct WorkspaceScope {
    explicit WorkspaceScope(Workspace *w);
    ~WorkspaceScope();
    Workspace *prev;
};

// Kernel launchers (each returns DADE_OK or DADE_ECUDA after checking the launch).
// Tensor-core GEMMs (tc_gemm.cu).  x' = W^T (x - mu) for n rows of x (row
// stride d): out[i * out_stride + k] for k < min(out_stride, dp); rotate()
// uses the index's workspace, rotate_direct() none (build time).
dade_status rotate(const dade_index *ix, const float *x, int64_t n, int32_t out_stride, float *out, cudaStream_t s);
dade_status rotate_direct(const dade_index *ix, const float *x, int64_t n, int32_t out_stride, float *out,
                          cudaStream_t s);
// dist[i * nc + j] = max(0, ||q_i||^2 + ||c_j||^2 - 2 <q_i, c_j>); the
// direct form allocates nothing (dade_probe_noalloc).
dade_status probe_distances(const dade_index *ix, const float *q_rot, int64_t nq, int32_t q_stride, float *dist,
                            cudaStream_t s);
dade_status probe_distances_direct(const dade_index *ix, const float *q_rot, int64_t nq, int32_t q_stride, float *dist,
                                   cudaStream_t s);
// Operand images of the centroids and of W^T (after build or load).
dade_status prepare_tensor_operands(dade_index *ix, cudaStream_t s);
dade_status probe(const dade_index *ix, const float *q_rot, int64_t nq, int32_t q_stride,
                  int32_t nprobe, int32_t *probe_out, cudaStream_t s);
dade_status centroid_norms(dade_index *ix, cudaStream_t s);

// Permutation of the queries of a scan that groups them by first probed list
// (order.cu); order[nq] on the device, written on stream s.
dade_status order_queries(const dade_index *ix, const int32_t *probe, int64_t nq, int32_t nprobe, int32_t *order,
                          cudaStream_t s);

struct ScanParams {
    const float *q_rot;      // [nq][q_stride]
    int32_t q_stride;
    const int32_t *probe;    // [nq][nprobe]
    int32_t nprobe, k, tile, mode, delta_d, n_inc, spec, threads, schedule, generic, use_lead;
    int64_t *lead_stats;     // [nq] or null
    const int32_t *order;    // [nq] execution order of the queries, or null (identity)
    int32_t use_tail;        // phase B reads the row-major tail copy
    int32_t pstride;         // row stride of probe (0: nprobe)
    int32_t seed_lists;      // DADE_SCHED_SEEDED
    int32_t stage_dims;      // FP32 DADE tile kernel: dims staged per tile (0: delta_d)
    int32_t seed_split;      // SEEDED: lists after the seeds run query-major, split over CTAs
    int32_t list_chunk;      // list-major passes: rows of a list per work item (0: 4096)
    int32_t stage_ring;      // tile kernel: staged units in flight per CTA (0: 2)
    // split mode of the tile kernel (parts > 0; see ScanArgs)
    int32_t parts, c0;
    int32_t row_lo, row_hi;  // split passes: rows [row_lo, min(len, row_hi)) of every list (row_hi 0: all)
    int32_t use_tc;          // list-major passes: the first increment's tensor-core prefilter
    int64_t wait_ns;         // limit of the scan kernels' bounded waits (0: 2 s)
    int32_t tc_min_rows;     // row rounds: the tensor-core prefilter only for windows this long
    int32_t check_timeout;   // failure-path check: every block's first wait runs out
    const int32_t *q_k = nullptr, *q_np = nullptr;   // per-query K and nprobe (tile schedule), or NULL
    const float *r2src;
    unsigned long long *acc;
    int *acnt;
    int64_t cap;
    float coef[DADE_MAX_DIM / DADE_BLOCK];   // per increment; prune iff P > coef[j] * r2
    int64_t *ids;            // [nq][k]
    float *dists;            // [nq][k]
    int64_t *stats;          // [nq][4] or null
};
dade_status scan(const dade_index *ix, int64_t nq, const ScanParams &p, cudaStream_t s);
// DADE_SCHED_SEEDED with 0 < p.seed_lists < p.nprobe (lm.cu).
dade_status scan_seeded(const dade_index *ix, int64_t nq, const ScanParams &p, cudaStream_t s);
// DADE_SCHED_ROUNDS (lm.cu).
dade_status scan_rounds(const dade_index *ix, int64_t nq, const ScanParams &p, cudaStream_t s);
// The TMA view of the packed FP32 data (after build or load).
dade_status make_data_tmap(dade_index *ix);

// FP32 basis W^T and mean on the device, from the host FP64 copies (build.cu).
dade_status upload_basis(dade_index *ix, cudaStream_t s);

// Drop the tuning choices cached for an index (tune.cpp).
void tune_forget(const dade_index *ix);

// Index file (index_io.cpp).
dade_status save_index(const dade_index *ix, const char *path);
dade_status load_index(const char *path, dade_index *ix);

// Host FP64 symmetric eigensolver (descending eigenvalues, column eigenvectors).
bool sym_eig(int n, std::vector<double> &a, std::vector<double> &w, std::vector<double> &v);

// Pruning coefficients of one (alpha, delta_d) for the DADE estimator, or of
// eps0 (>= 0 selects ADSampling); returns the number of increments.
int coef_table(const dade_index *ix, float alpha, int32_t delta_d, double *eps, float *coef, float eps0 = -1.f);

} // namespace dade
