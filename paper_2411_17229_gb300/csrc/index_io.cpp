// index_io.cpp -- dade_save_index / dade_load_index: the built index as one
// little-endian binary file (this library's own format; the paper stores no
// index).  Layout: an 8-byte magic, a version word, an endianness probe, the
// scalar description of the index, then every array as (u64 byte count,
// bytes): the host FP64 arrays (mean, basis, eigenvalues, their prefix sums,
// the sorted rho_d sample, list of every vector, list descriptors, k-means
// objectives) and the device arrays (rotated centroids and their squared
// norms, the packed dimension-blocked vectors, slot ids, the optional
// low-precision leading blocks and the optional row-major tail copy); the
// FP32 basis is rebuilt from the FP64 one.  Loading checks every size
// against the scalars and every list descriptor and id against the arrays it
// indexes before anything reaches the device, so a damaged file is refused
// instead of producing out-of-range reads in the kernels.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

namespace dade {
namespace {

constexpr char MAGIC[8] = {'D', 'A', 'D', 'E', 'I', 'X', '0', '1'};
constexpr uint32_t VERSION = 1, ENDIAN = 0x01020304u;

struct Scalars {
    int64_t n, eps_kept, data_floats, slots;
    int32_t d, dp, nb, nc, max_list, lead_format, lead_dims, lead_nb, tail_nb0, tail_w;
};

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

bool put(FILE *f, const void *p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool get(FILE *f, void *p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

bool put_section(FILE *f, const void *p, size_t bytes) {
    const uint64_t b = bytes;
    return put(f, &b, sizeof b) && put(f, p, bytes);
}

template <class T>
bool put_vec(FILE *f, const std::vector<T> &v) { return put_section(f, v.data(), sizeof(T) * v.size()); }

dade_status put_dev(FILE *f, const DevBuf &b, size_t bytes) {
    std::vector<unsigned char> h(bytes);
    if (bytes) DADE_TRY_CUDA(cudaMemcpy(h.data(), b.p, bytes, cudaMemcpyDeviceToHost));
    if (!put_section(f, h.data(), bytes)) {
        set_error("write failed");
        return DADE_EIO;
    }
    return DADE_OK;
}

// Reads one section whose size must be exactly `bytes`; the stored size is
// checked before the destination grows, so a damaged header cannot make the
// loader allocate what the scalars do not promise.
dade_status get_size(FILE *f, size_t bytes, const char *what) {
    uint64_t b = 0;
    if (!get(f, &b, sizeof b)) {
        set_error(std::string("index file truncated before ") + what);
        return DADE_EIO;
    }
    if (b != bytes) {
        set_error(std::string("index file: section ") + what + " has " + std::to_string(b) + " bytes, expected " +
                  std::to_string(bytes));
        return DADE_EINVAL;
    }
    return DADE_OK;
}

template <class T>
dade_status get_vec(FILE *f, std::vector<T> &v, size_t count, const char *what) {
    DADE_TRY(get_size(f, sizeof(T) * count, what));
    v.resize(count);
    if (!get(f, v.data(), sizeof(T) * count)) {
        set_error(std::string("index file truncated in ") + what);
        return DADE_EIO;
    }
    return DADE_OK;
}

dade_status get_dev(FILE *f, DevBuf &b, size_t bytes, const char *what, std::vector<unsigned char> *keep = nullptr) {
    std::vector<unsigned char> h;
    DADE_TRY(get_vec(f, h, bytes, what));
    DADE_TRY(b.alloc(bytes));
    if (bytes) DADE_TRY_CUDA(cudaMemcpy(b.p, h.data(), bytes, cudaMemcpyHostToDevice));
    if (keep) keep->swap(h);
    return DADE_OK;
}

size_t lead_code_bytes(const Scalars &s) {
    return s.lead_format == DADE_LEAD_NONE ? 0
                                           : (size_t)s.slots * s.lead_nb * 16 * (s.lead_format == DADE_LEAD_BF16 ? 2 : 1);
}

} // namespace

dade_status save_index(const dade_index *ix, const char *path) {
    DADE_CHECK_ARG(ix->shard < 0, "a shard (dade_index_subset) is not saved: save the full index and take the "
                                  "shard after loading it");
    File fh;
    fh.f = fopen(path, "wb");
    if (!fh.f) {
        set_error(std::string("cannot open ") + path + " for writing");
        return DADE_EIO;
    }
    FILE *f = fh.f;
    Scalars s{ix->n,        ix->eps_kept,  ix->data_floats, ix->slots,   ix->d,        ix->dp,      ix->nb,
              ix->nc,       ix->max_list,  ix->lead_format, ix->lead_dims, ix->lead_nb, ix->tail_nb0, ix->tail_w};
    bool ok = put(f, MAGIC, sizeof MAGIC) && put(f, &VERSION, 4) && put(f, &ENDIAN, 4) && put(f, &s, sizeof s) &&
              put_vec(f, ix->mu) && put_vec(f, ix->W) && put_vec(f, ix->lam) && put_vec(f, ix->Lam) &&
              put_vec(f, ix->rho) && put_vec(f, ix->assign) && put_vec(f, ix->lists) && put_vec(f, ix->kmeans_obj);
    if (!ok) {
        set_error("write failed");
        return DADE_EIO;
    }
    DADE_TRY(put_dev(f, ix->cent, sizeof(float) * (size_t)s.nc * s.dp));
    DADE_TRY(put_dev(f, ix->cnorm, sizeof(float) * (size_t)s.nc));
    DADE_TRY(put_dev(f, ix->data, sizeof(float) * (size_t)s.data_floats));
    DADE_TRY(put_dev(f, ix->ids, sizeof(int32_t) * (size_t)s.slots));
    if (s.lead_format != DADE_LEAD_NONE) {
        DADE_TRY(put_dev(f, ix->lead, lead_code_bytes(s)));
        DADE_TRY(put_dev(f, ix->lead_err, sizeof(float) * (size_t)s.slots * s.lead_nb));
        DADE_TRY(put_dev(f, ix->lead_scale, sizeof(float) * (size_t)s.nc * s.lead_nb));
    }
    if (s.tail_nb0 > 0) DADE_TRY(put_dev(f, ix->tail, sizeof(float) * (size_t)s.slots * s.tail_w));
    if (fflush(f) != 0) {
        set_error("write failed");
        return DADE_EIO;
    }
    return DADE_OK;
}

dade_status load_index(const char *path, dade_index *ix) {
    File fh;
    fh.f = fopen(path, "rb");
    if (!fh.f) {
        set_error(std::string("cannot open ") + path);
        return DADE_EIO;
    }
    FILE *f = fh.f;
    char magic[8];
    uint32_t version = 0, endian = 0;
    Scalars s{};
    if (!get(f, magic, 8) || !get(f, &version, 4) || !get(f, &endian, 4) || !get(f, &s, sizeof s)) {
        set_error("index file truncated in its header");
        return DADE_EIO;
    }
    DADE_CHECK_ARG(std::memcmp(magic, MAGIC, 8) == 0, "not a libdade index file");
    DADE_CHECK_ARG(version == VERSION, "unsupported index file version");
    DADE_CHECK_ARG(endian == ENDIAN, "index file written with another byte order");
    DADE_CHECK_ARG(s.d >= 1 && s.d <= DADE_MAX_DIM && s.dp == (s.d + 15) / 16 * 16 && s.nb == s.dp / 16 &&
                       s.n >= 2 && s.n <= 0x7fffffffLL && s.nc >= 1 && s.nc <= s.n && s.eps_kept >= 0 &&
                       s.slots >= 4 && s.slots % 4 == 0 && s.data_floats >= 64 && s.max_list >= 0,
                   "index file header out of range");
    DADE_CHECK_ARG((s.lead_format == DADE_LEAD_NONE && s.lead_dims == 0 && s.lead_nb == 0) ||
                       ((s.lead_format == DADE_LEAD_BF16 || s.lead_format == DADE_LEAD_FP8) && s.lead_dims >= 16 &&
                        s.lead_dims % 16 == 0 && s.lead_dims <= s.dp && s.lead_nb == s.lead_dims / 16),
                   "index file lead description out of range");
    DADE_CHECK_ARG((s.tail_nb0 == 0 && s.tail_w == 0) ||
                       (s.tail_nb0 > 0 && s.tail_nb0 < s.nb && s.tail_w == s.dp - 16 * s.tail_nb0),
                   "index file tail description out of range");
    const size_t d = s.d;
    DADE_TRY(get_vec(f, ix->mu, d, "mean"));
    DADE_TRY(get_vec(f, ix->W, d * d, "basis"));
    DADE_TRY(get_vec(f, ix->lam, d, "eigenvalues"));
    DADE_TRY(get_vec(f, ix->Lam, d + 1, "eigenvalue prefix sums"));
    DADE_TRY(get_vec(f, ix->rho, (size_t)(s.nb - 1) * s.eps_kept, "rho sample"));
    DADE_TRY(get_vec(f, ix->assign, (size_t)s.n, "assignment"));
    DADE_TRY(get_vec(f, ix->lists, (size_t)s.nc, "list descriptors"));
    uint64_t kb = 0;
    if (!get(f, &kb, sizeof kb) || kb % sizeof(double) != 0 || kb > 8000) {
        set_error("index file: bad k-means objective section");
        return DADE_EINVAL;
    }
    ix->kmeans_obj.resize(kb / sizeof(double));
    if (!get(f, ix->kmeans_obj.data(), kb)) {
        set_error("index file truncated in k-means objectives");
        return DADE_EIO;
    }
    // every descriptor must stay inside the arrays the kernels read through it
    int64_t members = 0;
    int32_t mx = 0;
    for (const ListMeta &m : ix->lists) {
        DADE_CHECK_ARG(m.len >= 0 && m.np >= m.len && m.np % 4 == 0 && m.np - m.len < 4 && m.base >= 0 &&
                           m.base % 64 == 0 && m.base + (int64_t)m.np * s.dp <= s.data_floats && m.slot >= 0 &&
                           m.slot % 4 == 0 && m.slot + m.np <= s.slots,
                       "index file: list descriptor out of range");
        members += m.len;
        mx = std::max(mx, m.len);
    }
    DADE_CHECK_ARG(members == s.n && mx == s.max_list, "index file: list sizes do not add up");
    for (int32_t a : ix->assign) DADE_CHECK_ARG(a >= 0 && a < s.nc, "index file: assignment out of range");

    ix->n = s.n;
    ix->d = s.d;
    ix->dp = s.dp;
    ix->nb = s.nb;
    ix->nc = s.nc;
    ix->max_list = s.max_list;
    ix->eps_kept = s.eps_kept;
    ix->data_floats = s.data_floats;
    ix->slots = s.slots;
    DADE_TRY(get_dev(f, ix->cent, sizeof(float) * (size_t)s.nc * s.dp, "centroids"));
    DADE_TRY(get_dev(f, ix->cnorm, sizeof(float) * (size_t)s.nc, "centroid norms"));
    DADE_TRY(get_dev(f, ix->data, sizeof(float) * (size_t)s.data_floats, "packed vectors"));
    std::vector<unsigned char> idb;
    DADE_TRY(get_dev(f, ix->ids, sizeof(int32_t) * (size_t)s.slots, "slot ids", &idb));
    {
        std::vector<int32_t> ids(s.slots);
        std::memcpy(ids.data(), idb.data(), idb.size());
        for (const ListMeta &m : ix->lists)
            for (int i = 0; i < m.np; ++i) {
                const int32_t id = ids[m.slot + i];
                DADE_CHECK_ARG(i < m.len ? (id >= 0 && id < s.n && ix->assign[id] == (int32_t)(&m - ix->lists.data()))
                                         : id == -1,
                               "index file: slot id out of range");
            }
    }
    if (s.lead_format != DADE_LEAD_NONE) {
        ix->lead_format = s.lead_format;
        ix->lead_dims = s.lead_dims;
        ix->lead_nb = s.lead_nb;
        DADE_TRY(get_dev(f, ix->lead, lead_code_bytes(s), "lead codes"));
        DADE_TRY(get_dev(f, ix->lead_err, sizeof(float) * (size_t)s.slots * s.lead_nb, "lead error norms"));
        DADE_TRY(get_dev(f, ix->lead_scale, sizeof(float) * (size_t)s.nc * s.lead_nb, "lead scales"));
    }
    if (s.tail_nb0 > 0) {
        ix->tail_nb0 = s.tail_nb0;
        ix->tail_w = s.tail_w;
        DADE_TRY(get_dev(f, ix->tail, sizeof(float) * (size_t)s.slots * s.tail_w, "row-major tail"));
    }
    DADE_TRY(upload_basis(ix, 0));
    DADE_TRY(prepare_tensor_operands(ix, 0));
    DADE_TRY(make_data_tmap(ix));
    DADE_TRY(ix->meta.alloc(sizeof(ListMeta) * (size_t)s.nc));
    DADE_TRY_CUDA(cudaMemcpy(ix->meta.p, ix->lists.data(), sizeof(ListMeta) * (size_t)s.nc, cudaMemcpyHostToDevice));
    DADE_TRY(ix->errflag.alloc(sizeof(int32_t) * 4));
    DADE_TRY_CUDA(cudaMemset(ix->errflag.p, 0, sizeof(int32_t) * 4));
    return DADE_OK;
}

} // namespace dade
