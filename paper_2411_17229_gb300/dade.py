"""ctypes binding of libdade (include/dade.h): argument marshalling only.

Every function takes torch tensors (CUDA or CPU) or numpy arrays and passes
raw pointers, sizes and the current CUDA stream to the C ABI; all arithmetic
of the path runs in the library's CUDA kernels.  Loading fails loudly when
the library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdade.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, EIO, ECANCELLED = range(8)
MODE_DADE, MODE_FD = 0, 1
SCHED_TILE, SCHED_PIPELINED, SCHED_SEEDED, SCHED_ROUNDS = 0, 1, 2, 3
FLAG_GENERIC_KERNEL, FLAG_LEAD, FLAG_QUERY_ORDER, FLAG_ROW_TAIL, FLAG_SEED_SPLIT = 1, 2, 4, 8, 16
FLAG_TC_PREFILTER = 32
FLAG_CHECK_TIMEOUT = 64
AUTOTUNE_FORCE = 1
LEAD_NONE, LEAD_BF16, LEAD_FP8 = 0, 1, 2
TRANSFORM_PCA, TRANSFORM_RANDOM, TRANSFORM_GIVEN = 0, 1, 2
ESTIMATOR_DADE, ESTIMATOR_ADSAMPLING = 0, 1
PIPE_MAX = 8
(FIELD_MEAN, FIELD_BASIS, FIELD_EIGVAL, FIELD_CENTROIDS, FIELD_ASSIGN, FIELD_ROTATED, FIELD_RHO, FIELD_KMEANS_OBJ,
 FIELD_LEAD_DEQ, FIELD_LEAD_ERR, FIELD_LEAD_SCALE) = range(11)
MAX_DIM, MAX_K = 1024, 256
PROBE_NOALLOC_MAX = 4194304


class DadeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libdade status {status}: {msg}")
        self.status = status


class BuildOpts(C.Structure):
    _fields_ = [("n_clusters", C.c_int32), ("kmeans_iters", C.c_int32), ("seed", C.c_uint64),
                ("eps_pairs", C.c_int64), ("assign", C.c_void_p), ("kmeans_init", C.c_void_p),
                ("pairs", C.c_void_p), ("lead_format", C.c_int32), ("lead_dims", C.c_int32),
                ("tail_from", C.c_int32), ("transform", C.c_int32), ("basis", C.c_void_p),
                ("reserved", C.c_int32 * 2)]


class SearchOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("tile", C.c_int32), ("stats", C.c_void_p), ("spec", C.c_int32),
                ("threads", C.c_int32), ("schedule", C.c_int32), ("flags", C.c_int32),
                ("lead_stats", C.c_void_p), ("seed_lists", C.c_int32), ("estimator", C.c_int32),
                ("eps0", C.c_float), ("stage_dims", C.c_int32), ("list_chunk", C.c_int32),
                ("stage_ring", C.c_int32), ("wait_ns", C.c_int64), ("tc_min_rows", C.c_int32)]

class AutotuneOpts(C.Structure):
    _fields_ = [("recall_target", C.c_float), ("n_nprobe", C.c_int32), ("nprobe_ladder", C.c_void_p),
                ("reps", C.c_int32), ("flags", C.c_int32), ("cache_path", C.c_char_p), ("reserved", C.c_int32 * 4)]


class AutotuneResult(C.Structure):
    _fields_ = [("nprobe", C.c_int32), ("delta_d", C.c_int32), ("alpha", C.c_float), ("opts", SearchOpts),
                ("recall", C.c_float), ("ms", C.c_float), ("from_cache", C.c_int32), ("points_tried", C.c_int32)]


class ServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("max_batch", C.c_int32), ("max_k", C.c_int32), ("max_nprobe", C.c_int32),
                ("device_budget", C.c_int64), ("mode", C.c_int32), ("tile", C.c_int32), ("threads", C.c_int32),
                ("schedule", C.c_int32), ("seed_lists", C.c_int32), ("flags", C.c_int32),
                ("stage_dims", C.c_int32), ("list_chunk", C.c_int32), ("tc_min_rows", C.c_int32),
                ("reserved", C.c_int32)]


class HnswBuildOpts(C.Structure):
    _fields_ = [("M", C.c_int32), ("M0", C.c_int32), ("kc", C.c_int32), ("nprobe", C.c_int32),
                ("reserved", C.c_int32 * 4)]


class HnswSearchOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("n_entry", C.c_int32), ("entry", C.c_void_p), ("max_visits", C.c_int64),
                ("coef", C.c_void_p), ("stats", C.c_void_p), ("reserved", C.c_int32 * 4)]


class HnswInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("m0", C.c_int32), ("entry", C.c_int64),
                ("device_bytes", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("slots", C.c_int64), ("slot_bytes", C.c_int64), ("requests", C.c_int64),
                ("requests_done", C.c_int64), ("batches", C.c_int64), ("queries", C.c_int64),
                ("max_inflight", C.c_int64)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("d_pad", C.c_int32), ("n_clusters", C.c_int32),
                ("max_list", C.c_int32), ("eps_kept", C.c_int64), ("device_bytes", C.c_int64),
                ("data_bytes", C.c_int64), ("kmeans_iters", C.c_int32), ("lead_format", C.c_int32),
                ("lead_dims", C.c_int32), ("tail_from", C.c_int32)]


# name -> (restype, argtypes); every symbol declared in include/dade.h
_vp, _i64, _i32, _f32 = C.c_void_p, C.c_int64, C.c_int32, C.c_float
SIGNATURES = {
    "dade_build_opts_default": (None, [_vp]),
    "dade_build_index": (_i32, [_vp, _i64, _i32, _vp, _vp, _vp]),
    "dade_free_index": (None, [_vp]),
    "dade_save_index": (_i32, [_vp, C.c_char_p]),
    "dade_graph_create": (_i32, [_vp, _vp, _i64, _i32, _i32, _f32, _i32, _vp, _vp, _vp, _vp]),
    "dade_server_opts_default": (None, [_vp]),
    "dade_server_create": (_i32, [_vp, _vp, _vp]),
    "dade_server_submit": (_i32, [_vp, _vp, _i64, _i32, _i32, _f32, _i32, _vp, _vp, _vp]),
    "dade_server_wait": (_i32, [_vp, C.c_uint64, _i64, _vp]),
    "dade_server_stats_get": (_i32, [_vp, _vp]),
    "dade_server_cancel": (_i32, [_vp, C.c_uint64]),
    "dade_server_replay": (_i32, [_vp, _vp, _i64, _vp, _vp, _f32, _i32, _vp, _i32, _vp, _vp, _vp, _vp]),
    "dade_server_free": (None, [_vp]),
    "dade_hnsw_build_opts_default": (None, [_vp]),
    "dade_hnsw_search_opts_default": (None, [_vp]),
    "dade_hnsw_build": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "dade_hnsw_create": (_i32, [_vp, _vp, _i64, _i32, _vp, _i32, _i64, _vp]),
    "dade_hnsw_search": (_i32, [_vp, _vp, _i64, _i32, _i32, _f32, _i32, _vp, _vp, _vp, _vp]),
    "dade_hnsw_query": (_i32, [_vp, _vp, _i64, _i32, _i32, _f32, _i32, _vp, _vp, _vp, _vp]),
    "dade_hnsw_info_get": (_i32, [_vp, _vp]),
    "dade_hnsw_graph": (_i32, [_vp, _vp]),
    "dade_hnsw_free": (None, [_vp]),
    "dade_graph_launch": (_i32, [_vp, _vp]),
    "dade_graph_free": (None, [_vp]),
    "dade_load_index": (_i32, [C.c_char_p, _vp]),
    "dade_rotate_queries": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "dade_probe": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp]),
    "dade_search": (_i32, [_vp, _vp, _i64, _i32, _i32, _f32, _i32, _vp, _vp, _vp, _vp]),
    "dade_query": (_i32, [_vp, _vp, _i64, _i32, _i32, _f32, _i32, _vp, _vp, _vp, _vp]),
    "dade_scan": (_i32, [_vp, _vp, _vp, _i64, _i32, _i32, _f32, _i32, _vp, _vp, _vp, _vp]),
    "dade_tune": (_i32, [_vp, _vp, _vp, _i64, _i32, _i32, _f32, _i32, _vp, _vp, _vp, _vp]),
    "dade_launch_count": (C.c_uint64, []),
    "dade_reserve": (_i32, [_vp, _i64, _i32]),
    "dade_eps_table": (_i32, [_vp, _f32, _i32, _vp, _vp]),
    "dade_index_info": (_i32, [_vp, _vp]),
    "dade_index_export": (_i32, [_vp, _i32, _vp, C.c_size_t]),
    "dade_host_sym_eig": (_i32, [_vp, _i32, _vp, _vp]),
    "dade_sync": (_i32, [_vp, _vp]),
    "dade_probe_noalloc": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp]),
    "dade_fp32_fma_peak": (_i32, [_i32, _vp, _vp]),
    "dade_set_alloc_hook": (None, [_vp, _vp]),
    "dade_shard_lists": (_i32, [_vp, _i32, _i32, _vp]),
    "dade_autotune_opts_default": (None, [_vp]),
    "dade_query_mixed": (_i32, [_vp, _vp, _i64, _vp, _vp, _i32, _i32, C.c_float, _i32, _vp, _vp, _vp, _vp]),
    "dade_autotune": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp]),
    "dade_index_subset": (_i32, [_vp, _vp, _i32, _vp]),
    "dade_merge_shards": (_i32, [_vp, _vp, _i32, _i64, _i32, _vp, _vp, _vp]),
    "dade_last_error": (C.c_char_p, []),
    "dade_version": (C.c_char_p, []),
}

_lib = None


def lib():
    """Load libdade.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdade.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def shard_lists(list_rows, n_shards: int):
    """dade_shard_lists: owner[c] of every list, lists dealt to n_shards shards balanced by rows."""
    rows = np.ascontiguousarray(list_rows, dtype=np.int64)
    owner = np.empty(rows.shape[0], np.int32)
    _check(lib().dade_shard_lists(rows.ctypes.data, int(rows.shape[0]), int(n_shards), owner.ctypes.data))
    return owner


def merge_shards(ids, dists, out_ids, out_dists, stream=None):
    """dade_merge_shards: ids / dists device [G, nq, K] -> the K nearest per query in out_* [nq, K]."""
    g, nq, k = ids.shape
    _check(lib().dade_merge_shards(_ptr(ids), _ptr(dists), int(g), int(nq), int(k), _ptr(out_ids), _ptr(out_dists),
                                   _stream(stream)))
    return out_ids, out_dists


def fp32_fma_peak(iters: int = 4096, stream=None) -> float:
    """Measured FP32 FMA throughput of the current GPU, TFLOP/s (dade_fp32_fma_peak)."""
    out = C.c_double()
    _check(lib().dade_fp32_fma_peak(int(iters), C.byref(out), _stream(stream)))
    return out.value


def _check(status: int):
    if status != OK:
        raise DadeError(status, lib().dade_last_error().decode())


def _ptr(x):
    """Raw pointer of a torch tensor or numpy array (contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _stream(stream=None):
    if stream is not None:
        return stream
    import torch
    if torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return None


class Index:
    """A libdade index resident in device memory."""

    def __init__(self, base, n_clusters: int, kmeans_iters: int = 10, seed: int = 0, eps_pairs: int = 100000,
                 assign=None, kmeans_init=None, pairs=None, lead_format=LEAD_NONE, lead_dims=0, tail_from=0,
                 transform=TRANSFORM_PCA, basis=None, stream=None):
        L = lib()
        o = BuildOpts()
        L.dade_build_opts_default(C.byref(o))
        o.n_clusters, o.kmeans_iters, o.seed, o.eps_pairs = int(n_clusters), int(kmeans_iters), int(seed), int(eps_pairs)
        o.lead_format, o.lead_dims, o.tail_from = int(lead_format), int(lead_dims), int(tail_from)
        o.transform = int(transform)
        keep = []
        if assign is not None:
            a = np.ascontiguousarray(assign, np.int32)
            keep.append(a)
            o.assign = a.ctypes.data
        if kmeans_init is not None:
            a = np.ascontiguousarray(kmeans_init, np.int64)
            keep.append(a)
            o.kmeans_init = a.ctypes.data
        if basis is not None:
            a = np.ascontiguousarray(basis, np.float64)
            keep.append(a)
            o.basis = a.ctypes.data
            o.transform = TRANSFORM_GIVEN
        if pairs is not None:
            a = np.ascontiguousarray(pairs, np.int64).reshape(-1)
            keep.append(a)
            o.pairs = a.ctypes.data
            o.eps_pairs = a.size // 2
        n, d = base.shape
        h = C.c_void_p()
        _check(L.dade_build_index(_ptr(base), n, d, C.byref(o), C.byref(h), _stream(stream)))
        self._h = h
        info = Info()
        _check(L.dade_index_info(h, C.byref(info)))
        self.info = info
        self.n, self.d, self.n_clusters = info.n, info.d, info.n_clusters

    @classmethod
    def load(cls, path):
        """An index read back from a file written by save()."""
        h = C.c_void_p()
        _check(lib().dade_load_index(os.fsencode(path), C.byref(h)))
        self = cls.__new__(cls)
        self._h = h
        info = Info()
        _check(lib().dade_index_info(h, C.byref(info)))
        self.info = info
        self.n, self.d, self.n_clusters = info.n, info.d, info.n_clusters
        return self

    def save(self, path):
        _check(lib().dade_save_index(self._h, os.fsencode(path)))

    def autotune(self, q, k, gt_ids, recall_target=0.95, ladder=None, reps=3, force=False, cache_path=None,
                 stream=None):
        """dade_autotune: the fastest (nprobe, delta_d, alpha, options) whose recall@k on the queries q
        (host or device [nq, d]) against their exact neighbours gt_ids (host [nq, k]) reaches the
        target.  Returns a dict; ``point`` holds the keyword arguments of query()/search()."""
        o = AutotuneOpts()
        lib().dade_autotune_opts_default(C.byref(o))
        o.recall_target, o.reps = float(recall_target), int(reps)
        o.flags = AUTOTUNE_FORCE if force else 0
        lad = None
        if ladder is not None:
            lad = np.ascontiguousarray(ladder, dtype=np.int32)
            o.n_nprobe, o.nprobe_ladder = int(lad.shape[0]), lad.ctypes.data
        if cache_path is not None:
            o.cache_path = os.fsencode(cache_path)
        gt = np.ascontiguousarray(gt_ids, dtype=np.int64)
        assert gt.shape == (q.shape[0], k)
        r = AutotuneResult()
        _check(lib().dade_autotune(self._h, _ptr(q), q.shape[0], int(k), gt.ctypes.data, C.byref(o), C.byref(r),
                                   _stream(stream)))
        so = r.opts
        point = dict(mode=so.mode, tile=so.tile, threads=so.threads, schedule=so.schedule, flags=so.flags,
                     seed_lists=so.seed_lists, list_chunk=so.list_chunk, tc_min_rows=so.tc_min_rows)
        return {"nprobe": r.nprobe, "delta_d": r.delta_d, "alpha": r.alpha, "point": point, "recall": r.recall,
                "ms": r.ms, "from_cache": bool(r.from_cache), "points_tried": r.points_tried}

    def list_sizes(self):
        """Rows of every inverted list (from the exported assignment)."""
        return np.bincount(self.export(FIELD_ASSIGN), minlength=self.n_clusters).astype(np.int64)

    def subset(self, owner, shard):
        """dade_index_subset: a new index holding the lists c with owner[c] == shard (the rest empty)."""
        own = np.ascontiguousarray(owner, dtype=np.int32)
        assert own.shape[0] == self.n_clusters
        h = C.c_void_p()
        _check(lib().dade_index_subset(self._h, own.ctypes.data, int(shard), C.byref(h)))
        sub = Index.__new__(Index)
        sub._h = h
        info = Info()
        _check(lib().dade_index_info(h, C.byref(info)))
        sub.info = info
        sub.n, sub.d, sub.n_clusters = info.n, info.d, info.n_clusters
        return sub

    def close(self):
        if getattr(self, "_h", None):
            lib().dade_free_index(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    @property
    def handle(self):
        return self._h

    # -- query path ---------------------------------------------------------
    def rotate(self, q, out, stream=None):
        _check(lib().dade_rotate_queries(self._h, _ptr(q), q.shape[0], _ptr(out), _stream(stream)))
        return out

    def probe(self, q_rot, nprobe, out, stream=None):
        _check(lib().dade_probe(self._h, _ptr(q_rot), q_rot.shape[0], int(nprobe), _ptr(out), _stream(stream)))
        return out

    def search(self, q_rot, k, nprobe, alpha, delta_d, ids, dists, mode=MODE_DADE, tile=0, stats=None, spec=0,
               threads=0, schedule=SCHED_TILE, flags=0, lead_stats=None, seed_lists=0, estimator=ESTIMATOR_DADE,
             eps0=0.0, stage_dims=0, list_chunk=0, stage_ring=0, wait_ns=0, tc_min_rows=0, stream=None):
        o = SearchOpts(mode=mode, tile=tile, stats=_ptr(stats), spec=spec, threads=threads, schedule=schedule,
                       flags=flags, lead_stats=_ptr(lead_stats), seed_lists=seed_lists, estimator=estimator,
                       eps0=eps0, stage_dims=stage_dims, list_chunk=list_chunk,
                       stage_ring=stage_ring, wait_ns=wait_ns, tc_min_rows=tc_min_rows)
        _check(lib().dade_search(self._h, _ptr(q_rot), q_rot.shape[0], int(k), int(nprobe), float(alpha), int(delta_d),
                                 C.byref(o), _ptr(ids), _ptr(dists), _stream(stream)))
        return ids, dists

    def scan(self, q_rot, probe, k, alpha, delta_d, ids, dists, mode=MODE_DADE, tile=0, stats=None, spec=0,
             threads=0, schedule=SCHED_TILE, flags=0, lead_stats=None, seed_lists=0, estimator=ESTIMATOR_DADE,
             eps0=0.0, stage_dims=0, list_chunk=0, stage_ring=0, wait_ns=0, tc_min_rows=0, stream=None):
        o = SearchOpts(mode=mode, tile=tile, stats=_ptr(stats), spec=spec, threads=threads, schedule=schedule,
                       flags=flags, lead_stats=_ptr(lead_stats), seed_lists=seed_lists, estimator=estimator,
                       eps0=eps0, stage_dims=stage_dims, list_chunk=list_chunk,
                       stage_ring=stage_ring, wait_ns=wait_ns, tc_min_rows=tc_min_rows)
        _check(lib().dade_scan(self._h, _ptr(q_rot), _ptr(probe), q_rot.shape[0], int(k), probe.shape[1],
                               float(alpha), int(delta_d), C.byref(o), _ptr(ids), _ptr(dists), _stream(stream)))
        return ids, dists

    def query(self, q, k, nprobe, alpha, delta_d, ids, dists, mode=MODE_DADE, tile=0, stats=None, spec=0,
              threads=0, schedule=SCHED_TILE, flags=0, lead_stats=None, seed_lists=0, estimator=ESTIMATOR_DADE,
             eps0=0.0, stage_dims=0, list_chunk=0, stage_ring=0, wait_ns=0, tc_min_rows=0, stream=None):
        o = SearchOpts(mode=mode, tile=tile, stats=_ptr(stats), spec=spec, threads=threads, schedule=schedule,
                       flags=flags, lead_stats=_ptr(lead_stats), seed_lists=seed_lists, estimator=estimator,
                       eps0=eps0, stage_dims=stage_dims, list_chunk=list_chunk,
                       stage_ring=stage_ring, wait_ns=wait_ns, tc_min_rows=tc_min_rows)
        _check(lib().dade_query(self._h, _ptr(q), q.shape[0], int(k), int(nprobe), float(alpha), int(delta_d),
                                C.byref(o), _ptr(ids), _ptr(dists), _stream(stream)))
        return ids, dists

    def query_mixed(self, q, k, nprobe, alpha, delta_d, ids, dists, mode=MODE_DADE, tile=0, threads=0, flags=0,
                    stage_dims=0, wait_ns=0, schedule=SCHED_TILE, list_chunk=0, tc_min_rows=0, stream=None):
        """dade_query_mixed: per-query K and nprobe (int32 arrays [nq], host or device); ids / dists
        [nq, max K].  Tile schedule or list-major row rounds."""
        kk = k if hasattr(k, "data_ptr") else np.ascontiguousarray(k, dtype=np.int32)
        pp = nprobe if hasattr(nprobe, "data_ptr") else np.ascontiguousarray(nprobe, dtype=np.int32)
        k_max = int(kk.max().item() if hasattr(kk, "data_ptr") else kk.max())
        np_max = int(pp.max().item() if hasattr(pp, "data_ptr") else pp.max())
        o = SearchOpts(mode=mode, tile=tile, threads=threads, schedule=schedule, flags=flags, stage_dims=stage_dims,
                       wait_ns=wait_ns, list_chunk=list_chunk, tc_min_rows=tc_min_rows)
        _check(lib().dade_query_mixed(self._h, _ptr(q), q.shape[0], _ptr(kk), _ptr(pp), k_max, np_max, float(alpha),
                                      int(delta_d), C.byref(o), _ptr(ids), _ptr(dists), _stream(stream)))
        return ids, dists

    def graph(self, q, k, nprobe, alpha, delta_d, ids, dists, mode=MODE_DADE, tile=0, stats=None, spec=0,
              threads=0, schedule=SCHED_TILE, flags=0, seed_lists=0, estimator=ESTIMATOR_DADE, eps0=0.0,
              stage_dims=0, list_chunk=0, stage_ring=0, wait_ns=0, tc_min_rows=0):
        """A query step captured into a CUDA graph (device buffers, bound to the graph)."""
        return Graph(self, q, k, nprobe, alpha, delta_d, ids, dists,
                     SearchOpts(mode=mode, tile=tile, stats=_ptr(stats), spec=spec, threads=threads,
                                schedule=schedule, flags=flags, seed_lists=seed_lists, estimator=estimator,
                                eps0=eps0, stage_dims=stage_dims, list_chunk=list_chunk,
                                stage_ring=stage_ring, wait_ns=wait_ns, tc_min_rows=tc_min_rows))

    def tune(self, q_rot, probe, k, nprobe, alpha, delta_d, ids, dists, mode=MODE_DADE, tile=0, spec=0,
             threads=0, schedule=SCHED_TILE, flags=0, seed_lists=0, estimator=ESTIMATOR_DADE, eps0=0.0,
             stage_dims=0, list_chunk=0, stage_ring=0, tc_min_rows=0, stream=None):
        """dade_tune: the fastest result-neutral options for this shape, as {"threads", "flags"}."""
        o = SearchOpts(mode=mode, tile=tile, spec=spec, threads=threads, schedule=schedule, flags=flags,
                       seed_lists=seed_lists, estimator=estimator, eps0=eps0, stage_dims=stage_dims,
                       list_chunk=list_chunk, stage_ring=stage_ring, tc_min_rows=tc_min_rows)
        _check(lib().dade_tune(self._h, _ptr(q_rot), _ptr(probe), q_rot.shape[0], int(k), int(nprobe), float(alpha),
                               int(delta_d), C.byref(o), _ptr(ids), _ptr(dists), _stream(stream)))
        return {"threads": o.threads, "flags": o.flags}

    def reserve(self, max_nq, max_nprobe):
        _check(lib().dade_reserve(self._h, int(max_nq), int(max_nprobe)))

    def sync(self, stream=None):
        _check(lib().dade_sync(self._h, _stream(stream)))

    # -- inspection -----------------------------------------------------------
    def eps_table(self, alpha, delta_d):
        eps = np.empty(self.d + 1)
        coef = np.empty(self.d + 1, np.float32)
        _check(lib().dade_eps_table(self._h, float(alpha), int(delta_d), eps.ctypes.data, coef.ctypes.data))
        return eps, coef

    def export(self, field):
        d, n, nc = self.d, self.n, self.n_clusters
        shapes = {FIELD_MEAN: ((d,), np.float64), FIELD_BASIS: ((d, d), np.float64), FIELD_EIGVAL: ((d,), np.float64),
                  FIELD_CENTROIDS: ((nc, d), np.float32), FIELD_ASSIGN: ((n,), np.int32),
                  FIELD_ROTATED: ((n, d), np.float32),
                  FIELD_RHO: ((max(0, self.info.d_pad // 16 - 1), self.info.eps_kept), np.float64)}
        shapes[FIELD_KMEANS_OBJ] = ((self.info.kmeans_iters,), np.float64)
        ld = self.info.lead_dims
        shapes[FIELD_LEAD_DEQ] = ((n, ld), np.float32)
        shapes[FIELD_LEAD_ERR] = ((ld // 16, n), np.float32)
        shapes[FIELD_LEAD_SCALE] = ((nc, ld // 16), np.float32)
        shape, dt = shapes[field]
        out = np.empty(shape, dt)
        _check(lib().dade_index_export(self._h, field, out.ctypes.data, out.nbytes))
        return out


def schedule_lag(d: int, delta_d: int, schedule: int = SCHED_TILE) -> int:
    """Tiles of threshold lag of a DADE search (see dade_schedule)."""
    nb = (d + 15) // 16
    gb = min(delta_d // 16, nb)
    n_inc = (nb + gb - 1) // gb
    return n_inc - 1 if schedule == SCHED_PIPELINED and n_inc <= PIPE_MAX else 0


def host_sym_eig(a):
    a = np.array(a, np.float64, order="C")
    n = a.shape[0]
    w, v = np.empty(n), np.empty((n, n))
    _check(lib().dade_host_sym_eig(a.ctypes.data, n, w.ctypes.data, v.ctypes.data))
    return w, v


class Graph:
    """A captured query step of an Index (see dade_graph_create)."""

    def __init__(self, index, q, k, nprobe, alpha, delta_d, ids, dists, opts):
        self._index, self._keep = index, (q, ids, dists, opts)
        h = C.c_void_p()
        _check(lib().dade_graph_create(index.handle, _ptr(q), q.shape[0], int(k), int(nprobe), float(alpha),
                                       int(delta_d), C.byref(opts), _ptr(ids), _ptr(dists), C.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib().dade_graph_launch(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().dade_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class Hnsw:
    """HNSW* (dade_hnsw_*): a layer-0 graph over rotated vectors, searched by
    a greedy beam search with one DADE DCO per neighbour."""

    def __init__(self, handle, index=None):
        self._h, self._index = handle, index
        info = HnswInfo()
        _check(lib().dade_hnsw_info_get(self._h, C.byref(info)))
        self.n, self.d, self.m0, self.entry = int(info.n), int(info.d), int(info.m0), int(info.entry)
        self.device_bytes = int(info.device_bytes)

    @classmethod
    def build(cls, index, base, M=16, M0=32, kc=64, nprobe=0):
        """Graph over the index's own vectors (base: those vectors, host or device [n, d])."""
        o = HnswBuildOpts()
        lib().dade_hnsw_build_opts_default(C.byref(o))
        o.M, o.M0, o.kc, o.nprobe = int(M), int(M0), int(kc), int(nprobe)
        h = C.c_void_p()
        _check(lib().dade_hnsw_build(index.handle, _ptr(base), int(base.shape[0]), C.byref(o), C.byref(h)))
        return cls(h, index)

    @classmethod
    def create(cls, x_rot, nbr, entry, index=None):
        """From given rotated vectors [n, d] float32 and links [n, m0] int32 (host or device)."""
        h = C.c_void_p()
        _check(lib().dade_hnsw_create(index.handle if index is not None else None, _ptr(x_rot), int(x_rot.shape[0]),
                                      int(x_rot.shape[1]), _ptr(nbr), int(nbr.shape[1]), int(entry), C.byref(h)))
        return cls(h, index)

    def _opts(self, mode, entry, max_visits, coef, stats):
        o = HnswSearchOpts()
        lib().dade_hnsw_search_opts_default(C.byref(o))
        o.mode, o.max_visits = int(mode), int(max_visits)
        keep = []
        if entry is not None:
            if not hasattr(entry, "data_ptr"):
                entry = np.ascontiguousarray(entry, np.int64)
                keep.append(entry)
            o.entry, o.n_entry = _ptr(entry), int(entry.shape[1])
        if coef is not None:
            c = np.ascontiguousarray(coef, np.float32)
            keep.append(c)
            o.coef = c.ctypes.data
        o.stats = _ptr(stats)
        return o, keep

    def search(self, q_rot, k, ef, alpha, delta_d, ids, dists, mode=MODE_DADE, entry=None, max_visits=0,
               coef=None, stats=None, stream=None):
        """dade_hnsw_search on rotated queries [nq, d]; ids [nq, k] int64, dists [nq, k] float32;
        entry [nq, n_entry] int64; coef: FP32 c_j (None: the index's at alpha); stats [nq, 5] int64."""
        o, keep = self._opts(mode, entry, max_visits, coef, stats)
        _check(lib().dade_hnsw_search(self._h, _ptr(q_rot), int(q_rot.shape[0]), int(k), int(ef), float(alpha),
                                      int(delta_d), C.byref(o), _ptr(ids), _ptr(dists), _stream(stream)))
        del keep
        return ids, dists

    def query(self, q, k, ef, alpha, delta_d, ids, dists, mode=MODE_DADE, entry=None, max_visits=0, coef=None,
              stats=None, stream=None):
        """dade_hnsw_query on raw queries [nq, d] (rotated with the structure's index)."""
        o, keep = self._opts(mode, entry, max_visits, coef, stats)
        _check(lib().dade_hnsw_query(self._h, _ptr(q), int(q.shape[0]), int(k), int(ef), float(alpha), int(delta_d),
                                     C.byref(o), _ptr(ids), _ptr(dists), _stream(stream)))
        del keep
        return ids, dists

    def graph(self):
        nbr = np.empty((self.n, self.m0), np.int32)
        _check(lib().dade_hnsw_graph(self._h, nbr.ctypes.data))
        return nbr

    def close(self):
        if getattr(self, "_h", None):
            lib().dade_hnsw_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class Server:
    """Continuous-batching request server over an Index (see dade_server_create)."""

    def __init__(self, index, **opts):
        o = ServerOpts()
        lib().dade_server_opts_default(C.byref(o))
        for k, v in opts.items():
            setattr(o, k, v)
        h = C.c_void_p()
        _check(lib().dade_server_create(index.handle, C.byref(o), C.byref(h)))
        self._index, self._h, self.d = index, h, index.d
        self._live = {}

    def submit(self, q, k, nprobe, alpha=0.1, delta_d=32):
        """Queue host queries q [nq, d]; returns a ticket.  result(ticket) gives (ids, dists, latency)."""
        q = np.ascontiguousarray(q, np.float32)
        ids = np.empty((q.shape[0], k), np.int64)
        dists = np.empty((q.shape[0], k), np.float32)
        t = C.c_uint64()
        _check(lib().dade_server_submit(self._h, q.ctypes.data, q.shape[0], int(k), int(nprobe), float(alpha),
                                        int(delta_d), ids.ctypes.data, dists.ctypes.data, C.byref(t)))
        self._live[t.value] = (q, ids, dists)
        return t.value

    def result(self, ticket, timeout_ms=-1):
        lat = C.c_double()
        rc = lib().dade_server_wait(self._h, C.c_uint64(ticket), int(timeout_ms), C.byref(lat))
        if rc not in (OK, ETIMEOUT):   # the ticket is settled: its buffers are the caller's again
            self._live.pop(ticket, None)
        _check(rc)
        q, ids, dists = self._live.pop(ticket)
        return ids, dists, lat.value

    def replay(self, q, k, nprobe, alpha, delta_d, arrival_s):
        """dade_server_replay: one-query requests q [n, d] submitted natively at arrival_s [n] seconds;
        returns ids, dists [n, max k] (row i: its k[i] results), latencies [n] and the submit time."""
        q = np.ascontiguousarray(q, np.float32)
        k = np.ascontiguousarray(k, np.int32)
        nprobe = np.ascontiguousarray(nprobe, np.int32)
        arr = np.ascontiguousarray(arrival_s, np.float64)
        n, ks = q.shape[0], int(k.max())
        ids = np.empty((n, ks), np.int64)
        dists = np.empty((n, ks), np.float32)
        lat = np.empty(n, np.float64)
        sub = C.c_double()
        _check(lib().dade_server_replay(self._h, q.ctypes.data, n, k.ctypes.data, nprobe.ctypes.data, float(alpha),
                                        int(delta_d), arr.ctypes.data, ks, ids.ctypes.data, dists.ctypes.data,
                                        lat.ctypes.data, C.byref(sub)))
        return ids, dists, lat, sub.value

    def cancel(self, ticket):
        """dade_server_cancel: result(ticket) then raises DadeError with status ECANCELLED."""
        _check(lib().dade_server_cancel(self._h, C.c_uint64(ticket)))

    def stats(self):
        st = ServerStats()
        _check(lib().dade_server_stats_get(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().dade_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass
