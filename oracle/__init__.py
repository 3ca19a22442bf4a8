"""FP64 CPU oracle for DADE-IVF and HNSW* -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and it
never calls the CUDA library; the two share only the seeded input generators.

Thin ctypes wrapper over ``dade_oracle.c`` (plain C, double precision).  Each
wrapper names the passage of the paper it follows; the C file holds the
arithmetic.  ``build()`` compiles the shared object with gcc in-tree.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "dade_oracle.c")
LIB = os.path.join(_HERE, "_build", "liboracle.so")

SEQUENTIAL, TILE, PROBE_ROUNDS, ROW_ROUNDS = 0, 1, 2, 3
HNSW_SEQUENTIAL, HNSW_NODE = 0, 1   # beam-search threshold schedules (or_hnsw_search)
TIE_TOL = 1e-5
# Relative width of the decision bracket of ``search_bracket``: decisions of
# the FP32 path whose two sides lie within this of each other may go either
# way (the FP32 partial distances and thresholds carry relative errors of a
# few 1e-6 on these workloads; the bracket covers them with a margin).
BRACKET_TOL = 2e-5


def build(src: str = SRC, out: str = LIB, extra: tuple = ()) -> str:
    """Compile the oracle with gcc (OpenMP across independent outputs only)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    # contraction off: no fused multiply-add merges a product into a sum (the FP32
    # DCO of the beam search rounds every step, as the paper's scalar code does)
    cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", *extra, "-o", out, src,
           "-lm"]
    subprocess.run(cmd, check=True)
    return out


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Oracle:
    """Bound instance of one compiled oracle library."""

    def __init__(self, path: str | None = None):
        path = path or LIB
        if not os.path.exists(path) or (path == LIB and os.path.getmtime(path) < os.path.getmtime(SRC)):
            build(out=path)
        self.lib = C.CDLL(path)
        L = self.lib
        vp, i64, i32, f64 = C.c_void_p, C.c_int64, C.c_int, C.c_double
        sig = {
            "or_set_threads": (None, [i32]),
            "or_get_threads": (i32, []),
            "or_mean_cov": (None, [vp, i64, i32, vp, vp]),
            "or_jacobi_eig": (i32, [vp, i32, vp, vp]),
            "or_pca": (i32, [vp, i64, i32, vp, vp, vp]),
            "or_rotate": (None, [vp, i64, i32, vp, vp, vp]),
            "or_kmeans": (None, [vp, i64, i32, i32, vp, i32, vp, vp, vp, vp]),
            "or_assign": (f64, [vp, i64, i32, vp, i32, vp]),
            "or_list_means": (None, [vp, i64, i32, vp, i32, vp]),
            "or_probe": (None, [vp, i64, i32, vp, i32, i32, vp, vp, f64]),
            "or_eps_sample": (i64, [vp, i64, i32, vp, vp, i64, vp, i32, vp]),
            "or_eps_quantile": (f64, [vp, i64, f64]),
            "or_search": (i32, [vp, i64, i32, vp, i32, vp, vp, vp, i64, i32, i32, i32, vp, i32, i32, i32,
                                i32, f64, f64, vp, vp, vp, vp]),
            "or_exact_knn": (None, [vp, i64, i32, vp, i64, i32, vp, vp]),
            "or_estimate_sq": (f64, [vp, vp, i32, i32, vp]),
            "or_dco": (i32, [vp, vp, i32, i32, f64, vp, vp, i32, f64, vp, vp, vp]),
            "or_hnsw_graph": (i32, [vp, i64, i32, i32, i32, i32, vp, vp, vp]),
            "or_hnsw_search": (i32, [vp, vp, i64, i32, vp, i32, vp, vp, vp, i64, vp, i32, i32, i32, i32, vp, vp,
                                     i32, i64, f64, f64, vp, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args

    # -- threads ---------------------------------------------------------
    def set_threads(self, t: int):
        self.lib.or_set_threads(int(t))

    def threads(self) -> int:
        return int(self.lib.or_get_threads())

    # -- Section 3.2: PCA (Eq. 10-12) -----------------------------------
    def mean_cov(self, X):
        X = np.ascontiguousarray(X, np.float32)
        n, d = X.shape
        mu, Cm = np.empty(d), np.empty((d, d))
        self.lib.or_mean_cov(_p(X), n, d, _p(mu), _p(Cm))
        return mu, Cm

    def jacobi_eig(self, A):
        A = _f64(A).copy()
        d = A.shape[0]
        lam, V = np.empty(d), np.empty((d, d))
        sweeps = self.lib.or_jacobi_eig(_p(A), d, _p(lam), _p(V))
        if sweeps < 0:
            raise RuntimeError("Jacobi did not converge")
        return lam, V

    def pca(self, X):
        """Returns (mu, W, lam): column k of W is w_k, lam descending."""
        X = np.ascontiguousarray(X, np.float32)
        n, d = X.shape
        mu, W, lam = np.empty(d), np.empty((d, d)), np.empty(d)
        if self.lib.or_pca(_p(X), n, d, _p(mu), _p(W), _p(lam)) < 0:
            raise RuntimeError("PCA failed")
        return mu, W, lam

    def rotate(self, X, mu, W):
        """x' = W^T (x - mu) (Lemma 1), FP64 output."""
        X = np.ascontiguousarray(X, np.float32)
        n, d = X.shape
        out = np.empty((n, d))
        self.lib.or_rotate(_p(X), n, d, _p(_f64(mu)), _p(_f64(W)), _p(out))
        return out

    # -- Section 3.4: IVF ------------------------------------------------
    def kmeans(self, Xr, init, iters):
        Xr = _f64(Xr)
        n, d = Xr.shape
        init = np.ascontiguousarray(init, np.int64)
        nc = init.size
        cent, assign = np.empty((nc, d)), np.empty(n, np.int32)
        obj, gap = np.empty(max(iters, 1)), np.empty(1)
        self.lib.or_kmeans(_p(Xr), n, d, nc, _p(init), iters, _p(cent), _p(assign), _p(obj), _p(gap))
        return cent, assign, obj[:iters], float(gap[0])

    def assign(self, Xr, cent):
        Xr, cent = _f64(Xr), _f64(cent)
        a = np.empty(Xr.shape[0], np.int32)
        gap = self.lib.or_assign(_p(Xr), Xr.shape[0], Xr.shape[1], _p(cent), cent.shape[0], _p(a))
        return a, gap

    def list_means(self, Xr, assign, nc):
        Xr = _f64(Xr)
        assign = np.ascontiguousarray(assign, np.int32)
        cent = np.empty((nc, Xr.shape[1]))
        self.lib.or_list_means(_p(Xr), Xr.shape[0], Xr.shape[1], _p(assign), nc, _p(cent))
        return cent

    def probe(self, Qr, cent, nprobe, tol=TIE_TOL):
        Qr, cent = _f64(Qr), _f64(cent)
        nq = Qr.shape[0]
        pr, tie = np.empty((nq, nprobe), np.int32), np.empty(nq, np.int32)
        self.lib.or_probe(_p(Qr), nq, Qr.shape[1], _p(cent), cent.shape[0], nprobe, _p(pr), _p(tie), tol)
        return pr, tie

    # -- Section 3.3: epsilon_d (Eq. 14) ---------------------------------
    def eps_sample(self, Xr, lam, pairs, dlist):
        """Sorted rho_d samples, shape [len(dlist), m_kept]."""
        Xr = _f64(Xr)
        pairs = np.ascontiguousarray(pairs, np.int64).reshape(-1, 2)
        dl = np.ascontiguousarray(dlist, np.int32)
        m = pairs.shape[0]
        rho = np.empty((dl.size, m))
        kept = self.lib.or_eps_sample(_p(Xr), Xr.shape[0], Xr.shape[1], _p(_f64(lam)), _p(pairs), m,
                                      _p(dl), dl.size, _p(rho))
        return rho[:, :kept].copy()

    def eps_quantile(self, rho_sorted_row, alpha):
        row = _f64(rho_sorted_row)
        return float(self.lib.or_eps_quantile(_p(row), row.size, float(alpha)))

    def eps_table(self, rho, dlist, D, alpha):
        """eps indexed by d (length D + 1), filled at the d in dlist."""
        eps = np.full(D + 1, np.nan)
        for t, d in enumerate(dlist):
            eps[d] = self.eps_quantile(rho[t], alpha)
        return eps

    # -- Algorithm 1 inside IVF -------------------------------------------
    def search(self, Xr, assign, cent, lam, Qr, K, nprobe, delta_d, eps, schedule=TILE, tile=128, lag=0,
               tol=TIE_TOL, seed=0, bias=0.0):
        """Returns ids [nq,K] int64, dists [nq,K] (squared), stats [nq,4], flags [nq].
        seed > 0: the seeded schedule (threshold frozen after the first `seed` lists).
        schedule ROW_ROUNDS: epochs of rows [R_e, R_{e+1}) of every probed list, R_1 = tile.
        bias: every decision uses r^2 (1 + bias) (0: the method; see search_bracket)."""
        Xr, cent, Qr = _f64(Xr), _f64(cent), _f64(Qr)
        n, D = Xr.shape
        nq = Qr.shape[0]
        assign = np.ascontiguousarray(assign, np.int32)
        ids, dists = np.empty((nq, K), np.int64), np.empty((nq, K))
        stats, flags = np.empty((nq, 4), np.int64), np.empty(nq, np.int32)
        e = None if eps is None else _f64(eps)
        rc = self.lib.or_search(_p(Xr), n, D, _p(assign), cent.shape[0], _p(cent), _p(_f64(lam)),
                                _p(Qr), nq, K, nprobe, delta_d, _p(e), schedule, tile, lag, seed, tol,
                                float(bias), _p(ids), _p(dists), _p(stats), _p(flags))
        if rc != 0:
            raise ValueError("or_search rejected its arguments")
        return ids, dists, stats, flags

    def search_bracket(self, *args, btol=BRACKET_TOL, **kw):
        """``search`` plus its decision bracket.  The search runs three times:
        as the method (bias 0), with every test and final compare moved a
        relative ``btol`` towards pruning (bias -btol), and towards keeping
        (bias +btol).  The results of a query split at its boundary
        kth / (1 + 2 btol), kth the K-th distance: the prefix below it is
        unique, while the places at the boundary may hold any of the
        candidates whose distances tie with the K-th within the bracket.  A
        query is *stable* when the three runs agree on the prefix: a
        computation that scans the same probe lists and whose decisions err by
        less than ``btol`` returns that prefix, followed by boundary
        candidates.  (Flag 8 marks a near-tie in the probe order; a caller
        that cannot check the other side's probe lists treats it as unstable.)
        Its work counters are stable when the three runs count the same.
        Returns ids, dists, stats, flags, stable, stats_stable, boundary
        (the boundary distance per query; +inf when fewer than K are found)."""
        kw = dict(kw, tol=btol)
        ids, dists, stats, flags = self.search(*args, **kw, bias=0.0)
        lo = self.search(*args, **kw, bias=-btol)
        hi = self.search(*args, **kw, bias=btol)
        boundary = dists[:, -1] / (1.0 + 2.0 * btol)
        # every run's results below the boundary (its own exact distances) are the method's
        stable = np.array([np.array_equal(ids[q][dists[q] < boundary[q]], r[0][q][r[1][q] < boundary[q]])
                           for r in (lo, hi) for q in range(ids.shape[0])]).reshape(2, -1).all(0)
        stats_stable = (stats == lo[2]).all(1) & (stats == hi[2]).all(1)
        return ids, dists, stats, flags, stable, stats_stable, boundary

    def estimate_sq(self, q, o, d, lam):
        """Eq. 13 for one pair from its first d rotated dimensions."""
        q, o = _f64(q), _f64(o)
        return float(self.lib.or_estimate_sq(_p(q), _p(o), q.size, int(d), _p(_f64(lam))))

    def dco(self, q, o, delta_d, r, lam, eps, prune=True, tol=TIE_TOL):
        """Algorithm 1 for one pair: (accept, dist2, dims, tie bits)."""
        q, o = _f64(q), _f64(o)
        d2, dims, tie = C.c_double(), C.c_int(), C.c_int()
        e = _f64(eps) if eps is not None else _f64(np.zeros(q.size + 1))
        acc = self.lib.or_dco(_p(q), _p(o), q.size, int(delta_d), float(r), _p(_f64(lam)), _p(e),
                              int(bool(prune)), tol, C.byref(d2), C.byref(dims), C.byref(tie))
        return bool(acc), d2.value, dims.value, tie.value

    def exact_knn(self, X, Q, K):
        X = np.ascontiguousarray(X, np.float32)
        Q = np.ascontiguousarray(Q, np.float32)
        ids, dists = np.empty((Q.shape[0], K), np.int64), np.empty((Q.shape[0], K))
        self.lib.or_exact_knn(_p(X), X.shape[0], X.shape[1], _p(Q), Q.shape[0], K, _p(ids), _p(dists))
        return ids, dists


    # -- HNSW* (Section 3.4): layer-0 graph and beam search ------------------
    def hnsw_graph(self, Xr, kc, M, M0):
        """Layer-0 graph by the reading of ``or_hnsw_graph``: nbr [n, M0] int32
        (-1 unused), gap_sel [n], gap_fin [n] (smallest relative gaps of the
        decisions that built each node's lists)."""
        Xr = _f64(Xr)
        n, D = Xr.shape
        nbr = np.empty((n, M0), np.int32)
        gs, gf = np.empty(n), np.empty(n)
        if self.lib.or_hnsw_graph(_p(Xr), n, D, int(kc), int(M), int(M0), _p(nbr), _p(gs), _p(gf)) != 0:
            raise ValueError("or_hnsw_graph rejected its arguments")
        return nbr, gs, gf

    def hnsw_search(self, Xr, nbr, lam, Qr, entry, K, ef, delta_d, eps, schedule=HNSW_NODE, max_visits=0,
                    tol=TIE_TOL, bias=0.0, coef32=None):
        """Greedy beam search with DCOs (``or_hnsw_search``).  entry: [n_entry]
        or [nq, n_entry] object ids.  FP64 arithmetic with eps (None:
        FDScanning); with Xr, Qr given as float32 arrays, the FP32 arithmetic
        of the paper's implementation with the FP32 coefficients coef32 (None:
        FDScanning).  Returns ids [nq,K] int64, dists [nq,K] (squared),
        stats [nq,5] (DCOs, dims, accepted, pruned, expansions), flags [nq]."""
        f32 = np.asarray(Xr).dtype == np.float32
        if f32:
            Xr, Qr = np.ascontiguousarray(Xr, np.float32), np.ascontiguousarray(Qr, np.float32)
        else:
            Xr, Qr = _f64(Xr), _f64(Qr)
        n, D = Xr.shape
        nq = Qr.shape[0]
        nbr = np.ascontiguousarray(nbr, np.int32)
        entry = np.asarray(entry, np.int64)
        if entry.ndim < 2:                       # the same entry objects for every query
            entry = np.broadcast_to(entry.reshape(1, -1), (nq, entry.size))
        entry = np.ascontiguousarray(entry)
        ids, dists = np.empty((nq, K), np.int64), np.empty((nq, K))
        stats, flags = np.empty((nq, 5), np.int64), np.empty(nq, np.int32)
        e = None if (eps is None or f32) else _f64(eps)
        c32 = None if (coef32 is None or not f32) else np.ascontiguousarray(coef32, np.float32)
        rc = self.lib.or_hnsw_search(None if f32 else _p(Xr), _p(Xr) if f32 else None, n, D, _p(nbr), nbr.shape[1],
                                     _p(_f64(lam)), None if f32 else _p(Qr), _p(Qr) if f32 else None, nq,
                                     _p(entry), entry.shape[1], int(K), int(ef), int(delta_d), _p(e), _p(c32),
                                     int(schedule), int(max_visits), float(tol), float(bias), _p(ids), _p(dists),
                                     _p(stats), _p(flags))
        if rc != 0:
            raise ValueError("or_hnsw_search rejected its arguments")
        return ids, dists, stats, flags


# flags of hnsw_search that make a query's path depend on rounding: DCO,
# pop-order and eviction near-ties (a search with no such decision within tol
# takes the same path under any computation whose errors stay below tol)
HNSW_PATH_TIES = 1 | 2 | 4 | 8


_default: Oracle | None = None


def get() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def coef_f32(lam, eps, D: int, delta_d: int):
    """The Section 3.3 test in squared form, P_d > c_j r^2: c_j = (1 + eps_d)^2
    Lambda_d / Lambda_D (Eq. 13 moved to the right-hand side) for the j-th
    tested d = (j + 1) delta_d < D, computed in FP64 and rounded to FP32 (the
    coefficients of the FP32 DCO of ``hnsw_search``)."""
    Lam = np.concatenate([[0.0], np.cumsum(np.asarray(lam, np.float64))])
    return np.array([(1.0 + eps[d]) ** 2 * Lam[d] / Lam[D] for d in increments(D, delta_d)], np.float32)


def increments(D: int, delta_d: int):
    """The d at which Algorithm 1 tests (d < D): delta_d, 2 delta_d, ..."""
    return [d for d in range(delta_d, D, delta_d)]


class Index:
    """The oracle's own DADE-IVF index: PCA, rotated base, lists, eps sample.

    ``assign`` fixes the inverted lists (list centroids = member means); else
    k-means from the given initial ids runs first, followed by the nearest-
    centroid assignment of every base point."""

    def __init__(self, base, n_clusters=None, init=None, iters=10, pairs=None, assign=None,
                 oracle: Oracle | None = None, eps_step=16):
        o = self.o = oracle or get()
        self.mu, self.W, self.lam = o.pca(base)
        self.Xr = o.rotate(base, self.mu, self.W)
        n, D = self.Xr.shape
        self.D = D
        if assign is not None:
            self.nc = int(n_clusters if n_clusters is not None else int(assign.max()) + 1)
            self.assign = np.ascontiguousarray(assign, np.int32)
            self.cent = o.list_means(self.Xr, self.assign, self.nc)
            self.kmeans_obj, self.kmeans_gap = None, None
        else:
            self.nc = int(init.size)
            cent, _, self.kmeans_obj, self.kmeans_gap = o.kmeans(self.Xr, init, iters)
            self.cent = cent
            self.assign, self.assign_gap = o.assign(self.Xr, cent)
        self.dlist = list(range(eps_step, D, eps_step)) if pairs is not None else []
        self.rho = o.eps_sample(self.Xr, self.lam, pairs, self.dlist) if pairs is not None else None

    def eps(self, alpha, delta_d):
        eps = np.full(self.D + 1, np.nan)
        for d in increments(self.D, delta_d):
            eps[d] = self.o.eps_quantile(self.rho[self.dlist.index(d)], alpha)
        return eps

    def rotate(self, Q):
        return self.o.rotate(Q, self.mu, self.W)

    def search(self, Q, K, nprobe, delta_d, alpha, schedule=TILE, tile=128, prune=True, lag=0, seed=0, bias=0.0):
        Qr = self.rotate(Q)
        eps = self.eps(alpha, delta_d) if prune else None
        return self.o.search(self.Xr, self.assign, self.cent, self.lam, Qr, K, nprobe, delta_d, eps,
                             schedule, tile, lag, seed=seed, bias=bias)

    def search_bracket(self, Q, K, nprobe, delta_d, alpha, schedule=TILE, tile=128, prune=True, lag=0, seed=0,
                       btol=BRACKET_TOL):
        """``search`` with the decision bracket of ``Oracle.search_bracket``."""
        Qr = self.rotate(Q)
        eps = self.eps(alpha, delta_d) if prune else None
        return self.o.search_bracket(self.Xr, self.assign, self.cent, self.lam, Qr, K, nprobe, delta_d, eps,
                                     schedule, tile, lag, seed=seed, btol=btol)


class SampledIndex:
    """The oracle's index for a sample of queries over a full-size base.

    The same steps as ``Index`` with a given list assignment -- PCA over all
    N objects (Section 3.2, Eq. 10-12), list centroids as member means, the
    eps sample of the given pairs (Eq. 14) -- but only the objects a search
    of the sampled queries can reach are rotated: the members of the lists
    those queries probe (Section 3.4) and the sampled pairs' objects.  A list
    centroid is computed as W^T (m - mu) from the list's raw FP64 mean m,
    which is the mean of the rotated members (the rotation is affine); the
    sums use numpy's weighted bincount as a library step.  ``search`` returns ids of
    the full base."""

    def __init__(self, base, assign, n_clusters, pairs, queries, nprobe, oracle: Oracle | None = None,
                 eps_step=16, pca_rows=None):
        o = self.o = oracle or get()
        X = np.ascontiguousarray(base, np.float32)
        n, D = X.shape
        self.D, self.nc = D, int(n_clusters)
        # PCA over all N objects, or (pca_rows) over the first rows only: the rows are
        # independent draws, so they form a random sample of the data (a timing setup
        # that keeps the FP64 covariance affordable at 10M x 768)
        self.mu, self.W, self.lam = o.pca(X if pca_rows is None or pca_rows >= n else X[:pca_rows])
        assign = np.ascontiguousarray(assign, np.int32)
        counts = np.bincount(assign, minlength=self.nc)
        if (counts == 0).any():
            raise ValueError("every list must have members")
        sums = np.empty((self.nc, D))
        for j in range(D):                       # one dimension at a time: no copy of the base
            sums[:, j] = np.bincount(assign, weights=X[:, j], minlength=self.nc)
        means = sums / counts[:, None]
        self.cent = (means - self.mu) @ self.W
        self.Qr = o.rotate(queries, self.mu, self.W)
        self.probe, self.probe_tie = o.probe(self.Qr, self.cent, nprobe)
        lists = np.unique(self.probe)
        self.rows = np.flatnonzero(np.isin(assign, lists))      # ascending ids: list order kept
        self.Xr = o.rotate(X[self.rows], self.mu, self.W)
        self.assign = assign[self.rows]
        pairs = np.ascontiguousarray(pairs, np.int64).reshape(-1, 2)
        prow, pinv = np.unique(pairs.ravel(), return_inverse=True)
        self.dlist = list(range(eps_step, D, eps_step))
        self.rho = o.eps_sample(o.rotate(X[prow], self.mu, self.W), self.lam, pinv.reshape(-1, 2), self.dlist)

    def eps(self, alpha, delta_d):
        eps = np.full(self.D + 1, np.nan)
        for d in increments(self.D, delta_d):
            eps[d] = self.o.eps_quantile(self.rho[self.dlist.index(d)], alpha)
        return eps

    def search(self, K, nprobe, delta_d, alpha, schedule=TILE, tile=128, prune=True, lag=0, seed=0, bias=0.0):
        eps = self.eps(alpha, delta_d) if prune else None
        ids, dists, stats, flags = self.o.search(self.Xr, self.assign, self.cent, self.lam, self.Qr, K, nprobe,
                                                 delta_d, eps, schedule, tile, lag, seed=seed, bias=bias)
        ids = np.where(ids >= 0, self.rows[np.maximum(ids, 0)], -1)
        return ids, dists, stats, flags

    def search_bracket(self, K, nprobe, delta_d, alpha, schedule=TILE, tile=128, prune=True, lag=0, seed=0,
                       btol=BRACKET_TOL):
        """``search`` with the decision bracket of ``Oracle.search_bracket``; ids of the full base."""
        eps = self.eps(alpha, delta_d) if prune else None
        out = self.o.search_bracket(self.Xr, self.assign, self.cent, self.lam, self.Qr, K, nprobe, delta_d, eps,
                                    schedule, tile, lag, seed=seed, btol=btol)
        ids = np.where(out[0] >= 0, self.rows[np.maximum(out[0], 0)], -1)
        return (ids,) + tuple(out[1:])
