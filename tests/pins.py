"""Pins of the FP64 oracle to facts fixed outside it.

Every pin takes an ``Oracle`` instance so the same checks can be run against
builds of the oracle with a deliberately planted mistake (see
test_oracle_plants.py).  Each pin cites the passage of the paper it checks and
compares against something other than the oracle itself: a closed form, a
hand-worked value under tests/golden/, a library routine on a special case,
brute force on tiny inputs, or a statistical property with its error bar.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from paper_2411_17229_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(1e-300, float(np.max(np.abs(b)))))


# --------------------------------------------------------------------------
# Section 3.2: PCA (Eq. 10-12), Lemma 1, Lemma 2, Lemma 4
# --------------------------------------------------------------------------

def pin_eigen_closed_form(o):
    """Eq. 11: eigenpairs of matrices with closed-form spectra."""
    g = golden("eigen_closed_form.json")
    for case in g["cases"]:
        A = np.array(case["A"], float)
        lam, V = o.jacobi_eig(A)
        assert _rel(lam, case["lam"]) < 1e-12, (lam, case["lam"])
        assert np.all(np.diff(lam) <= 0), "eigenvalues must be descending (Eq. 11)"
        assert np.allclose(A @ V, V * lam[None, :], atol=1e-12)
        assert np.allclose(V.T @ V, np.eye(A.shape[0]), atol=1e-12)


def pin_pca_cross(o):
    """Eq. 10-12 with Lemma 1's centring on a hand-derived point set."""
    g = golden("pca_cross.json")
    X = np.array(g["X"], np.float32)
    mu, W, lam = o.pca(X)
    # the inputs are FP32-rounded, so the closed form holds to ~1e-6
    assert np.allclose(mu, g["mu"], atol=1e-5)
    assert np.allclose(lam, g["lam"], rtol=1e-5)
    assert abs(abs(float(W[:, 0] @ np.array(g["w1"]))) - 1.0) < 1e-6


def pin_pca_vs_library(o):
    """Mean/covariance vs numpy, spectrum vs LAPACK eigh, Lemma 2 trace."""
    X, _, _ = synth.gaussian(3000, 24, 1.0, seed=11, basis_seed=12)
    X = X + np.float32(3.0)
    mu, Cm = o.mean_cov(X)
    Xd = X.astype(np.float64)
    assert _rel(mu, Xd.mean(0)) < 1e-12
    assert _rel(Cm, np.cov(Xd.T, bias=True)) < 1e-11
    mu2, W, lam = o.pca(X)
    ref = np.sort(np.linalg.eigvalsh(np.cov(Xd.T, bias=True)))[::-1]
    assert _rel(lam, ref) < 1e-10
    assert np.all(np.diff(lam) < 0)
    assert np.allclose(W.T @ W, np.eye(24), atol=1e-12)
    assert np.allclose(Cm @ W, W * lam[None, :], atol=1e-10 * lam[0])
    # Lemma 2: an orthogonal transform keeps the sum of variances
    assert abs(np.trace(Cm) - lam.sum()) < 1e-12 * lam.sum()


def pin_ky_fan(o):
    """Eq. 10 / Lemma 4: the PCA basis maximises sigma^2(1, d) for every d,
    so any other orthogonal basis has a smaller or equal prefix variance."""
    X, _, _ = synth.gaussian(4000, 32, 1.2, seed=21, basis_seed=22)
    mu, W, lam = o.pca(X)
    Cm = np.cov(X.astype(np.float64).T, bias=True)
    Lam = np.cumsum(lam)
    for s in range(3):
        R = synth.haar(32, np.random.default_rng(100 + s))
        var = np.einsum("ij,jk,ki->i", R.T, Cm, R)
        assert np.all(np.cumsum(var) <= Lam * (1 + 1e-12))
    # the spectrum recovered from data matches the generator's shape
    true = synth.spectrum(32, 1.2)
    assert np.all(np.abs(lam / lam.sum() - true / true.sum()) < 0.02)


def pin_rotation_isometry(o):
    """Lemma 1: W^T(x - mu) keeps every pairwise distance; mu maps to 0."""
    X, _, _ = synth.gaussian(200, 16, 1.0, seed=31, basis_seed=32)
    X = X + np.float32(5.0)
    mu, W, lam = o.pca(X)
    Xr = o.rotate(X, mu, W)
    Xd = X.astype(np.float64)
    d0 = ((Xd[:, None, :] - Xd[None, :, :]) ** 2).sum(-1)
    d1 = ((Xr[:, None, :] - Xr[None, :, :]) ** 2).sum(-1)
    assert _rel(d1, d0) < 1e-12
    assert np.allclose(Xr.mean(0), 0.0, atol=1e-12 * np.abs(Xr).max())
    assert np.allclose(Xr.T @ Xr / X.shape[0], np.diag(lam), atol=1e-11 * lam[0])


# --------------------------------------------------------------------------
# Section 3.1 / 3.2: the estimator (Lemma 3, Eq. 3, Eq. 4, Eq. 13)
# --------------------------------------------------------------------------

def pin_estimator_identity(o):
    """Eq. 13 at d = D: Lambda_D / Lambda_D = 1, so the estimate is the exact
    squared distance, bit for bit."""
    rng = np.random.default_rng(41)
    lam = synth.spectrum(24, 1.0)
    for _ in range(20):
        q, x = rng.standard_normal(24), rng.standard_normal(24)
        exact = 0.0
        for k in range(24):
            exact += (q[k] - x[k]) ** 2
        assert o.estimate_sq(q, x, 24, lam) == exact


def pin_estimator_unbiased(o):
    """Lemma 3 / Eq. 4 / Eq. 13: E[Lambda_D / Lambda_d * P_d] = E||X1 - X2||^2
    = 2 Lambda_D for iid X1, X2 with covariance diag(lambda) (PCA basis = I).
    Also checks the variance of the estimate's error against its closed form
    Var = sum_{k<=d} 2 (a-1)^2 (2 lambda_k)^2 + sum_{k>d} 2 (2 lambda_k)^2,
    a = Lambda_D / Lambda_d (Delta_k ~ N(0, 2 lambda_k) independent)."""
    D = 16
    lam = synth.spectrum(D, 1.0)
    rng = np.random.default_rng(43)
    m = 40000
    A = rng.standard_normal((m, D)) * np.sqrt(lam)
    B = rng.standard_normal((m, D)) * np.sqrt(lam)
    exact = ((A - B) ** 2).sum(1)
    for d in (2, 5, 9):
        est = np.array([o.estimate_sq(A[i], B[i], d, lam) for i in range(m)])
        mean, se = est.mean(), est.std(ddof=1) / math.sqrt(m)
        assert abs(mean - 2 * lam.sum()) < 5 * se, (d, mean, 2 * lam.sum(), se)
        a = lam.sum() / lam[:d].sum()
        var_cf = (2 * (a - 1) ** 2 * (2 * lam[:d]) ** 2).sum() + (2 * (2 * lam[d:]) ** 2).sum()
        var_mc = np.var(est - exact, ddof=1)
        assert abs(var_mc / var_cf - 1.0) < 0.06, (d, var_mc, var_cf)


# --------------------------------------------------------------------------
# Section 3.3: epsilon_d (Eq. 14) and the failure bound (Lemma 5)
# --------------------------------------------------------------------------

def pin_eps_quantile_golden(o):
    g = golden("eps_quantile.json")
    row = np.array(g["rho_sorted"])
    for case in g["cases"]:
        e = o.eps_quantile(row, case["alpha"])
        assert abs(e - case["eps"]) < 1e-15, (case, e)
        # library cross-check: inverted-CDF quantile = smallest x with F(x) >= 1 - alpha
        lib = np.quantile(row, 1.0 - case["alpha"], method="inverted_cdf") - 1.0
        assert abs(e - lib) < 1e-15
        assert np.mean(row - 1.0 > e) <= case["alpha"] + 1e-12


def pin_eps_ratio_golden(o):
    g = golden("eps_ratio.json")
    Xr = np.array([g["a"], g["b"]], float)
    rho = o.eps_sample(Xr, np.array(g["lam"], float), np.array([[0, 1]]), g["dlist"])
    assert rho.shape == (len(g["dlist"]), 1)
    assert _rel(rho[:, 0], g["rho"]) < 1e-15
    # a pair at distance zero has no ratio and is dropped
    rho0 = o.eps_sample(np.array([g["a"], g["a"]], float), np.array(g["lam"], float),
                        np.array([[0, 1]]), g["dlist"])
    assert rho0.shape[1] == 0


def _calib_setup(o, n=12000, D=32, p=1.0):
    X, _, _ = synth.gaussian(n, D, p, seed=51, basis_seed=52)
    mu, W, lam = o.pca(X)
    Xr = o.rotate(X, mu, W)
    return Xr, lam


def pin_eps_calibration(o):
    """Eq. 14: on held-out pairs the fraction with rho_d - 1 > eps_d is P_s
    within binomial error; rho_D = 1 exactly."""
    Xr, lam = _calib_setup(o)
    n, D = Xr.shape
    dl = [4, 8, 16, 24, D]
    cal = o.eps_sample(Xr, lam, synth.eps_pairs(n, 20000, seed=61), dl)
    held = o.eps_sample(Xr, lam, synth.eps_pairs(n, 20000, seed=62), dl)
    assert np.all(cal[-1] == 1.0) and np.all(held[-1] == 1.0)
    for alpha in (0.05, 0.1, 0.3):
        for t, d in enumerate(dl[:-1]):
            e = o.eps_quantile(cal[t], alpha)
            frac = float(np.mean(held[t] - 1.0 > e))
            sd = math.sqrt(alpha * (1 - alpha) / held.shape[1]) * math.sqrt(2)
            assert abs(frac - alpha) < 4 * sd, (alpha, d, frac)


def pin_failure_bound(o):
    """Lemma 5: when dis <= r a DCO fails (prunes) with probability at most
    floor((D-1)/delta_d) * P_s.  With r = dis for held-out pairs drawn like
    the calibration pairs, every failure is a test whose rho_d exceeded
    1 + eps_d, so the measured rate obeys the bound within binomial error."""
    Xr, lam = _calib_setup(o)
    n, D = Xr.shape
    dd = 8
    dl = list(range(dd, D, dd))
    cal = o.eps_sample(Xr, lam, synth.eps_pairs(n, 20000, seed=71), dl)
    alpha = 0.05
    eps = np.full(D + 1, np.nan)
    for t, d in enumerate(dl):
        eps[d] = o.eps_quantile(cal[t], alpha)
    pairs = synth.eps_pairs(n, 3000, seed=72)
    fails = 0
    for i, j in pairs:
        r = math.sqrt(((Xr[i] - Xr[j]) ** 2).sum()) * (1 + 1e-12)
        acc, d2, dims, _ = o.dco(Xr[i], Xr[j], dd, r, lam, eps)
        fails += (not acc)
        if acc:
            assert dims == D
    rate = fails / len(pairs)
    bound = ((D - 1) // dd) * alpha
    assert rate <= bound + 4 * math.sqrt(bound * (1 - bound) / len(pairs)), (rate, bound)
    assert rate > 0.0  # the test is active at this alpha


# --------------------------------------------------------------------------
# Algorithm 1 (Section 3.4), Definition 1
# --------------------------------------------------------------------------

def pin_dco_golden(o):
    g = golden("dco_traces.json")
    for case in g["cases"]:
        r = math.inf if case["r"] == "inf" else float(case["r"])
        acc, d2, dims, _ = o.dco(case["q"], case["o"], case["delta_d"], r, np.array(case["lam"], float),
                                 np.array(case["eps"], float), prune=case["prune"])
        assert acc == case["accept"], case["name"]
        assert dims == case["dims"], (case["name"], dims)
        if acc:
            assert d2 == case["dist2"], case["name"]


def _tiny_index(o, n=900, D=32, nc=7, dup=True, seed=81):
    X, _, _ = synth.gaussian(n, D, 1.0, seed=seed, basis_seed=seed + 1)
    if dup and n > 601:  # exact duplicates: distance ties that the (dist, id) order must break
        X[5] = X[17]
        X[300] = X[17]
        X[600] = X[401]
    mu, W, lam = o.pca(X)
    Xr = o.rotate(X, mu, W)
    init = synth.kmeans_init(n, nc, seed=seed + 2)
    cent, _, _, _ = o.kmeans(Xr, init, 5)
    assign, _ = o.assign(Xr, cent)
    Q, _, _ = synth.gaussian(25, D, 1.0, seed=seed + 3, basis_seed=seed + 1)
    Q[3] = X[17]
    Qr = o.rotate(Q, mu, W)
    return X, Xr, lam, cent, assign, Q, Qr


def _brute(Xr, Qr, K):
    d = ((Qr[:, None, :] - Xr[None, :, :]) ** 2).sum(-1)
    ids = np.empty((Qr.shape[0], K), np.int64)
    for i in range(Qr.shape[0]):
        order = np.lexsort((np.arange(Xr.shape[0]), d[i]))
        ids[i] = order[:K]
    return ids, np.take_along_axis(d, ids, 1)


def pin_search_fd_bruteforce(o):
    """IVF + FDScanning over every list (nprobe = N_c) is exact KNN; ordered
    by (distance, id), duplicates included."""
    X, Xr, lam, cent, assign, Q, Qr = _tiny_index(o)
    K = 12
    ids, dists, stats, _ = o.search(Xr, assign, cent, lam, Qr, K, cent.shape[0], 8, None, schedule=0)
    bid, bd = _brute(Xr, Qr, K)
    assert np.array_equal(ids, bid)
    assert _rel(dists, bd) < 1e-12
    assert np.all(stats[:, 0] == X.shape[0]) and np.all(stats[:, 1] == X.shape[0] * X.shape[1])
    # ground truth in the original coordinates agrees (Lemma 1)
    gid, _ = o.exact_knn(X, Q, K)
    assert np.mean(gid == bid) > 0.99


def _eps_for(o, Xr, lam, delta_d, alpha, seed=91):
    n, D = Xr.shape
    dl = list(range(delta_d, D, delta_d))
    rho = o.eps_sample(Xr, lam, synth.eps_pairs(n, 5000, seed=seed), dl)
    return o.eps_table(rho, dl, D, alpha)


def pin_search_dade_valid(o):
    """DADE results are exact distances of members of the probed lists, in
    (distance, id) order; an infinite eps reproduces FDScanning."""
    X, Xr, lam, cent, assign, Q, Qr = _tiny_index(o)
    K, nprobe = 10, 3
    eps = _eps_for(o, Xr, lam, 8, 0.1)
    ids, dists, stats, _ = o.search(Xr, assign, cent, lam, Qr, K, nprobe, 8, eps, schedule=1, tile=16)
    probe, _ = o.probe(Qr, cent, nprobe)
    for i in range(Qr.shape[0]):
        assert np.all(np.isin(assign[ids[i]], probe[i]))
        ex = ((Xr[ids[i]] - Qr[i]) ** 2).sum(1)
        assert _rel(dists[i], ex) < 1e-12
        key = list(zip(dists[i], ids[i]))
        assert key == sorted(key)
    assert np.all(stats[:, 1] < stats[:, 0] * X.shape[1])  # pruning saved dimensions
    fd = o.search(Xr, assign, cent, lam, Qr, K, nprobe, 8, None, schedule=1, tile=16)
    inf = o.search(Xr, assign, cent, lam, Qr, K, nprobe, 8, np.full(X.shape[1] + 1, np.inf),
                   schedule=1, tile=16)
    assert np.array_equal(fd[0], inf[0])
    # the same lists searched exhaustively: DADE recall close to FDScanning's
    assert np.mean([len(set(a) & set(b)) / K for a, b in zip(ids, fd[0])]) > 0.8


def pin_search_trace(o):
    """Brute-force re-run of the paper's sequential IVF loop: probe order,
    ascending ids, one DCO per candidate against the heap's current maximum,
    heap of the K best by (distance, id).  Built from single-pair DCO calls and
    a Python sorted list; must equal or_search's SEQUENTIAL schedule."""
    X, Xr, lam, cent, assign, Q, Qr = _tiny_index(o)
    K, nprobe, dd = 6, 3, 8
    eps = _eps_for(o, Xr, lam, dd, 0.2)
    ids, dists, _, _ = o.search(Xr, assign, cent, lam, Qr, K, nprobe, dd, eps, schedule=0)
    probe, _ = o.probe(Qr, cent, nprobe)
    for i in range(Qr.shape[0]):
        heap = []
        for c in probe[i]:
            for m in np.nonzero(assign == c)[0]:
                r = math.sqrt(heap[-1][0]) if len(heap) == K else math.inf
                acc, d2, _, _ = o.dco(Qr[i], Xr[m], dd, r, lam, eps)
                if acc:
                    heap = sorted(heap + [(d2, int(m))])[:K]
        assert [h[1] for h in heap] == list(ids[i][:len(heap)])
        assert np.allclose([h[0] for h in heap], dists[i][:len(heap)], rtol=0, atol=0)


def pin_search_schedules(o):
    """Epoch schedules: TILE(1) is SEQUENTIAL; a tile longer than every list
    is PROBE_ROUNDS."""
    X, Xr, lam, cent, assign, Q, Qr = _tiny_index(o)
    eps = _eps_for(o, Xr, lam, 8, 0.2)
    a = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=0)
    b = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=1, tile=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    c = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=2)
    d = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=1, tile=X.shape[0])
    assert np.array_equal(c[0], d[0]) and np.array_equal(c[2], d[2])


def pin_search_lagged_tiles(o):
    """Lagged tile schedule: lag 0 is the plain tile schedule; a lag longer
    than the scan never refreshes the threshold, so nothing is pruned and the
    result is FDScanning's over the same lists; a lag only prunes less."""
    X, Xr, lam, cent, assign, Q, Qr = _tiny_index(o)
    eps = _eps_for(o, Xr, lam, 8, 0.2)
    a = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=1, tile=16)
    b = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=1, tile=16, lag=0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    fd = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, None, schedule=1, tile=16)
    big = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=1, tile=16, lag=10**6)
    assert np.array_equal(big[0], fd[0]) and np.all(big[2][:, 3] == 0)
    lagged = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=1, tile=16, lag=3)
    assert np.all(lagged[2][:, 0] == a[2][:, 0])
    assert lagged[2][:, 3].sum() <= a[2][:, 3].sum()


def _hand_lists(points, assign, nlists, D=32):
    """Rotated points given by (dim, value) pairs, equal eigenvalues, eps_d = 0,
    lists probed in index order (centroid j sits at 100 j along dim 0, the
    query at the origin)."""
    Xr = np.zeros((len(points), D))
    for i, coords in enumerate(points):
        for dim, v in coords:
            Xr[i, dim] = v
    cent = np.zeros((nlists, D))
    cent[:, 0] = 100.0 * np.arange(nlists)
    return Xr, np.array(assign, np.int32), cent, np.ones(D), np.zeros(D + 1), np.zeros((1, D))


def pin_search_lagged_trace(o):
    """Lagged tile schedule, worked by hand (tile 1: every candidate is a tile;
    equal eigenvalues and eps_d = 0, D = 32, delta_d = 16, so a candidate is
    pruned at d = 16 iff 2 P_16 > r^2).  Query at the origin, K = 1, one list
    in id order: c0 = 10 (dim 0), c1 = 6 (dim 16), c2 = 5 (dim 0), c3 = 7
    (dim 0), c4 = 9 (dim 0).  Tile t is tested against r^2 after tiles
    0..t-1-L.
    L = 0: c0 exact (r = +inf), r^2 = 100; c1 (P_16 = 0) accepted at 36;
    c2 (2 x 25 = 50 > 36), c3 (98), c4 (162) pruned: id 1 at 36.
    L = 1: c1 sees r after tiles <= -1 (+inf) and is accepted; c2 sees r^2 =
    100 (after c0): 50 <= 100, exact 25 accepted, so id 2 at 25 wins; c3 sees
    r^2 = 36 (after c1): pruned; c4 sees 25 (after c2): pruned.
    L = 2: c1, c2 exact and accepted (+inf); c3 sees 100 (after c0): 98 <= 100,
    exact 49 accepted; c4 sees 36 (after c1): pruned.  Result id 2 at 25.
    Counters: (candidates, dims, accepted, pruned)."""
    Xr, assign, cent, lam, eps, Qr = _hand_lists(
        [[(0, 10.0)], [(16, 6.0)], [(0, 5.0)], [(0, 7.0)], [(0, 9.0)]], [0] * 5, 1)
    want = {0: (1, 36.0, [5, 32 + 32 + 16 + 16 + 16, 2, 3]),
            1: (2, 25.0, [5, 32 + 32 + 32 + 16 + 16, 3, 2]),
            2: (2, 25.0, [5, 32 * 4 + 16, 4, 1])}
    for lag, (wid, wd, wst) in want.items():
        ids, dists, stats, _ = o.search(Xr, assign, cent, lam, Qr, 1, 1, 16, eps, schedule=1, tile=1, lag=lag)
        assert ids[0, 0] == wid and dists[0, 0] == wd, (lag, ids, dists)
        assert stats[0].tolist() == wst, (lag, stats)


def _rerun_epochs(o, Xr, lam, eps, qr, K, dd, epochs):
    """Brute-force IVF loop from single-pair DCOs: epochs is a list of
    (candidate ids, index of the epoch whose result supplies r, or -1 for
    +inf); the K nearest by (distance, id) after every epoch."""
    heap, after, dims = [], [], 0
    for cands, src in epochs:
        r = math.sqrt(after[src]) if src >= 0 and math.isfinite(after[src]) else math.inf
        for m in cands:
            acc, d2, used, _ = o.dco(qr, Xr[m], dd, r, lam, eps)
            dims += used
            if acc:
                heap.append((d2, int(m)))
        heap = sorted(heap)[:K]
        after.append(heap[-1][0] if len(heap) == K else math.inf)
    return heap, dims


def pin_search_lagged_bruteforce(o):
    """Lagged tile schedule on a random index: tile t (tiles numbered over the
    query's scan, a tile never spans lists) is tested against r after tiles
    0..t-1-L; re-run from single-pair DCOs for L = 1, 2, 3."""
    X, Xr, lam, cent, assign, Q, Qr = _tiny_index(o)
    K, nprobe, dd, tile = 6, 3, 8, 16
    eps = _eps_for(o, Xr, lam, dd, 0.2)
    probe, _ = o.probe(Qr, cent, nprobe)
    for lag in (1, 2, 3):
        ids, dists, stats, _ = o.search(Xr, assign, cent, lam, Qr, K, nprobe, dd, eps, schedule=1, tile=tile,
                                        lag=lag)
        for i in range(0, Qr.shape[0], 3):
            tiles = [m[t:t + tile] for c in probe[i] for m in [np.nonzero(assign == c)[0]]
                     for t in range(0, len(m), tile)]
            heap, dims = _rerun_epochs(o, Xr, lam, eps, Qr[i], K, dd,
                                       [(tl, t - 1 - lag) for t, tl in enumerate(tiles)])
            assert [h[1] for h in heap] == list(ids[i][:len(heap)]), (lag, i)
            assert [h[0] for h in heap] == list(dists[i][:len(heap)])
            assert dims == stats[i, 1]


def pin_search_row_rounds_trace(o):
    """Row rounds, worked by hand (equal eigenvalues, eps_d = 0, D = 32,
    delta_d = 16: pruned at d = 16 iff 2 P_16 > r^2).  Query at the origin,
    K = 1, lists A (probed first) = {a0 (id 0): 10 in dim 0, a1 (id 1): 5 in
    dim 0}, B = {b0 (id 2): 6 in dim 16, b1 (id 3): 7 in dim 0}.
    Rounds of rows [0, 1), [1, 2) (R_1 = 1): round 0 takes a0 and b0 with
    r = +inf, both exact, r^2 = 36 (b0); round 1 tests a1 (2 x 25 = 50 > 36)
    and b1 (98 > 36): both pruned at d = 16, result b0 at 36.
    The sequential loop instead accepts a1 (50 <= 100 after a0) at 25.
    R_1 = 2: one round holds every row, all exact: a1 at 25."""
    Xr, assign, cent, lam, eps, Qr = _hand_lists(
        [[(0, 10.0)], [(0, 5.0)], [(16, 6.0)], [(0, 7.0)]], [0, 0, 1, 1], 2)
    r1 = o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=3, tile=1)
    assert r1[0][0, 0] == 2 and r1[1][0, 0] == 36.0
    assert r1[2][0].tolist() == [4, 32 + 32 + 16 + 16, 2, 2]
    seq = o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=0)
    assert seq[0][0, 0] == 1 and seq[1][0, 0] == 25.0
    assert seq[2][0].tolist() == [4, 32 * 3 + 16, 2, 1]
    r2 = o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=3, tile=2)
    assert r2[0][0, 0] == 1 and r2[1][0, 0] == 25.0
    assert r2[2][0].tolist() == [4, 32 * 4, 4, 0]


def pin_search_row_rounds_bruteforce(o):
    """Row rounds on a random index with uneven lists: round e holds rows
    [R_e, R_{e+1}) of every probed list (probe order, then row), R_0 = 0,
    R_1 = tile, R_{e+1} = 2 R_e, tested against r after the earlier rounds;
    re-run from single-pair DCOs.  FDScanning does not depend on the rounds,
    and R_1 above every list length is one exact round."""
    X, Xr, lam, cent, assign, Q, Qr = _tiny_index(o)
    K, nprobe, dd = 6, 4, 8
    eps = _eps_for(o, Xr, lam, dd, 0.2)
    probe, _ = o.probe(Qr, cent, nprobe)
    for tile in (1, 3, 16):
        ids, dists, stats, _ = o.search(Xr, assign, cent, lam, Qr, K, nprobe, dd, eps, schedule=3, tile=tile)
        for i in range(0, Qr.shape[0], 2):
            lists = [np.nonzero(assign == c)[0] for c in probe[i]]
            bounds, lo, hi = [], 0, tile
            while lo < max(len(m) for m in lists):
                bounds.append((lo, hi))
                lo, hi = hi, 2 * hi
            epochs = [([x for m in lists for x in m[a:b]], e - 1) for e, (a, b) in enumerate(bounds)]
            heap, dims = _rerun_epochs(o, Xr, lam, eps, Qr[i], K, dd, epochs)
            assert [h[1] for h in heap] == list(ids[i][:len(heap)]), (tile, i)
            assert [h[0] for h in heap] == list(dists[i][:len(heap)])
            assert dims == stats[i, 1] and stats[i, 0] == sum(len(m) for m in lists)
    fd = o.search(Xr, assign, cent, lam, Qr, K, nprobe, dd, None, schedule=1, tile=16)
    fdr = o.search(Xr, assign, cent, lam, Qr, K, nprobe, dd, None, schedule=3, tile=2)
    assert np.array_equal(fd[0], fdr[0]) and np.array_equal(fd[1], fdr[1])
    one = o.search(Xr, assign, cent, lam, Qr, K, nprobe, dd, eps, schedule=3, tile=X.shape[0])
    assert np.array_equal(one[0], fd[0]) and np.all(one[2][:, 3] == 0)


def pin_search_bracket(o):
    """The decision bracket (bias moves r^2 to r^2 (1 + bias) in every test
    and final compare), worked by hand: equal eigenvalues, eps_d = 0, D = 32,
    delta_d = 16, K = 1, query at the origin, list A = {a (id 0): 10 in dim 0}
    probed before B = {b (id 1): sqrt(50.0005) in dim 0}.  After a, r^2 = 100;
    b's estimate 2 x 50.0005 = 100.001 exceeds 100 by 1e-5 relative: pruned
    by the method (result a) and under bias -2e-5, kept under +2e-5 and then
    accepted at its exact 50.0005 (result b).  A final compare within the
    bracket: b' (id 1) = 10.000025 in dim 16 (P_16 = 0, exact 100.0005) is
    rejected by the method, accepted under +2e-5 but pushed out of the K
    nearest by a: a and b' tie at the K-th place within the bracket."""
    Xr, assign, cent, lam, eps, Qr = _hand_lists([[(0, 10.0)], [(0, math.sqrt(50.0005))]], [0, 1], 2)
    runs = {b: o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=1, bias=b, tol=2e-5)
            for b in (0.0, -2e-5, 2e-5)}
    assert runs[0.0][0][0, 0] == 0 and runs[-2e-5][0][0, 0] == 0 and runs[2e-5][0][0, 0] == 1
    assert abs(runs[2e-5][1][0, 0] - 50.0005) < 1e-12
    *_, stable, _, _ = o.search_bracket(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=1, btol=2e-5)
    assert not stable[0]        # b, far below the method's K-th distance, is one decision away
    Xr, assign, cent, lam, eps, Qr = _hand_lists([[(0, 10.0)], [(16, 10.000025)]], [0, 1], 2)
    base = o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=1, tol=2e-5)
    keep = o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=1, bias=2e-5, tol=2e-5)
    assert base[0][0, 0] == 0 and base[2][0].tolist() == [2, 64, 1, 0] and base[3][0] & 4 == 0
    assert keep[0][0, 0] == 0 and keep[2][0].tolist() == [2, 64, 2, 0] and keep[3][0] & 4
    *_, stable, sstable, boundary = o.search_bracket(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=1,
                                                     btol=2e-5)
    # a (100) and b' (100.0005) tie at the K-th place within the bracket: either is a
    # correct result (the boundary holds both), but the work counted differs
    assert stable[0] and not sstable[0]
    assert boundary[0] < 100.0 and 100.0005 <= 100.0 * (1 + 4e-5)
    # far from every threshold the three runs agree: stable
    Xr, assign, cent, lam, eps, Qr = _hand_lists([[(0, 10.0)], [(0, 2.0)]], [0, 1], 2)
    *_, stable, sstable, _ = o.search_bracket(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=1)
    assert stable[0] and sstable[0]


def pin_adsampling_as_uniform_spectrum(o):
    """ADSampling (the paper's baseline, Section 5) estimates sqrt(D/d) times
    the partial distance and prunes iff that exceeds (1 + eps0/sqrt(d)) r.
    With every lambda equal, Eq. 13's ratio Lambda_D/Lambda_d is D/d, so the
    oracle runs ADSampling through the same DCO with eps_d = eps0/sqrt(d).
    Worked case: D = 32, d = 16, eps0 = 2.1, q = 0, o with |o_:16|^2 = 9 and
    |o_16:|^2 = 16 (dis = 5): dis'_16 = sqrt(2 * 9) = 4.243; the bound is
    (1 + 2.1/4) r = 1.525 r, so r = 2.7 prunes (4.118 < 4.243) and r = 2.8
    does not (4.270), and then dis = 5 > 2.8 rejects at d = 32."""
    D = 32
    ones = np.ones(D)
    q = np.zeros(D)
    x = np.zeros(D)
    x[0] = 3.0
    x[16] = 4.0
    assert abs(o.estimate_sq(q, x, 16, ones) - 2.0 * 9.0) < 1e-12
    eps = np.zeros(D + 1)
    eps[16] = 2.1 / np.sqrt(16)
    acc, d2, dims, _ = o.dco(q, x, 16, 2.7, ones, eps)
    assert not acc and dims == 16
    acc, d2, dims, _ = o.dco(q, x, 16, 2.8, ones, eps)
    assert not acc and dims == 32
    acc, d2, dims, _ = o.dco(q, x, 16, 5.0, ones, eps)
    assert acc and dims == 32 and abs(d2 - 25.0) < 1e-12


def pin_search_seeded_trace(o):
    """Seeded schedule, worked by hand (Section 3.3 test with eps_d = 0 and
    equal eigenvalues, so Lambda_32 / Lambda_16 = 2).  Query at the origin,
    K = 1, two lists probed in order A, B, delta_d = 16, D = 32.
    A = {a: |a| = 10}; B = {p1 (id 1): 5 in dim 16, p2 (id 2): 4 in dim 0,
    p3 (id 3): 20 in dim 0}.
    Running threshold (TILE(1)): r = 10 after A; p1 is not pruned
    (P_16 = 0) and is accepted, r = 5; p2 has dis'_16 = sqrt(2) 4 = 5.66 > 5
    and is pruned, as is p3 (28.3 > 5): the result is p1 at 25.  Frozen
    threshold after A (seed 1): p2 is tested against r = 10, survives, and
    is accepted at its exact 16; p3 (28.3 > 10) is pruned: the result is p2."""
    D = 32
    Xr = np.zeros((4, D))
    Xr[0, 0] = 10.0
    Xr[1, 16] = 5.0
    Xr[2, 0] = 4.0
    Xr[3, 0] = 20.0
    assign = np.array([0, 1, 1, 1], np.int32)
    cent = np.zeros((2, D))
    cent[1, 0] = 100.0                     # list A (0) is probed first
    lam = np.ones(D)
    eps = np.zeros(D + 1)
    Qr = np.zeros((1, D))
    tile = o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=1)
    assert tile[0][0, 0] == 1 and tile[1][0, 0] == 25.0
    assert tile[2][0].tolist() == [4, 32 + 32 + 16 + 16, 2, 2]      # p2, p3 pruned at d = 16
    seeded = o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=1, seed=1)
    assert seeded[0][0, 0] == 2 and seeded[1][0, 0] == 16.0
    assert seeded[2][0].tolist() == [4, 32 * 3 + 16, 3, 1]


def pin_search_whole_list_epochs(o):
    """Tiles as threshold epochs, worked by hand (equal eigenvalues, eps_d = 0,
    D = 32, delta_d = 16: prune iff 2 P_16 > r^2).  Query at the origin, K = 1,
    lists probed A then B; A = {a1 (id 0): 10 in dim 0, a2 (id 1): 12 in dim 0},
    B = {b1 (id 2): 5 in dim 16}.  Tile 1 (seed 1): a1 is exact (r = +inf) and
    sets r = 10; a2 is pruned at d = 16 (2 x 144 > 100); b1 (P_16 = 0) is
    accepted at 25.  Whole-list tiles (tile 4, seed 1): all of A is one epoch
    with r = +inf, so a2 is computed exactly and accepted too; r = 10 after A
    and b1 is accepted at 25 either way."""
    D = 32
    Xr = np.zeros((3, D))
    Xr[0, 0], Xr[1, 0], Xr[2, 16] = 10.0, 12.0, 5.0
    assign = np.array([0, 0, 1], np.int32)
    cent = np.zeros((2, D))
    cent[1, 0] = 100.0
    lam, eps, Qr = np.ones(D), np.zeros(D + 1), np.zeros((1, D))
    per = o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=1, seed=1)
    whole = o.search(Xr, assign, cent, lam, Qr, 1, 2, 16, eps, schedule=1, tile=4, seed=1)
    for r in (per, whole):
        assert r[0][0, 0] == 2 and r[1][0, 0] == 25.0
    assert per[2][0].tolist() == [3, 32 + 16 + 32, 2, 1]
    assert whole[2][0].tolist() == [3, 32 * 3, 3, 0]


def pin_search_seeded_limits(o):
    """Seeded schedule limits: seed >= nprobe is the plain tile schedule;
    FDScanning does not depend on the schedule; freezing r after the seed
    lists can only prune less than the running threshold."""
    X, Xr, lam, cent, assign, Q, Qr = _tiny_index(o)
    eps = _eps_for(o, Xr, lam, 8, 0.2)
    a = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=1, tile=16)
    b = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=1, tile=16, seed=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    fd = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, None, schedule=1, tile=16)
    fds = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, None, schedule=1, tile=16, seed=1)
    assert np.array_equal(fd[0], fds[0]) and np.array_equal(fd[1], fds[1])
    for seed in (1, 2, 3):
        s = o.search(Xr, assign, cent, lam, Qr, 8, 4, 8, eps, schedule=1, tile=16, seed=seed)
        assert np.array_equal(s[2][:, 0], a[2][:, 0])
        assert np.all(s[2][:, 3] <= a[2][:, 3])
        for i in range(Qr.shape[0]):   # results: exact distances of distinct ids, ascending
            ok = s[0][i] >= 0
            ex = ((Xr[s[0][i][ok]] - Qr[i]) ** 2).sum(1)
            assert np.allclose(s[1][i][ok], ex, rtol=1e-12) and np.all(np.diff(s[1][i][ok]) >= 0)
            assert len(set(s[0][i][ok].tolist())) == int(ok.sum())


def pin_search_short_lists(o):
    """Fewer candidates than K: the missing slots are (-1, +inf)."""
    X, Xr, lam, cent, assign, Q, Qr = _tiny_index(o, n=40, nc=7, dup=False)
    K = 64
    ids, dists, stats, _ = o.search(Xr, assign, cent, lam, Qr, K, 2, 8, None, schedule=1, tile=4)
    for i in range(Qr.shape[0]):
        m = int(stats[i, 0])
        assert m < K
        assert np.all(ids[i, m:] == -1) and np.all(np.isinf(dists[i, m:]))
        assert np.all(ids[i, :m] >= 0)


# --------------------------------------------------------------------------
# IVF building blocks (Section 3.4) against library routines
# --------------------------------------------------------------------------

def pin_kmeans_vs_scipy(o):
    """Lloyd iterations from given initial points vs scipy's kmeans2 with the
    same initial matrix (ties to the lower index, empty clusters keep their
    centroid); the objective never increases."""
    from scipy.cluster.vq import kmeans2, vq
    X, _, _ = synth.gaussian(1500, 8, 0.5, seed=101, basis_seed=102)
    Xd = X.astype(np.float64)
    init = synth.kmeans_init(1500, 12, seed=103)
    init[5] = init[4]  # duplicated start: one cluster stays empty, ties resolved low
    cent, assign, obj, _ = o.kmeans(Xd, init, 6)
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        ref_c, ref_l = kmeans2(Xd, Xd[init].copy(), iter=6, minit="matrix", missing="warn")
    assert np.allclose(cent, ref_c, rtol=0, atol=1e-12 * np.abs(Xd).max())
    assert np.array_equal(assign, ref_l)
    assert np.all(np.diff(obj) <= 1e-9 * obj[0])
    a2, _ = o.assign(Xd, cent)
    assert np.array_equal(a2, vq(Xd, cent)[0])


def pin_list_means(o):
    X, _, _ = synth.gaussian(500, 6, 1.0, seed=111, basis_seed=112)
    Xd = X.astype(np.float64)
    lab = synth.zipf_assign(500, 9, seed=113)
    cent = o.list_means(Xd, lab, 10)
    for c in range(10):
        m = lab == c
        ref = Xd[m].mean(0) if m.any() else np.zeros(6)
        assert np.allclose(cent[c], ref, atol=1e-13)


def pin_probe_order(o):
    rng = np.random.default_rng(121)
    Qr = rng.standard_normal((30, 10))
    cent = rng.standard_normal((40, 10))
    cent[7] = cent[3]  # equal distances: order by centroid id
    pr, _ = o.probe(Qr, cent, 9)
    d = ((Qr[:, None, :] - cent[None, :, :]) ** 2).sum(-1)
    for i in range(30):
        assert list(pr[i]) == list(np.lexsort((np.arange(40), d[i]))[:9])


def pin_exact_knn(o):
    X, _, _ = synth.gaussian(400, 12, 1.0, seed=131, basis_seed=132)
    X[10] = X[20]
    Q, _, _ = synth.gaussian(15, 12, 1.0, seed=133, basis_seed=132)
    Q[0] = X[20]
    ids, dists = o.exact_knn(X, Q, 7)
    bid, bd = _brute(X.astype(np.float64), Q.astype(np.float64), 7)
    assert np.array_equal(ids, bid)
    assert _rel(dists, bd) < 1e-12


def pin_sampled_index(o):
    """The sampled index (PCA over all objects, only the reachable rows
    rotated, centroids from raw means) answers exactly as the full index."""
    import oracle
    w = synth.Workload("pin_mix", 4000, 48, 12, 1.0, 8, 0.0, 3.0, 1.0, False, False, 32, (6,), 10, (16,), 0.1)
    X, Q, lab = synth.make(w)
    assign = synth.component_lists(lab, 32)
    assert np.array_equal(assign // 4, lab)
    pairs = synth.eps_pairs(4000, 3000, seed=141)
    full = oracle.Index(X, n_clusters=32, assign=assign, pairs=pairs, oracle=o)
    samp = oracle.SampledIndex(X, assign, 32, pairs, Q, 6, oracle=o)
    assert samp.rows.size < 4000
    for dd, seed, tile in ((16, 0, 64), (32, 2, 128), (16, 1, 1 << 20)):
        a = full.search(Q, 10, 6, dd, 0.1, tile=tile, seed=seed)
        b = samp.search(10, 6, dd, 0.1, tile=tile, seed=seed)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
        assert _rel(a[1], b[1]) < 1e-11
    # every list probed, no pruning: exact nearest neighbours
    allp = oracle.SampledIndex(X, assign, 32, pairs, Q, 32, oracle=o)
    ids, dists, _, _ = allp.search(10, 32, 16, 0.1, prune=False)
    bid, bd = _brute(X.astype(np.float64), Q.astype(np.float64), 10)
    assert np.array_equal(ids, bid) and _rel(dists, bd) < 1e-10


# --------------------------------------------------------------------------
# Section 3.4: HNSW with DADE DCOs (HNSW*): the layer-0 graph and the beam search
# --------------------------------------------------------------------------

def pin_hnsw_graph_golden(o):
    """Hand-worked layer-0 graphs on a line (tests/golden/hnsw_graph.json)."""
    g = golden("hnsw_graph.json")
    X = np.asarray(g["points"], float)
    for c in g["cases"]:
        nbr, gs, gf = o.hnsw_graph(X, c["kc"], c["M"], c["M0"])
        assert nbr.tolist() == c["nbr"], c["name"]


def pin_hnsw_trace(o):
    """Hand-worked beam search with DCOs, both threshold schedules and
    FDScanning (tests/golden/hnsw_trace.json)."""
    g = golden("hnsw_trace.json")
    X = np.asarray(g["points"], float)
    q = np.asarray([g["query"]], float)
    for c in g["cases"]:
        eps = np.asarray(g["eps"], float) if c["prune"] else None
        ids, dists, stats, flags = o.hnsw_search(X, np.asarray(g["nbr"]), np.asarray(g["lam"], float), q,
                                                 g["entry"], g["K"], g["ef"], g["delta_d"], eps, c["schedule"])
        assert ids[0].tolist() == c["ids"], c["name"]
        assert _rel(dists[0], c["dists"]) < 1e-12, c["name"]
        assert stats[0].tolist() == c["stats"], c["name"]
        assert flags[0] == 0, c["name"]


def _hnsw_setup(o, n=700, D=24, seed=201):
    X, _, _ = synth.gaussian(n, D, 1.0, seed=seed, basis_seed=seed + 1)
    Q, _, _ = synth.gaussian(25, D, 1.0, seed=seed + 2, basis_seed=seed + 1)
    return X.astype(np.float64), Q.astype(np.float64)


def _reachable(nbr, start):
    seen, todo = {int(start)}, [int(start)]
    while todo:
        for v in nbr[todo.pop()]:
            if v >= 0 and int(v) not in seen:
                seen.add(int(v))
                todo.append(int(v))
    return seen


def pin_hnsw_exhaustive_is_exact(o):
    """With FDScanning and R as large as the data (ef = n), the search
    expands every object reachable from the entry: on a connected graph it
    returns the exact K nearest (brute force), in both schedules."""
    X, Q = _hnsw_setup(o)
    n = X.shape[0]
    nbr, _, _ = o.hnsw_graph(X, 24, 8, 16)
    assert len(_reachable(nbr, 0)) == n
    bid, bd = _brute(X, Q, 10)
    for sch in (0, 1):
        ids, dists, stats, _ = o.hnsw_search(X, nbr, np.ones(X.shape[1]), Q, [0], 10, n, 8, None, sch)
        assert np.array_equal(ids, bid) and _rel(dists, bd) < 1e-12
        assert (stats[:, 0] == n).all() and (stats[:, 4] == n).all()


def pin_hnsw_complete_graph(o):
    """On the complete graph the entry's expansion visits every object with
    r = +inf (R holds one object when the node schedule reads r), so even
    ef = K returns the exact K nearest; DADE with eps = +inf (no test can
    reject) gives FDScanning's results and counters."""
    X, Q = _hnsw_setup(o, n=200, D=16, seed=211)
    n, D = X.shape
    nbr = np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)
    bid, bd = _brute(X, Q, 7)
    lam = np.linspace(3.0, 0.5, D)
    fd = o.hnsw_search(X, nbr, lam, Q, [5], 7, 7, 4, None, 1)
    assert np.array_equal(fd[0], bid) and _rel(fd[1], bd) < 1e-12
    inf_eps = np.full(D + 1, np.inf)
    dade = o.hnsw_search(X, nbr, lam, Q, [5], 7, 7, 4, inf_eps, 1)
    assert np.array_equal(dade[0], fd[0]) and np.array_equal(dade[2], fd[2])


def pin_hnsw_dade_prunes_only_beyond_r(o):
    """Section 3.3: a pruned neighbour's estimate exceeded (1 + eps_d) r, and
    every reported distance is exact; with the eps of a sampled
    significance level the results stay near FDScanning's (recall of the
    FDScanning results at least 0.9 over the batch) while fewer dims are
    read."""
    X, Q = _hnsw_setup(o, n=900, D=32, seed=221)
    nbr, _, _ = o.hnsw_graph(X, 32, 8, 16)
    mu, W, lam = o.pca(X.astype(np.float32))
    Xr, Qr = o.rotate(X.astype(np.float32), mu, W), o.rotate(Q.astype(np.float32), mu, W)
    eps = _eps_for(o, Xr, lam, 8, 0.1)
    fd = o.hnsw_search(Xr, nbr, lam, Qr, [0], 10, 40, 8, None, 1)
    dd = o.hnsw_search(Xr, nbr, lam, Qr, [0], 10, 40, 8, eps, 1)
    exact = ((Qr[:, None, :] - Xr[dd[0]]) ** 2).sum(-1)
    assert _rel(dd[1], exact) < 1e-12
    hit = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(dd[0], fd[0])])
    assert hit >= 0.9
    assert dd[2][:, 1].sum() < fd[2][:, 1].sum() and dd[2][:, 3].sum() > 0


def pin_hnsw_path_flags(o):
    """A query with no path near-tie at tol takes the same path under every
    threshold moved by less than tol: runs with r^2 scaled by 1 -/+ tol/2
    return its ids and counters unchanged."""
    X, Q = _hnsw_setup(o, n=900, D=32, seed=231)
    nbr, _, _ = o.hnsw_graph(X, 32, 8, 16)
    mu, W, lam = o.pca(X.astype(np.float32))
    Xr, Qr = o.rotate(X.astype(np.float32), mu, W), o.rotate(Q.astype(np.float32), mu, W)
    eps = _eps_for(o, Xr, lam, 8, 0.1)
    Q = np.concatenate([Q] * 4) + 0.01 * np.random.default_rng(232).standard_normal((4 * Q.shape[0], Q.shape[1]))
    Qr = o.rotate(Q.astype(np.float32), mu, W)
    tol = 1e-4
    base = o.hnsw_search(Xr, nbr, lam, Qr, [0], 10, 30, 8, eps, 1, tol=tol)
    stable = (base[3] & 15) == 0
    assert 10 <= stable.sum() < stable.size
    moved = np.zeros(stable.size, bool)
    for b in (-tol / 2, tol / 2):
        r = o.hnsw_search(Xr, nbr, lam, Qr, [0], 10, 30, 8, eps, 1, tol=tol, bias=b)
        assert np.array_equal(r[0][stable], base[0][stable]) and np.array_equal(r[2][stable], base[2][stable])
        moved |= (r[2] != base[2]).any(1)
    assert moved.any()        # the moved thresholds do change the path of some flagged queries


def pin_hnsw_fp32_arithmetic(o):
    """The FP32 DCO (the paper's scalar FP32 arithmetic, test in squared form
    with FP32 c_j) decides as the FP64 DCO wherever no decision of the FP64
    path lies within 1e-5: same ids and counters on those queries, distances
    within FP32 rounding.  On the hand-worked trace it gives the golden
    counters."""
    import oracle
    g = golden("hnsw_trace.json")
    X32 = np.asarray(g["points"], np.float32)
    q32 = np.asarray([g["query"]], np.float32)
    lam, eps = np.asarray(g["lam"], float), np.asarray(g["eps"], float)
    for c in g["cases"]:
        coef = oracle.coef_f32(lam, eps, 2, g["delta_d"]) if c["prune"] else None
        ids, dists, stats, _ = o.hnsw_search(X32, np.asarray(g["nbr"]), lam, q32, g["entry"], g["K"], g["ef"],
                                             g["delta_d"], None, c["schedule"], coef32=coef)
        assert ids[0].tolist() == c["ids"] and stats[0].tolist() == c["stats"], c["name"]
        assert _rel(dists[0], c["dists"]) < 1e-6, c["name"]
    X, Q = _hnsw_setup(o, n=1500, D=48, seed=251)
    nbr, _, _ = o.hnsw_graph(X, 32, 8, 16)
    mu, W, lam = o.pca(X.astype(np.float32))
    Xr32 = o.rotate(X.astype(np.float32), mu, W).astype(np.float32)
    Qr32 = o.rotate(Q.astype(np.float32), mu, W).astype(np.float32)
    eps = _eps_for(o, Xr32.astype(np.float64), lam, 16, 0.1)
    coef = oracle.coef_f32(lam, eps, 48, 16)
    for sch in (0, 1):
        a = o.hnsw_search(Xr32.astype(np.float64), nbr, lam, Qr32.astype(np.float64), [0], 10, 40, 16, eps, sch)
        b = o.hnsw_search(Xr32, nbr, lam, Qr32, [0], 10, 40, 16, None, sch, coef32=coef)
        stable = (a[3] & 15) == 0
        assert stable.sum() >= 15
        assert np.array_equal(a[0][stable], b[0][stable]) and np.array_equal(a[2][stable], b[2][stable])
        assert _rel(b[1][stable], a[1][stable]) < 1e-5
        assert b[2][:, 3].sum() > 0                       # the FP32 test does prune


def pin_hnsw_visit_budget(o):
    """The visit budget stops the search at the first pop after max_visits
    DCOs (flag 32); without it the search is the same up to that point."""
    X, Q = _hnsw_setup(o, n=500, D=16, seed=241)
    nbr, _, _ = o.hnsw_graph(X, 24, 8, 16)
    full = o.hnsw_search(X, nbr, np.ones(16), Q, [0], 5, 50, 16, None, 1)
    cut = o.hnsw_search(X, nbr, np.ones(16), Q, [0], 5, 50, 16, None, 1, max_visits=40)
    assert (cut[3] & 32).all() and not (full[3] & 32).any()
    assert (cut[2][:, 0] >= 40).all() and (cut[2][:, 0] < 40 + 16 + 1).all()
    assert (cut[2][:, 0] <= full[2][:, 0]).all()


ALL = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
