"""Seeded synthetic workloads for DADE-IVF.

This module draws inputs only: base vectors, queries, mixture labels, the
k-means initial centroid ids and the pairs used to estimate epsilon_d.  It
holds none of the method's arithmetic (no PCA, no distances, no k-means, no
estimates), so both the CUDA path and the CPU oracle may consume what it
produces.

The paper's datasets (Table 1: MSong, DEEP, Word2Vec, GIST, GloVe, Tiny5M)
are not available here; these generators stand in for them with the shapes,
spectra and cluster structure listed in ``WORKLOADS``.  Nothing from those
datasets is reproduced.

Recipe shared by every workload (numpy PCG64, fixed seeds):
  * spectrum  lambda_i = i^-p, rescaled so that sum(lambda) = D;
  * basis     a Haar-random orthogonal matrix (QR of a Gaussian, sign fixed
              so that R has a positive diagonal);
  * component x = m_c + s * Q (sqrt(lambda) * z),  z ~ N(0, I).
Mixtures are anisotropic as a whole: every component shares the basis Q, and
the component means are drawn along the same spectrum,
m_c = offset + t * Q (sqrt(lambda) * g_c), so the mixture's covariance has the
power-law spectrum in the basis Q (``shared_basis=True``, the default).  With
``shared_basis=False`` every component gets its own Haar basis and the means
are isotropic, which averages the mixture's covariance towards isotropy.
Seeds: 0 base, 1 queries, 2 basis/means, 3 k-means init, 4 epsilon pairs.
"""
from __future__ import annotations

import dataclasses
import numpy as np

SEED_BASE, SEED_QUERY, SEED_BASIS, SEED_KMEANS, SEED_PAIRS = 0, 1, 2, 3, 4


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int              # base vectors
    d: int              # dimension
    nq: int             # queries
    p: float            # spectrum exponent, lambda_i ~ i^-p
    n_comp: int         # mixture components (1 = single Gaussian)
    mean_offset: float  # component means m_c = mean_offset + mean_scale * g_c
    mean_scale: float
    within_scale: float
    integer: bool       # round and clip to 0..255 (stored as float32)
    normalise: bool     # L2-normalise every vector
    n_clusters: int
    nprobe: tuple
    k: int
    delta_d: tuple
    alpha: float
    kmeans_iters: int = 10
    shared_basis: bool = True
    comp_zipf: float = 0.0   # > 0: component weights Zipf(comp_zipf) over a seeded rank permutation
    lists_are_components: bool = False   # the IVF lists are the generating components (no k-means)


# Constants proposed for the workloads (sizes from the benchmark configs; the
# paper fixes P_s = 0.1, delta_d = 32, N_c ~ sqrt(N) = 4096 in Section 4.1).
WORKLOADS = {
    "c1_gauss_10k_d128": Workload("c1_gauss_10k_d128", 10_000, 128, 100, 1.2, 1,
                                  0.0, 0.0, 1.0, False, False, 64, (8,), 10, (32,), 0.05),
    "c2_mix_1m_d128": Workload("c2_mix_1m_d128", 1_000_000, 128, 10_000, 1.0, 64,
                               40.0, 25.0, 20.0, True, False, 4096,
                               (16, 32, 64, 128, 256), 100, (16, 32, 64), 0.05),
    "c3_mix_1m_d960": Workload("c3_mix_1m_d960", 1_000_000, 960, 1_000, 0.8, 64,
                               0.0, 2.0, 1.0, False, False, 4096,
                               (32, 64, 128), 10, (32,), 0.05),
    "c4_zipf_10m_d768": Workload("c4_zipf_10m_d768", 10_000_000, 768, 10_000, 1.5, 16384,
                                 0.0, 2.0, 1.0, False, True, 16384,
                                 (64,), 10, (32,), 0.05, comp_zipf=1.1, lists_are_components=True),
    "c5_mix_5m_d256": Workload("c5_mix_5m_d256", 5_000_000, 256, 10_000, 1.0, 32,
                               0.0, 2.0, 1.0, False, False, 8192,
                               (16, 64, 128), 10, (32,), 0.05),
}


def spectrum(d: int, p: float) -> np.ndarray:
    """lambda_i = i^-p (i = 1..d), rescaled so that the sum is d."""
    lam = np.arange(1, d + 1, dtype=np.float64) ** (-float(p))
    return lam * (d / lam.sum())


def haar(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random orthogonal d x d matrix (QR of a Gaussian with sign fix)."""
    g = rng.standard_normal((d, d))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def _components(w: Workload):
    """Component means and rotations, all drawn from the basis seed."""
    rng = np.random.default_rng(SEED_BASIS)
    lam = spectrum(w.d, w.p)
    if w.shared_basis or w.n_comp == 1:
        Q = haar(w.d, rng)
        rots = [Q] * w.n_comp
        g = rng.standard_normal((w.n_comp, w.d)) * np.sqrt(lam)[None, :]
        means = np.zeros((1, w.d)) if w.n_comp == 1 else w.mean_offset + w.mean_scale * (g @ Q.T)
    else:
        means = w.mean_offset + w.mean_scale * rng.standard_normal((w.n_comp, w.d))
        rots = [haar(w.d, rng) for _ in range(w.n_comp)]
    return lam, means, rots


def component_weights(w: Workload) -> np.ndarray:
    """Mixture weights: uniform, or Zipf(comp_zipf) by rank with the ranks
    dealt to components by a seeded permutation."""
    if w.comp_zipf <= 0:
        return np.full(w.n_comp, 1.0 / w.n_comp)
    rng = np.random.default_rng(SEED_BASIS + 5)
    wts = np.arange(1, w.n_comp + 1, dtype=np.float64) ** (-w.comp_zipf)
    wts = wts[rng.permutation(w.n_comp)]
    return wts / wts.sum()


def _draw_weighted(w: Workload, n: int, seed: int, comps):
    """Shared-basis mixture with uneven weights, drawn in row chunks (FP32
    products): x = m_c + s Q (sqrt(lambda) z), optionally L2-normalised.
    Chunk k draws its z from its own generator seeded by (seed, k), so the
    chunks can be drawn on several threads with the same result."""
    import concurrent.futures as cf
    import os
    lam, means, rots = comps
    rng = np.random.default_rng(seed)
    labels = rng.choice(w.n_comp, size=n, p=component_weights(w)).astype(np.int32)
    out = np.empty((n, w.d), np.float32)
    sl = np.sqrt(lam).astype(np.float32)
    QT = np.ascontiguousarray(rots[0].T, np.float32)
    M = means.astype(np.float32)
    chunk = 1 << 17

    def one(k):
        s, e = k * chunk, min(n, (k + 1) * chunk)
        z = np.random.default_rng([seed, k]).standard_normal((e - s, w.d), dtype=np.float32)
        z *= sl[None, :]
        x = M[labels[s:e]] + np.float32(w.within_scale) * (z @ QT)
        if w.normalise:
            x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[s:e] = x

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(one, range((n + chunk - 1) // chunk)))
    return out, labels


def _draw(w: Workload, n: int, seed: int, comps=None):
    lam, means, rots = comps if comps is not None else _components(w)
    if w.comp_zipf > 0:
        return _draw_weighted(w, n, seed, (lam, means, rots))
    rng = np.random.default_rng(seed)
    labels = rng.integers(0, w.n_comp, size=n).astype(np.int32) if w.n_comp > 1 \
        else np.zeros(n, np.int32)
    out = np.empty((n, w.d), np.float32)
    sl = np.sqrt(lam)
    chunk = 1 << 16
    for c in range(w.n_comp):
        idx = np.nonzero(labels == c)[0]
        for s in range(0, idx.size, chunk):
            sub = idx[s:s + chunk]
            z = rng.standard_normal((sub.size, w.d)) * sl[None, :]
            x = means[c][None, :] + w.within_scale * (z @ rots[c].T)
            if w.integer:
                x = np.clip(np.rint(x), 0.0, 255.0)
            if w.normalise:
                x = x / np.linalg.norm(x, axis=1, keepdims=True)
            out[sub] = x.astype(np.float32)
    return out, labels


def make(name_or_w, n: int | None = None, nq: int | None = None):
    """Return (base float32 [n,d], queries float32 [nq,d], base labels int32 [n]).

    ``n`` / ``nq`` shrink a workload (same distribution, fewer draws)."""
    w = WORKLOADS[name_or_w] if isinstance(name_or_w, str) else name_or_w
    comps = _components(w)
    base, labels = _draw(w, w.n if n is None else n, SEED_BASE, comps)
    queries, _ = _draw(w, w.nq if nq is None else nq, SEED_QUERY, comps)
    return base, queries, labels


def gaussian(n: int, d: int, p: float, seed: int = SEED_BASE, basis_seed: int = SEED_BASIS):
    """Single zero-mean Gaussian with lambda_i ~ i^-p in a Haar basis."""
    lam = spectrum(d, p)
    q = haar(d, np.random.default_rng(basis_seed))
    z = np.random.default_rng(seed).standard_normal((n, d)) * np.sqrt(lam)[None, :]
    return (z @ q.T).astype(np.float32), lam, q


def kmeans_init(n: int, n_clusters: int, seed: int = SEED_KMEANS) -> np.ndarray:
    """n_clusters distinct base ids drawn by a seeded permutation."""
    rng = np.random.default_rng(seed)
    return rng.permutation(n)[:n_clusters].astype(np.int64)


def eps_pairs(n: int, m: int, seed: int = SEED_PAIRS) -> np.ndarray:
    """m pairs (i, j), i != j, drawn uniformly; returned as int64 [m, 2]."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n, size=m)
    j = rng.integers(0, n - 1, size=m)
    j = j + (j >= i)
    return np.stack([i, j], axis=1).astype(np.int64)


def zipf_assign(n: int, n_lists: int, s: float = 1.1, seed: int = SEED_BASE + 7) -> np.ndarray:
    """Random list labels with Zipf(s)-skewed list sizes (a seeded rank
    permutation decides which list gets which rank).  Used to exercise
    uneven inverted lists."""
    rng = np.random.default_rng(seed)
    wts = np.arange(1, n_lists + 1, dtype=np.float64) ** (-s)
    wts = wts[rng.permutation(n_lists)]
    wts /= wts.sum()
    return rng.choice(n_lists, size=n, p=wts).astype(np.int32)


def component_lists(labels: np.ndarray, n_lists: int, seed: int = SEED_BASE + 11) -> np.ndarray:
    """Seeded list labels that follow the mixture: each component's members
    are dealt uniformly at random to n_lists / n_components lists of their
    own (list = component * per + draw).  A fixed list assignment that both
    sides of a full-size comparison can share."""
    labels = np.asarray(labels, np.int64)
    n_comp = int(labels.max()) + 1
    per = n_lists // n_comp
    if per < 1 or per * n_comp != n_lists:
        raise ValueError("n_lists must be a multiple of the number of components")
    rng = np.random.default_rng(seed)
    return (labels * per + rng.integers(0, per, size=labels.size)).astype(np.int32)
