"""Comparison of CUDA-path results with the FP64 oracle.

Tolerance (stated here, used by every parity test):
  * ids: equal, position by position, for every query whose oracle trace has
    no near-tie (oracle flags: a test or compare whose two sides are within
    TIE_TOL = 1e-5 relative, the K-th place of a merge, or the probe order);
    within a run of results whose oracle distances agree to 1e-5 relative
    only the set of ids must match (their order is decided by rounding).
  * distances: |gpu - oracle| <= 1e-5 * oracle + ATOL_REL * scale, where
    scale is the mean squared norm of the rotated base vectors.  The FP32
    path rounds the rotation (a D-term FP32 dot product per coordinate) and
    the D-term sum of squares; both errors are a few 1e-7 of the squared
    norms involved, so the absolute term only matters for distances far
    below the data's scale (near-duplicates).
  * flagged queries are validated instead: ids distinct and from the
    database, distances exact for those ids, ascending order, and at least
    90% of the oracle's ids present (a flipped near-tie decision moves a few
    results, not the list).  A query runs thousands of threshold tests, so
    the flagged fraction grows with nprobe and K; it must stay below 30%.
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-5
ATOL_REL = 2e-6
TIE_TOL = 1e-5


def _runs(d, tol=TIE_TOL):
    """Split positions into runs of near-equal distances."""
    runs, start = [], 0
    for i in range(1, len(d) + 1):
        if i == len(d) or not (np.isfinite(d[i]) and np.isfinite(d[i - 1])
                               and abs(d[i] - d[i - 1]) <= tol * max(abs(d[i]), abs(d[i - 1]))):
            runs.append((start, i))
            start = i
    return runs


def compare(g_ids, g_d, o_ids, o_d, flags, scale, exact_d=None, max_flagged_frac=0.3):
    """Assert GPU results (g_*) match the oracle's (o_*).  exact_d(q, ids) -> FP64
    distances, used to validate flagged queries.  Returns a summary dict."""
    nq, K = o_ids.shape
    atol = ATOL_REL * scale
    flagged, mismatched_flagged = 0, 0
    for q in range(nq):
        ok_ids = True
        for a, b in _runs(o_d[q]):
            if b - a == 1:
                ok_ids &= g_ids[q, a] == o_ids[q, a]
            else:
                ok_ids &= set(g_ids[q, a:b].tolist()) == set(o_ids[q, a:b].tolist())
        if flags[q]:
            flagged += 1
            mismatched_flagged += not ok_ids
            if exact_d is not None:
                valid = g_ids[q] >= 0
                assert len(set(g_ids[q][valid].tolist())) == int(valid.sum())
                ex = exact_d(q, g_ids[q][valid])
                assert np.all(np.abs(g_d[q][valid] - ex) <= RTOL * ex + atol)
                assert np.all(np.diff(g_d[q][valid]) >= 0)
            ov = len(set(g_ids[q].tolist()) & set(o_ids[q].tolist()))
            assert ov >= int(np.ceil(0.9 * int((o_ids[q] >= 0).sum()))), f"query {q}: overlap {ov} of {K}"
            continue
        assert ok_ids, f"query {q}: ids differ\n gpu {g_ids[q]}\n orc {o_ids[q]}\n gd {g_d[q]}\n od {o_d[q]}"
        fin = np.isfinite(o_d[q])
        assert np.array_equal(fin, np.isfinite(g_d[q])), f"query {q}: filled slots differ"
        err = np.abs(g_d[q][fin] - o_d[q][fin])
        assert np.all(err <= RTOL * o_d[q][fin] + atol), f"query {q}: distance error {err.max()}"
    assert flagged <= max(2, max_flagged_frac * nq), f"{flagged} of {nq} queries flagged as near-ties"
    return {"flagged": flagged, "flagged_mismatched": mismatched_flagged}
