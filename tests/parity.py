"""Comparison of CUDA-path results with the FP64 oracle.

The oracle runs every search three times (``Oracle.search_bracket``): as the
method, and with every threshold decision moved a relative BRACKET_TOL
towards pruning and towards keeping.  The CUDA path computes in FP32: its
rotated vectors are within ROT_TOL of the exact ones (relative to the
vector's norm, checked by test_rotation_parity), so its partial distances
near a threshold carry relative errors of a few 1e-6 on the workloads here,
below BRACKET_TOL.  Tolerance (used by every parity test):

  * stable queries (the three oracle runs agree on the results strictly
    below the query's boundary kth / (1 + 2 BRACKET_TOL), and the probe order
    has no near-tie): those ids equal, position by position (within a run of
    results whose oracle distances agree to BRACKET_TOL only the set must
    match: their order is decided by rounding); the remaining places, at the
    K-th distance, hold distinct other candidates whose exact distances lie
    within the bracket of the K-th (where several candidates tie at the K-th
    place, any of them is a correct result).  Distances within RTOL = 1e-5
    relative of the exact ones, with no absolute term.
  * unstable queries: at most max_unstable_frac of the batch (default 10%),
    each validated instead: ids distinct and from the database, distances
    within RTOL of the exact ones for those ids, ascending, and at least 90%
    of the oracle's ids present.
  * work counters (compare_stats): candidates scanned equal for every query;
    dims used, accepted and pruned equal for every query whose three oracle
    runs count the same.
"""
from __future__ import annotations

import numpy as np

import oracle

RTOL = 1e-5
ROT_TOL = 2e-6
BRACKET_TOL = oracle.BRACKET_TOL


def _runs(d, tol=BRACKET_TOL):
    """Split positions into runs of near-equal distances."""
    runs, start = [], 0
    for i in range(1, len(d) + 1):
        if i == len(d) or not (np.isfinite(d[i]) and np.isfinite(d[i - 1])
                               and abs(d[i] - d[i - 1]) <= tol * max(abs(d[i]), abs(d[i - 1]))):
            runs.append((start, i))
            start = i
    return runs


def same_ids(g, o, od):
    """ids equal position by position, near-equal distance runs as sets."""
    for a, b in _runs(od):
        if b - a == 1:
            if g[a] != o[a]:
                return False
        elif set(g[a:b].tolist()) != set(o[a:b].tolist()):
            return False
    return True


def compare(g_ids, g_d, o, exact_d=None, max_unstable_frac=0.1, same_probe=None):
    """Assert GPU results (g_*) match the oracle's bracketed search o =
    (ids, dists, stats, flags, stable, stats_stable, boundary[, same_probe]).
    exact_d(q, ids) -> FP64 distances of the given ids (needed when a result
    reaches its boundary, and to validate unstable queries).  same_probe[q]:
    the GPU probed the oracle's lists in the oracle's order (then the scan had
    the same input and the probe order's near-ties do not matter); without
    it, a near-tie in the oracle's probe order (flag 8) makes a query
    unstable.  Returns a summary."""
    o_ids, o_d, boundary = o[0], o[1], o[6]
    if same_probe is None and len(o) > 7:
        same_probe = o[7]
    stable = o[4] & (same_probe if same_probe is not None else (o[3] & 8) == 0)
    nq, K = o_ids.shape
    unstable, mismatched_unstable, at_boundary = 0, 0, 0
    for q in range(nq):
        valid = g_ids[q] >= 0
        assert len(set(g_ids[q][valid].tolist())) == int(valid.sum()), f"query {q}: repeated id"
        assert np.all(np.diff(g_d[q][valid]) >= 0), f"query {q}: not ascending"
        assert np.array_equal(valid, o_ids[q] >= 0), f"query {q}: filled slots differ"
        if not stable[q]:
            unstable += 1
            mismatched_unstable += not same_ids(g_ids[q], o_ids[q], o_d[q])
            if exact_d is not None:
                ex = exact_d(q, g_ids[q][valid])
                assert np.all(np.abs(g_d[q][valid] - ex) <= RTOL * ex), f"query {q}: inexact distance"
            ov = len(set(g_ids[q].tolist()) & set(o_ids[q].tolist()))
            assert ov >= int(np.ceil(0.9 * int(valid.sum()))), f"query {q}: overlap {ov} of {K}"
            continue
        j = int((o_d[q] < boundary[q]).sum())
        assert same_ids(g_ids[q][:j], o_ids[q][:j], o_d[q][:j]), \
            f"query {q}: ids differ\n gpu {g_ids[q]}\n orc {o_ids[q]}\n gd {g_d[q]}\n od {o_d[q]}"
        err = np.abs(g_d[q][:j] - o_d[q][:j])
        assert np.all(err <= RTOL * o_d[q][:j]), f"query {q}: distance error {err.max()} (relative " \
                                                 f"{(err / np.maximum(o_d[q][:j], 1e-300)).max():.2e})"
        if j < K and valid[j:].any():
            # the places at the K-th distance: other candidates tied with it within the bracket
            at_boundary += 1
            tail = g_ids[q][j:][valid[j:]]
            assert not set(tail.tolist()) & set(g_ids[q][:j].tolist())
            assert exact_d is not None, "a result reaches its boundary: exact_d needed"
            ex = exact_d(q, tail)
            kth = o_d[q][K - 1]
            assert np.all(ex >= boundary[q] / (1.0 + 2.0 * BRACKET_TOL)) and np.all(ex <= kth * (1.0 + 2.0 * BRACKET_TOL)), \
                f"query {q}: boundary ids {tail} at {ex}, K-th {kth}"
            assert np.all(np.abs(g_d[q][j:][valid[j:]] - ex) <= RTOL * ex), f"query {q}: inexact boundary distance"
    assert unstable <= max(1, int(max_unstable_frac * nq)), f"{unstable} of {nq} queries unstable"
    return {"unstable": unstable, "unstable_mismatched": mismatched_unstable, "at_boundary": at_boundary,
            "queries": nq}


def compare_stats(g_st, o):
    """Work counters of the GPU (candidates, dims used, accepted, pruned)
    against the oracle's: candidates everywhere, the rest where the
    oracle's three bracket runs count the same."""
    o_st, sstable = o[2], o[5]
    assert np.array_equal(g_st[:, 0], o_st[:, 0]), "candidates scanned differ"
    assert np.array_equal(g_st[sstable, 1:], o_st[sstable, 1:]), "work counters differ on bracket-stable queries"
    return int(sstable.sum())
