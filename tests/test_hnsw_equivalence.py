"""The bounded form of the HNSW* beam search (CPU).

Section 3.4's search keeps an unbounded search set S beside the result set
R.  The GPU kernel keeps only R (the ef nearest, ascending by (squared
distance, id)) with an "expanded" mark per entry, and pops R's nearest
unexpanded entry: an object that left R is farther than all of R, so the
method pops it only after R has no unexpanded entry left, and its stop
compare then ends the search.  This test restates that bounded form in plain
Python -- FP32 DCOs in dimension order, threshold read once per expanded
object, accepted neighbours entering R in slot order -- and requires the
oracle's literal S/R search (FP32 arithmetic, NODE schedule) to return the
same ids, distance bits and work counters on every query, with and without
a visit budget and with several entry objects.
"""
import numpy as np
import pytest

import oracle
import pins

f32 = np.float32


def _dco(q, x, D, delta_d, coef, r2):
    P, d, j = f32(0), 0, 0
    while True:
        dn = min(d + delta_d, D)
        for k in range(d, dn):
            t = f32(q[k] - x[k])
            P = f32(P + f32(t * t))
        d = dn
        if d >= D:
            return bool(P <= r2), P, D
        if coef is not None and P > f32(coef[j] * r2):
            return False, None, d
        j += 1


def _bounded(X, nbr, q, K, ef, delta_d, coef, entry, max_visits):
    n, D = X.shape
    R, vis, st = [], set(), [0, 0, 0, 0, 0]     # R: [distance, id, expanded]

    def admit(acc):
        for p, e in acc:
            pos = sum(1 for r in R if r[0] < p or (r[0] == p and r[1] < e))
            if pos < ef:
                R.insert(pos, [p, e, False])
                del R[ef:]

    def visit(e, r2, acc):
        vis.add(e)
        ok, p, dims = _dco(q, X[e], D, delta_d, coef, r2)
        st[0] += 1
        st[1] += dims
        if ok:
            st[2] += 1
            acc.append((p, e))
        elif dims < D:
            st[3] += 1

    acc = []
    for e in entry:
        if 0 <= e < n and e not in vis:
            visit(e, f32(np.inf), acc)
    admit(acc)
    while st[0] < max_visits:
        c = next((r for r in R if not r[2]), None)
        if c is None:
            break
        r2 = R[ef - 1][0] if len(R) == ef else f32(np.inf)
        c[2] = True
        st[4] += 1
        acc = []
        for e in nbr[c[1]]:
            if 0 <= e < n and e not in vis:
                visit(int(e), r2, acc)
        admit(acc)
    ids = [R[s][1] if s < len(R) else -1 for s in range(K)]
    ds = [R[s][0] if s < len(R) else f32(np.inf) for s in range(K)]
    return ids, np.array(ds, np.float32), st


@pytest.mark.parametrize("n,D,ef,K,delta_d,budget,n_entry", [(500, 24, 16, 5, 16, 0, 1), (600, 40, 24, 10, 16, 70, 1),
                                                             (500, 48, 12, 10, 32, 0, 3)])
def test_bounded_search_is_the_method(orc, n, D, ef, K, delta_d, budget, n_entry):
    X, Q = pins._hnsw_setup(orc, n=n, D=D, seed=500 + n + D)
    Q = Q[:12]
    nbr, _, _ = orc.hnsw_graph(X, 24, 8, 16)
    mu, W, lam = orc.pca(X.astype(np.float32))
    Xr = orc.rotate(X.astype(np.float32), mu, W).astype(np.float32)
    Qr = orc.rotate(Q.astype(np.float32), mu, W).astype(np.float32)
    eps = pins._eps_for(orc, Xr.astype(np.float64), lam, delta_d, 0.1)
    coef = oracle.coef_f32(lam, eps, D, delta_d)
    entry = np.random.default_rng(n).integers(0, n, (Q.shape[0], n_entry))
    mv = budget or min(n, 64 * ef + 1024)
    ref = orc.hnsw_search(Xr, nbr, lam, Qr, entry, K, ef, delta_d, None, oracle.HNSW_NODE, max_visits=mv,
                          coef32=coef)
    assert ref[2][:, 3].sum() > 0
    for i in range(Q.shape[0]):
        ids, ds, st = _bounded(Xr, nbr, Qr[i], K, ef, delta_d, coef, entry[i], mv)
        assert ids == ref[0][i].tolist()
        assert np.array_equal(ds.view(np.uint32), ref[1][i].astype(np.float32).view(np.uint32))
        assert st == ref[2][i].tolist()
