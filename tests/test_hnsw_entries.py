"""Why HNSW* searches need entry objects near the query (CPU, oracle only).

The layer-0 graph of the reading in or_hnsw_graph links an object only to
objects near it, so on data of well-separated components it has no links
between components: a beam search from one medoid stays in the medoid's
component.  Entry objects taken from the query's nearest coarse list (the
role HNSW's upper layers play; the benchmark takes them from the IVF index)
reach the query's component and give the exact neighbours.
"""
import numpy as np

import oracle


def test_separated_components_need_near_entries(orc):
    rng = np.random.default_rng(61)
    centers = rng.standard_normal((16, 32)) * 12.0
    lab = rng.integers(0, 16, 3000)
    X = centers[lab] + rng.standard_normal((3000, 32))
    qlab = rng.integers(0, 16, 60)
    Q = centers[qlab] + rng.standard_normal((60, 32))
    nbr, _, _ = orc.hnsw_graph(X, 32, 8, 16)
    med = int(np.argmin(((X - X.mean(0)) ** 2).sum(1)))
    seen, todo = {med}, [med]
    while todo:
        for v in nbr[todo.pop()]:
            if v >= 0 and int(v) not in seen:
                seen.add(int(v))
                todo.append(int(v))
    assert len(seen) < 3000 // 4                          # the medoid's component and few more
    gt, _ = orc.exact_knn(X.astype(np.float32), Q.astype(np.float32), 10)
    # entries: the 4 nearest members of the component whose center is nearest the query
    near = np.argmin(((Q[:, None, :] - centers[None]) ** 2).sum(-1), 1)
    ent = np.stack([np.flatnonzero(lab == c)[np.argsort(((X[lab == c] - Q[i]) ** 2).sum(1), kind="stable")[:4]]
                    for i, c in enumerate(near)])
    lam = np.ones(32)
    a = orc.hnsw_search(X, nbr, lam, Q, [med], 10, 32, 16, None, oracle.HNSW_NODE, max_visits=3072)
    b = orc.hnsw_search(X, nbr, lam, Q, ent, 10, 32, 16, None, oracle.HNSW_NODE, max_visits=3072)
    rec = lambda r: np.mean([len(set(x) & set(y)) / 10 for x, y in zip(r[0], gt)])  # noqa: E731
    assert rec(a) <= 0.25
    assert rec(b) >= 0.95
