"""Parity at the benchmark sizes (GPU only).

Each workload is generated at its full size and indexed by both sides with
the same seeded list assignment (every mixture component's members dealt to
lists of their own) and the same eps pairs.  The CUDA path then runs the
whole query batch in the launch configuration the benchmark times (rotate,
probe, scan; the benchmark's schedule, tile, threads, delta_d, alpha and
flags), and a seeded sample of its queries is compared with the oracle's
sampled index element by element, under the tolerance of ``parity.py``: the
oracle brackets every threshold decision, ids must match on every stable
query, and at most a tenth of the sample may be unstable.
Every query of the batch is also checked against properties that hold at
any size: distinct ids in range, ascending distances, and each distance
equal to the FP64 squared distance of the raw vectors (the rotation is an
isometry, Lemma 1).  The serving workload runs through the request server,
with per-request K and nprobe.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_SAMPLE = 24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()


def _build(w, n_pairs, **kw):
    base, queries, labels = synth.make(w)
    assign = synth.component_lists(labels, w.n_clusters)
    pairs = synth.eps_pairs(w.n, n_pairs)
    ix = dade.Index(torch.from_numpy(base).cuda(), w.n_clusters, assign=assign, pairs=pairs, **kw)
    return base, queries, assign, pairs, ix


def _check_properties(base, queries, ids, dists):
    """Any size: ids distinct and in range, ascending, distances exact."""
    nq, K = ids.shape
    valid = ids >= 0
    assert valid.all(), "fewer than K results"
    assert (ids < base.shape[0]).all()
    srt = np.sort(ids, axis=1)
    assert (srt[:, 1:] != srt[:, :-1]).all(), "repeated id in a result"
    assert (np.diff(dists, axis=1) >= 0).all(), "distances not ascending"
    for q0 in range(0, nq, 256):
        q1 = min(nq, q0 + 256)
        diff = base[ids[q0:q1]].astype(np.float64) - queries[q0:q1, None, :].astype(np.float64)
        ex = (diff ** 2).sum(-1)
        err = np.abs(dists[q0:q1].astype(np.float64) - ex)
        assert (err <= parity.RTOL * ex).all(), f"distance error {(err / np.maximum(ex, 1e-300)).max():.2e} relative"


def _scan_batch(ix, queries, K, pt):
    """The benchmark's step: rotate, probe, scan over the whole batch."""
    q = torch.from_numpy(queries).cuda()
    nq = q.shape[0]
    qr = torch.empty_like(q)
    pr = torch.empty(nq, pt["nprobe"], dtype=torch.int32, device="cuda")
    ids = torch.empty(nq, K, dtype=torch.int64, device="cuda")
    d = torch.empty(nq, K, dtype=torch.float32, device="cuda")
    ix.rotate(q, qr)
    ix.probe(qr, pt["nprobe"], pr)
    ix.scan(qr, pr, K, pt["alpha"], pt["delta_d"], ids, d, tile=pt["tile"], threads=pt["threads"],
            schedule=pt["schedule"], seed_lists=pt["seed_lists"], flags=pt["flags"],
            list_chunk=pt.get("list_chunk", 0), tc_min_rows=pt.get("tc_min_rows", 0))
    ix.sync()
    return pr.cpu().numpy(), ids.cpu().numpy(), d.cpu().numpy()


def _run_batch_case(wname, pt, n_pairs, **build_kw):
    w = synth.WORKLOADS[wname]
    base, queries, assign, pairs, ix = _build(w, n_pairs, **build_kw)
    K = w.k
    probe, ids, dists = _scan_batch(ix, queries, K, pt)
    sample = np.sort(np.random.default_rng(17).choice(queries.shape[0], N_SAMPLE, replace=False))
    orc = oracle.SampledIndex(base, assign, w.n_clusters, pairs, queries[sample], pt["nprobe"])
    # the probe (Section 3.4): the oracle's nearest lists, by (distance, list id)
    same = [np.array_equal(probe[s], orc.probe[i]) for i, s in enumerate(sample) if not orc.probe_tie[i]]
    assert all(same)
    same_probe = np.array([np.array_equal(probe[s], orc.probe[i]) for i, s in enumerate(sample)])
    o = _oracle_point(orc, K, pt)

    def exact_d(i, sel):
        return ((base[sel].astype(np.float64) - queries[sample[i]].astype(np.float64)) ** 2).sum(-1)

    summary = parity.compare(ids[sample], dists[sample], o, exact_d, same_probe=same_probe)
    print(f"{wname}: {summary}")
    _check_properties(base, queries, ids, dists)
    ix.close()


def _oracle_point(orc, K, pt):
    """The oracle's bracketed search in the schedule of a benchmark point."""
    if pt["schedule"] == dade.SCHED_ROUNDS:
        return orc.search_bracket(K, pt["nprobe"], pt["delta_d"], pt["alpha"], schedule=oracle.ROW_ROUNDS,
                                  tile=pt["tile"])
    seed = pt["seed_lists"] if pt["schedule"] == dade.SCHED_SEEDED else 0
    return orc.search_bracket(K, pt["nprobe"], pt["delta_d"], pt["alpha"], tile=pt["tile"], seed=seed)


def test_c2_full_size_benchmark_point():
    """1M x 128 integer mixture, 10,000 queries, K = 100, at the benchmark's
    point: nprobe 20, seeded schedule (2 lists), tile 128, delta_d 64,
    alpha 0.98, query order; index with the BF16 lead copy and the row-major
    tail from dim 32, as the benchmark builds it."""
    pt = {"nprobe": 20, "alpha": 0.98, "delta_d": 64, "tile": 128, "threads": 128, "schedule": dade.SCHED_SEEDED,
          "seed_lists": 2, "flags": dade.FLAG_QUERY_ORDER}
    _run_batch_case("c2_mix_1m_d128", pt, 100000, lead_format=dade.LEAD_BF16, lead_dims=64, tail_from=32)


def test_c3_full_size_benchmark_point():
    """1M x 960 mixture, 1,000 queries, K = 10, at the benchmark's point:
    nprobe 24, seeded schedule (2 lists) with the later lists split over
    thread blocks, tile 128, 128 threads, delta_d 16, alpha 0.98."""
    pt = {"nprobe": 24, "alpha": 0.98, "delta_d": 16, "tile": 128, "threads": 128, "schedule": dade.SCHED_SEEDED,
          "seed_lists": 2, "flags": dade.FLAG_SEED_SPLIT}
    _run_batch_case("c3_mix_1m_d960", pt, 20000, lead_format=dade.LEAD_BF16, lead_dims=64, tail_from=32)


def test_c5_full_size_serving():
    """5M x 256 mixture, 8,192 lists, served: 240 single-query requests with
    K in {1, 10, 100} and nprobe in {16, 64, 128} drawn per request, all in
    flight together on the request server (4 slots, batches up to 1,024);
    sampled requests against the oracle with their own K and nprobe."""
    w = synth.WORKLOADS["c5_mix_5m_d256"]
    base, queries, assign, pairs, ix = _build(w, 20000, tail_from=32)
    rng = np.random.default_rng(23)
    n_req = 240
    picks = rng.choice(queries.shape[0], n_req, replace=False)
    ks = rng.choice([1, 10, 100], n_req)
    nps = rng.choice([16, 64, 128], n_req)
    alpha, delta_d = 0.1, 32
    srv = dade.Server(ix, slots=4, max_batch=1024, max_k=100, max_nprobe=128, tile=128, threads=128)
    tickets = [srv.submit(queries[picks[i]:picks[i] + 1], int(ks[i]), int(nps[i]), alpha, delta_d)
               for i in range(n_req)]
    res = [srv.result(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["requests_done"] == n_req and st["batches"] < n_req
    sample = np.sort(rng.choice(n_req, N_SAMPLE, replace=False))
    orc = oracle.SampledIndex(base, assign, w.n_clusters, pairs, queries[picks[sample]], 128)
    # the lists the server's batches probed for the sampled requests: each query's probe
    # depends on that query alone, so probing it on its own gives the same lists
    qs = torch.from_numpy(queries[picks[sample]]).cuda()
    qsr = torch.empty_like(qs)
    pg = torch.empty(len(sample), 128, dtype=torch.int32, device="cuda")
    ix.rotate(qs, qsr)
    ix.probe(qsr, 128, pg)
    ix.sync()
    pg = pg.cpu().numpy()
    unstable = 0
    for K, nprobe in sorted({(int(ks[i]), int(nps[i])) for i in sample}):
        rows = [j for j, i in enumerate(sample) if ks[i] == K and nps[i] == nprobe]
        o = orc.search_bracket(K, nprobe, delta_d, alpha, tile=128)
        g_ids = np.stack([res[sample[j]][0][0] for j in rows])
        g_d = np.stack([res[sample[j]][1][0] for j in rows])

        def exact_d(i, sel, rows=rows):
            q = queries[picks[sample[rows[i]]]].astype(np.float64)
            return ((base[sel].astype(np.float64) - q) ** 2).sum(-1)

        sp = np.array([np.array_equal(pg[j, :nprobe], orc.probe[j, :nprobe]) for j in rows])
        summary = parity.compare(g_ids, g_d, tuple(x[rows] for x in o), exact_d, max_unstable_frac=1.0,
                                 same_probe=sp)
        unstable += summary["unstable"]
    assert unstable <= max(1, N_SAMPLE // 10), unstable
    for i in range(n_req):
        _check_properties(base, queries[picks[i]:picks[i] + 1], res[i][0], res[i][1])
    ix.close()


def test_c4_full_size_benchmark_point():
    """10M x 768 normalised mixture over 16,384 components with Zipf(1.1)
    weights (largest list 1.47M, median 72), lists = the generating
    components, 10,000 queries, K = 10, at the benchmark's point: row rounds
    from 16 rows, work items of 1,024 rows, delta_d 32, alpha 0.98, nprobe 12,
    256 threads, row-major tail from dim 32, the tensor-core prefilter for
    windows of 16,384 rows and more; index with the FP8 leading-block copy.  At full size the tensor-core prefilter
    must return the FP32 list-major path's results bit for bit, and the FP8
    prefilter (which runs the rounds query-major on the tile kernel) the
    same kernel's FP32 results."""
    w = synth.WORKLOADS["c4_zipf_10m_d768"]
    base, queries, labels = synth.make(w)
    pairs = synth.eps_pairs(w.n, 20000)
    ix = dade.Index(torch.from_numpy(base).cuda(), w.n_clusters, assign=labels, pairs=pairs,
                    lead_format=dade.LEAD_FP8, lead_dims=64, tail_from=32)
    pt = {"nprobe": 12, "alpha": 0.98, "delta_d": 32, "tile": 16, "threads": 256, "schedule": dade.SCHED_ROUNDS,
          "seed_lists": 0, "list_chunk": 1024, "tc_min_rows": 16384,
          "flags": dade.FLAG_ROW_TAIL | dade.FLAG_TC_PREFILTER}
    probe, ids, dists = _scan_batch(ix, queries, w.k, pt)
    _, idsf, distsf = _scan_batch(ix, queries, w.k, dict(pt, flags=pt["flags"] & ~dade.FLAG_TC_PREFILTER))
    assert np.array_equal(ids, idsf) and np.array_equal(dists.view(np.uint32), distsf.view(np.uint32))
    split = dict(pt, flags=(pt["flags"] & ~dade.FLAG_TC_PREFILTER) | dade.FLAG_SEED_SPLIT)
    _, idss, distss = _scan_batch(ix, queries, w.k, split)
    _, ids8, dists8 = _scan_batch(ix, queries, w.k, dict(split, flags=split["flags"] | dade.FLAG_LEAD))
    assert np.array_equal(idss, ids8) and np.array_equal(distss.view(np.uint32), dists8.view(np.uint32))
    sample = np.sort(np.random.default_rng(17).choice(queries.shape[0], N_SAMPLE, replace=False))
    orc = oracle.SampledIndex(base, labels, w.n_clusters, pairs, queries[sample], pt["nprobe"])
    same = [np.array_equal(probe[s], orc.probe[i]) for i, s in enumerate(sample) if not orc.probe_tie[i]]
    assert all(same)
    same_probe = np.array([np.array_equal(probe[s], orc.probe[i]) for i, s in enumerate(sample)])
    o = _oracle_point(orc, w.k, pt)

    def exact_d(i, sel):
        return ((base[sel].astype(np.float64) - queries[sample[i]].astype(np.float64)) ** 2).sum(-1)

    summary = parity.compare(ids[sample], dists[sample], o, exact_d, same_probe=same_probe)
    print(f"c4: {summary}")
    summary = parity.compare(idss[sample], distss[sample], o, exact_d, same_probe=same_probe)
    print(f"c4 (rounds on the tile kernel): {summary}")
    _check_properties(base, queries, ids, dists)
    ix.close()
