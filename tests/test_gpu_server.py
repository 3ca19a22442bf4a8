"""The continuous-batching request server (GPU only).

Requests with mixed K and nprobe are submitted back to back; the server
batches compatible ones, runs batches on several streams at once, and every
request's result must equal what a direct dade_query gives for that request
alone, bit for bit.  The same request is also served alone and in the mix.
"""
import numpy as np
import pytest

from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()
    base, queries, _ = synth.make("c2_mix_1m_d128", n=200000, nq=600)
    ix = dade.Index(torch.from_numpy(base).cuda(), 819, kmeans_iters=3, seed=3, eps_pairs=20000, tail_from=32)
    return ix, queries


def _direct(ix, q, k, nprobe, **opts):
    ids = np.empty((q.shape[0], k), np.int64)
    d = np.empty((q.shape[0], k), np.float32)
    ix.query(np.ascontiguousarray(q), k, nprobe, 0.1, 32, ids, d, **opts)
    return ids, d


@pytest.mark.parametrize("opts", [dict(tile=256), dict(tile=256, schedule=dade.SCHED_SEEDED, seed_lists=2,
                                                        flags=dade.FLAG_QUERY_ORDER | dade.FLAG_ROW_TAIL)])
def test_results_alone_and_in_the_mix(index, opts):
    ix, queries = index
    rng = np.random.default_rng(11)
    srv = dade.Server(ix, slots=4, max_batch=256, max_k=100, max_nprobe=64, **opts)
    reqs = []
    start = 0
    for _ in range(48):
        nq = int(rng.integers(1, 24))
        if start + nq > queries.shape[0]:
            start = 0
        reqs.append((queries[start:start + nq], int(rng.choice([1, 10, 100])), int(rng.choice([16, 32, 64]))))
        start += nq
    probe_req = reqs[7]
    # alone
    t = srv.submit(probe_req[0], probe_req[1], probe_req[2])
    alone_ids, alone_d, _ = srv.result(t)
    # in the mix: everything back to back
    tickets = [srv.submit(q, k, npr) for q, k, npr in reqs]
    got = [srv.result(t) for t in tickets]
    st = srv.stats()
    srv.close()
    for (q, k, npr), (ids, d, lat) in zip(reqs, got):
        e_ids, e_d = _direct(ix, q, k, npr, **opts)
        assert np.array_equal(ids, e_ids) and np.array_equal(d.view(np.uint32), e_d.view(np.uint32))
        assert lat > 0
    assert np.array_equal(got[7][0], alone_ids) and np.array_equal(got[7][1].view(np.uint32), alone_d.view(np.uint32))
    assert st["requests_done"] == st["requests"] == 49
    assert st["batches"] < 49                # compatible requests were batched together
    assert st["max_inflight"] >= 2           # batches overlapped on the GPU


def test_rejections(index):
    ix, queries = index
    srv = dade.Server(ix, slots=2, max_batch=8, max_k=10, max_nprobe=16)
    for q, k, npr in ((queries[:9], 5, 8), (queries[:2], 11, 8), (queries[:2], 5, 17)):
        with pytest.raises(dade.DadeError) as e:
            srv.submit(q, k, npr)
        assert e.value.status == dade.EINVAL
    with pytest.raises(dade.DadeError) as e:
        dade.Server(ix, slots=4, max_batch=1024, max_k=100, max_nprobe=64, device_budget=1024)
    assert e.value.status == dade.ENOMEM
    srv.close()
