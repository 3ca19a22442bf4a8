"""The continuous-batching request server and per-query K / nprobe (GPU only).

dade_query_mixed runs queries with their own K and nprobe in one launch; each
query's result must equal dade_query's for that query alone, bit for bit.
Requests with mixed K and nprobe are submitted back to back; the server
batches them (under the tile schedule all of them, in a few large batches;
under the seeded schedule those with equal K and nprobe), runs batches on
several streams at once, and every request's result must equal what a
direct dade_query gives for that request alone, bit for bit.  The same
request is also served alone and in the mix, under the row rounds also with
a list chunk and a tensor-core window passed through.  Cancelled requests complete
with DADE_ECANCELLED and leave the others untouched; with a device budget,
batches are admitted by bytes and a request that cannot fit completes with
DADE_ENOMEM.
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
                                                        flags=dade.FLAG_QUERY_ORDER | dade.FLAG_ROW_TAIL),
                                  dict(tile=16, schedule=dade.SCHED_ROUNDS, flags=dade.FLAG_QUERY_ORDER),
                                  dict(tile=16, schedule=dade.SCHED_ROUNDS, flags=dade.FLAG_TC_PREFILTER,
                                       list_chunk=1024, tc_min_rows=128)],
                         ids=["tile", "seeded", "rounds", "rounds-tc-window"])
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
    if opts.get("schedule", dade.SCHED_TILE) in (dade.SCHED_TILE, dade.SCHED_ROUNDS):
        assert st["batches"] <= 12           # mixed K and nprobe in the same batches
    assert st["max_inflight"] >= 2           # batches overlapped on the GPU


SCHEDULES = {"tile": dict(tile=128), "rounds": dict(tile=16, schedule=dade.SCHED_ROUNDS),
             "rounds-tc": dict(tile=16, schedule=dade.SCHED_ROUNDS, flags=dade.FLAG_TC_PREFILTER)}


@pytest.mark.parametrize("sched", list(SCHEDULES))
@pytest.mark.parametrize("mode", [dade.MODE_DADE, dade.MODE_FD])
def test_query_mixed_equals_each_query_alone(index, mode, sched):
    ix, queries = index
    rng = np.random.default_rng(5)
    q = np.ascontiguousarray(queries[:200])
    ks = rng.choice([1, 10, 37, 100], q.shape[0]).astype(np.int32)
    nps = rng.choice([16, 24, 32, 64], q.shape[0]).astype(np.int32)
    kmax = int(ks.max())
    ids = np.empty((q.shape[0], kmax), np.int64)
    d = np.empty((q.shape[0], kmax), np.float32)
    kw = SCHEDULES[sched]
    ix.query_mixed(q, ks, nps, 0.1, 32, ids, d, mode=mode, **kw)
    for (k, npr) in {(int(a), int(b)) for a, b in zip(ks, nps)}:
        rows = np.flatnonzero((ks == k) & (nps == npr))
        e_ids, e_d = _direct(ix, q[rows], k, npr, mode=mode, **kw)
        assert np.array_equal(ids[rows, :k], e_ids)
        assert np.array_equal(d[rows, :k].view(np.uint32), e_d.view(np.uint32))
        assert (ids[rows, k:] == -1).all() and np.isinf(d[rows, k:]).all()
    # device arrays give the same bits
    kt, nt = torch.from_numpy(ks).cuda(), torch.from_numpy(nps).cuda()
    qd = torch.from_numpy(q).cuda()
    ids2 = torch.empty(q.shape[0], kmax, dtype=torch.int64, device="cuda")
    d2 = torch.empty(q.shape[0], kmax, dtype=torch.float32, device="cuda")
    ix.query_mixed(qd, kt, nt, 0.1, 32, ids2, d2, mode=mode, **kw)
    ix.sync()
    assert np.array_equal(ids2.cpu().numpy(), ids)
    assert np.array_equal(d2.cpu().numpy().view(np.uint32), d.view(np.uint32))
    # another schedule is refused
    o = dade.SearchOpts(schedule=dade.SCHED_SEEDED, seed_lists=2)
    rc = dade.lib().dade_query_mixed(ix.handle, q.ctypes.data, q.shape[0], ks.ctypes.data, nps.ctypes.data, kmax,
                                     int(nps.max()), 0.1, 32, dade.C.byref(o), ids.ctypes.data, d.ctypes.data, None)
    assert rc == dade.EINVAL


def test_server_options_checked(index):
    ix, _ = index
    for bad in (dict(list_chunk=100), dict(list_chunk=32), dict(tc_min_rows=-1)):
        with pytest.raises(dade.DadeError) as e:
            dade.Server(ix, **bad)
        assert e.value.status == dade.EINVAL


def test_cancel(index):
    ix, queries = index
    srv = dade.Server(ix, slots=1, max_batch=8, max_k=10, max_nprobe=32, tile=128)
    tickets = [srv.submit(queries[i:i + 8], 10, 32) for i in range(0, 160, 8)]
    srv.cancel(tickets[-1])                    # still queued behind 19 batches on one slot
    try:
        srv.cancel(tickets[0])                 # admitted first: in flight, unless already done
        first_cancelled = True
    except dade.DadeError as e:
        assert e.status == dade.EINVAL         # it had completed
        first_cancelled = False
    for i, t in enumerate(tickets):
        if i == len(tickets) - 1 or (i == 0 and first_cancelled):
            with pytest.raises(dade.DadeError) as e:
                srv.result(t)
            assert e.value.status == dade.ECANCELLED
        else:
            ids, d, _ = srv.result(t)
            e_ids, e_d = _direct(ix, queries[8 * i:8 * i + 8], 10, 32, tile=128)
            assert np.array_equal(ids, e_ids) and np.array_equal(d.view(np.uint32), e_d.view(np.uint32))
    with pytest.raises(dade.DadeError) as e:
        srv.cancel(tickets[3])                 # completed
    assert e.value.status == dade.EINVAL
    srv.close()


def test_native_replay(index):
    """dade_server_replay submits one-query requests at given times from C++; every request's
    result equals dade_query's for it alone, and the latencies are measured."""
    ix, queries = index
    rng = np.random.default_rng(9)
    n = 300
    picks = rng.integers(0, queries.shape[0], n)
    ks = rng.choice([1, 10, 100], n).astype(np.int32)
    nps = rng.choice([16, 32, 64], n).astype(np.int32)
    arrivals = np.cumsum(rng.exponential(1.0 / 20000, n))
    srv = dade.Server(ix, slots=4, max_batch=1024, max_k=100, max_nprobe=64, tile=128)
    ids, d, lat, t_sub = srv.replay(queries[picks], ks, nps, 0.1, 32, arrivals)
    st = srv.stats()
    srv.close()
    assert (lat > 0).all() and t_sub >= arrivals[-1]
    assert st["requests_done"] == n and st["batches"] < n
    for i in range(0, n, 7):
        e_ids, e_d = _direct(ix, queries[picks[i]:picks[i] + 1], int(ks[i]), int(nps[i]), tile=128)
        assert np.array_equal(ids[i, :ks[i]], e_ids[0])
        assert np.array_equal(d[i, :ks[i]].view(np.uint32), e_d[0].view(np.uint32))


def test_admission_by_bytes(index):
    ix, queries = index
    d, nc = ix.d, ix.n_clusters
    max_batch, max_k = 64, 10
    fixed = max_batch * (d * 4 + max_k * 12)
    per_query = d * 8 + nc * 4 + 32 * 4 + max_k * 12 + d * 8 + 72       # K 10, nprobe 32
    budget = 2 * fixed + 6 * per_query                                   # two slots, six queries in flight
    srv = dade.Server(ix, slots=4, max_batch=max_batch, max_k=max_k, max_nprobe=32, tile=128, device_budget=budget)
    assert srv.stats()["slots"] == 2
    tickets = [srv.submit(queries[i:i + 2], 10, 32) for i in range(0, 80, 2)]
    for i, t in zip(range(0, 80, 2), tickets):
        ids, dd, _ = srv.result(t)
        e_ids, e_d = _direct(ix, queries[i:i + 2], 10, 32, tile=128)
        assert np.array_equal(ids, e_ids) and np.array_equal(dd.view(np.uint32), e_d.view(np.uint32))
    st = srv.stats()
    assert st["queries"] == 80 and st["queries"] / st["batches"] <= 6
    t = srv.submit(queries[:8], 10, 32)                                  # eight queries never fit
    with pytest.raises(dade.DadeError) as e:
        srv.result(t)
    assert e.value.status == dade.ENOMEM
    srv.close()


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
