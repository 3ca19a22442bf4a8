"""A query step captured into a CUDA graph and replayed (GPU only): every
replay gives what dade_query gives for the queries the bound buffer holds at
launch time."""
import numpy as np
import pytest

from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()
    base, queries, _ = synth.make("c1_gauss_10k_d128", n=8000, nq=192)
    ix = dade.Index(torch.from_numpy(base).cuda(), 48, kmeans_iters=4, seed=5, eps_pairs=4000, tail_from=32)
    return ix, torch.from_numpy(queries).cuda()


def _direct(ix, q, k, nprobe, **kw):
    ids = torch.empty(q.shape[0], k, dtype=torch.int64, device="cuda")
    d = torch.empty(q.shape[0], k, dtype=torch.float32, device="cuda")
    ix.query(q, k, nprobe, 0.1, 32, ids, d, **kw)
    ix.sync()
    return ids.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("kw", [dict(), dict(schedule=dade.SCHED_SEEDED, seed_lists=2,
                                              flags=dade.FLAG_QUERY_ORDER | dade.FLAG_ROW_TAIL),
                                dict(mode=dade.MODE_FD, schedule=dade.SCHED_SEEDED, seed_lists=1)])
def test_graph_replays_match_direct_calls(setup, kw):
    ix, queries = setup
    qa, qb = queries[:96].contiguous(), queries[96:].contiguous()
    buf = qa.clone()
    ids = torch.empty(96, 10, dtype=torch.int64, device="cuda")
    d = torch.empty(96, 10, dtype=torch.float32, device="cuda")
    g = ix.graph(buf, 10, 12, 0.1, 32, ids, d, **kw)
    for src in (qa, qb, qa):
        buf.copy_(src)
        g.launch()
        torch.cuda.synchronize()
        e_ids, e_d = _direct(ix, src, 10, 12, **kw)
        assert np.array_equal(ids.cpu().numpy(), e_ids)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), e_d.view(np.uint32))
    g.close()


def test_graph_needs_device_buffers(setup):
    ix, queries = setup
    host_ids = np.zeros((4, 5), np.int64)
    host_d = np.zeros((4, 5), np.float32)
    with pytest.raises(dade.DadeError) as e:
        ix.graph(queries[:4].contiguous(), 5, 4, 0.1, 32, host_ids, host_d)
    assert e.value.status == dade.EINVAL
