"""The library autotuner (dade_autotune), GPU only.

A tuned point must reach the recall target on the tuning queries and, up to
the sampling error of 1,000 queries, on held-out queries of the same
distribution; a second call with the same key returns the cached point
without running a search; the JSON-lines cache file is written and read
back (a line for another recall target, written by hand with the file's own
key, is returned as is); bad arguments are refused before any search.
"""
import numpy as np
import pytest

from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = 10


def _exact(base, queries, k):
    """Exact K nearest ids (FP64 on the GPU; measurement only)."""
    xb = torch.from_numpy(base).cuda().double()
    out = []
    for s in range(0, queries.shape[0], 256):
        qq = torch.from_numpy(queries[s:s + 256]).cuda().double()
        d = (qq * qq).sum(1, keepdim=True) - 2.0 * qq @ xb.T + (xb * xb).sum(1)[None, :]
        out.append(torch.topk(d, k, dim=1, largest=False).indices.cpu().numpy())
    return np.concatenate(out).astype(np.int64)


def _recall(ids, gt):
    return float(np.mean([len(set(a.tolist()) & set(b.tolist())) / gt.shape[1] for a, b in zip(ids, gt)]))


@pytest.fixture(scope="module", params=[128, 96], ids=["d128", "d96"])
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()
    d = request.param
    w = synth.Workload(f"tune{d}", 40000, d, 2000, 1.0, 16, 0.0, 2.0, 1.0, False, False, 64, (8,), K, (32,), 0.1)
    base, queries, _ = synth.make(w)
    ix = dade.Index(torch.from_numpy(base).cuda(), 64, eps_pairs=5000, tail_from=32)
    gt = _exact(base, queries, K)
    return ix, queries, gt


def test_tuned_point_meets_the_target_and_is_cached(case, tmp_path):
    ix, queries, gt = case
    qt, qh = queries[:1000], queries[1000:]
    path = tmp_path / "tune.jsonl"
    r = ix.autotune(qt, K, gt[:1000], recall_target=0.9, cache_path=path)
    assert not r["from_cache"] and r["points_tried"] > 0 and r["recall"] >= 0.9
    alphas = np.float32([0.98, 0.95, 0.9, 0.8, 0.6, 0.4, 0.2, 0.1, 0.05])
    assert r["delta_d"] in (16, 32, 64) and np.float32(r["alpha"]) in alphas and r["ms"] > 0
    # held-out queries at the tuned point, through dade_query
    q = torch.from_numpy(qh).cuda()
    ids = torch.empty(q.shape[0], K, dtype=torch.int64, device="cuda")
    dists = torch.empty(q.shape[0], K, dtype=torch.float32, device="cuda")
    ix.query(q, K, r["nprobe"], r["alpha"], r["delta_d"], ids, dists, **r["point"])
    ix.sync()
    assert _recall(ids.cpu().numpy(), gt[1000:]) >= 0.9 - 0.01
    # the same key again: the process cache, no search
    r2 = ix.autotune(qt, K, gt[:1000], recall_target=0.9, cache_path=path)
    assert r2["from_cache"] and r2["points_tried"] == 0
    assert (r2["nprobe"], r2["delta_d"], r2["alpha"], r2["point"]) == (r["nprobe"], r["delta_d"], r["alpha"],
                                                                        r["point"])
    # the file: one line for this key; a hand-written line for target 0.85 is read back as is
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and '"nprobe": %d' % r["nprobe"] in lines[0]
    key = lines[0].split('"key": "')[1].split('"')[0]
    assert "/r0.9000/" in key
    crafted = lines[0].replace(key, key.replace("/r0.9000/", "/r0.8500/")).replace(
        '"nprobe": %d' % r["nprobe"], '"nprobe": 7')
    path.write_text(lines[0] + "\n" + crafted + "\n")
    r3 = ix.autotune(qt, K, gt[:1000], recall_target=0.85, cache_path=path)
    assert r3["from_cache"] and r3["nprobe"] == 7 and r3["delta_d"] == r["delta_d"]


def test_autotune_refuses_bad_arguments(case):
    ix, queries, gt = case
    with pytest.raises(dade.DadeError) as e:
        ix.autotune(queries[:100], K, gt[:100], recall_target=0.9, ladder=[8, 4])
    assert e.value.status == dade.EINVAL
    with pytest.raises(dade.DadeError) as e:
        ix.autotune(queries[:100], K, gt[:100], recall_target=1.5)
    assert e.value.status == dade.EINVAL
    # a target the ladder cannot reach: one list probed
    with pytest.raises(dade.DadeError) as e:
        ix.autotune(queries[:100], K, gt[:100], recall_target=1.0, ladder=[1], force=True)
    assert e.value.status == dade.EUNSUPPORTED
