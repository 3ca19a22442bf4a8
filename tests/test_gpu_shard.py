"""The index split by inverted lists, on one GPU (GPU only).

The shards of one index are made on the same GPU (dade_index_subset), each
runs the whole query batch, and dade_merge_shards keeps the K nearest of
their [G, nq, K] results (the layout an all-gather delivers); nothing waits
on another shard, so one GPU runs them one after the other.
* A shard holds exactly its lists: its exported rotated vectors are the
  full index's for its lists' members and zero elsewhere.
* Each shard's search equals the oracle's search over the rows of its lists
  (bracketed parity), and options that leave results unchanged on the full
  index (the BF16 prefilter and the row-major tail, the tensor-core
  prefilter of the row rounds) leave them unchanged on a shard: its copies
  and its TMA descriptor were rebuilt for its own packing.
* The merge equals the K nearest by (distance, id) of the shards' rows,
  bit for bit, also with empty places; in FD mode the merged result equals
  the unsharded search bit for bit; in DADE mode every position is at least
  as near as the unsharded result's (a shard's threshold is never below the
  unsharded one at the same point of the scan).
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K, NPROBE, ALPHA, DD = 10, 6, 0.1, 32


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()
    w = synth.Workload("shard160", 12000, 160, 200, 1.0, 12, 0.0, 2.0, 1.0, False, False, 12, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    assign = synth.component_lists(labels, 36)
    pairs = synth.eps_pairs(w.n, 3000)
    ix = dade.Index(torch.from_numpy(base).cuda(), 36, assign=assign, pairs=pairs, lead_format=dade.LEAD_BF16,
                    lead_dims=64, tail_from=32)
    orc = oracle.Index(base, 36, assign=assign, pairs=pairs)
    return base, queries, assign, ix, orc


def _query(ix, q, **kw):
    ids = torch.empty(q.shape[0], K, dtype=torch.int64, device="cuda")
    d = torch.empty(q.shape[0], K, dtype=torch.float32, device="cuda")
    ix.query(q, K, NPROBE, ALPHA, DD, ids, d, **kw)
    ix.sync()
    return ids, d


def _np_merge(ids, d):
    g, nq, k = ids.shape
    out_i, out_d = np.empty((nq, k), np.int64), np.empty((nq, k), np.float32)
    for q in range(nq):
        keys = sorted(zip(d[:, q].ravel().tolist(), ids[:, q].ravel().tolist(), np.repeat(np.arange(g), k).tolist()),
                      key=lambda t: (t[0], t[1] if t[1] >= 0 else 1 << 62, t[2]))
        out_d[q] = [t[0] for t in keys[:k]]
        out_i[q] = [t[1] for t in keys[:k]]
    return out_i, out_d


@pytest.mark.parametrize("g", [2, 3])
def test_shards_hold_their_lists(case, g):
    base, queries, assign, ix, orc = case
    owner = dade.shard_lists(ix.list_sizes(), g)
    full = ix.export(dade.FIELD_ROTATED)
    for s in range(g):
        sub = ix.subset(owner, s)
        rot = sub.export(dade.FIELD_ROTATED)
        mine = owner[assign] == s
        assert np.array_equal(rot[mine], full[mine]) and not rot[~mine].any()
        assert np.array_equal(sub.export(dade.FIELD_CENTROIDS), ix.export(dade.FIELD_CENTROIDS))
        assert np.array_equal(sub.export(dade.FIELD_RHO), ix.export(dade.FIELD_RHO))
        with pytest.raises(dade.DadeError):
            sub.subset(owner, 0)
        sub.close()


@pytest.mark.parametrize("g", [2, 3])
def test_sharded_search(case, g):
    base, queries, assign, ix, orc = case
    q = torch.from_numpy(queries).cuda()
    owner = dade.shard_lists(ix.list_sizes(), g)
    subs = [ix.subset(owner, s) for s in range(g)]
    Qr = orc.rotate(queries)
    eps = orc.eps(ALPHA, DD)
    for mode, flags_alt in ((dade.MODE_FD, 0), (dade.MODE_DADE, dade.FLAG_LEAD | dade.FLAG_ROW_TAIL)):
        kw = dict(mode=mode, tile=64)
        per = [_query(s, q, **kw) for s in subs]
        for s, (si, sd) in enumerate(per):
            # the same shard with its lead and tail copies: the same bits
            if flags_alt:
                ai, ad = _query(subs[s], q, flags=flags_alt, **kw)
                assert torch.equal(ai, si) and torch.equal(ad.view(torch.int32), sd.view(torch.int32))
            # against the oracle's search over the shard's rows (ids mapped back)
            rows = np.flatnonzero(owner[assign] == s)
            o = orc.o.search_bracket(orc.Xr[rows], orc.assign[rows], orc.cent, orc.lam, Qr, K, NPROBE, DD,
                                     eps if mode == dade.MODE_DADE else None, oracle.TILE, 64)
            oi = np.where(o[0] >= 0, rows[np.maximum(o[0], 0)], -1)

            def exact_d(qi, sel):
                return ((base[sel].astype(np.float64) - queries[qi].astype(np.float64)) ** 2).sum(-1)

            parity.compare(si.cpu().numpy(), sd.cpu().numpy(), (oi,) + tuple(o[1:]), exact_d)
        gi = torch.stack([p[0] for p in per])
        gd = torch.stack([p[1] for p in per])
        mi = torch.empty(q.shape[0], K, dtype=torch.int64, device="cuda")
        md = torch.empty(q.shape[0], K, dtype=torch.float32, device="cuda")
        dade.merge_shards(gi, gd, mi, md)
        torch.cuda.synchronize()
        wi, wd = _np_merge(gi.cpu().numpy(), gd.cpu().numpy())
        assert np.array_equal(mi.cpu().numpy(), wi) and np.array_equal(md.cpu().numpy().view(np.uint32),
                                                                        wd.view(np.uint32))
        ui, ud = _query(ix, q, **kw)
        if mode == dade.MODE_FD:
            assert torch.equal(mi, ui) and torch.equal(md.view(torch.int32), ud.view(torch.int32))
        else:
            assert bool((md <= ud).all())
    for s in subs:
        s.close()


def test_tensor_core_rounds_on_a_shard(case):
    base, queries, assign, ix, orc = case
    q = torch.from_numpy(queries).cuda()
    owner = dade.shard_lists(ix.list_sizes(), 2)
    sub = ix.subset(owner, 1)
    kw = dict(schedule=dade.SCHED_ROUNDS, tile=32)
    fi, fd = _query(sub, q, **kw)
    ti, td = _query(sub, q, flags=dade.FLAG_TC_PREFILTER, **kw)
    assert torch.equal(fi, ti) and torch.equal(fd.view(torch.int32), td.view(torch.int32))
    sub.close()


def test_merge_with_empty_places(case):
    # shard 0 holds 3 results per query, shard 1 none, shard 2 two: K = 4 takes all but one
    nq, k = 5, 4
    ids = torch.full((3, nq, k), -1, dtype=torch.int64)
    d = torch.full((3, nq, k), float("inf"), dtype=torch.float32)
    rng = np.random.default_rng(2)
    for q in range(nq):
        a = np.sort(rng.random(3)).astype(np.float32)
        b = np.sort(rng.random(2)).astype(np.float32)
        ids[0, q, :3] = torch.tensor([10 * q + 1, 10 * q + 2, 10 * q + 3])
        d[0, q, :3] = torch.from_numpy(a)
        ids[2, q, :2] = torch.tensor([10 * q + 4, 10 * q + 5])
        d[2, q, :2] = torch.from_numpy(b)
    d[0, 0, :3] = torch.tensor([0.25, 0.5, 0.75])   # query 0: an equal distance, the lower id first
    d[2, 0, :2] = torch.tensor([0.25, 0.375])
    mi = torch.empty(nq, k, dtype=torch.int64, device="cuda")
    md = torch.empty(nq, k, dtype=torch.float32, device="cuda")
    dade.merge_shards(ids.cuda(), d.cuda(), mi, md)
    torch.cuda.synchronize()
    wi, wd = _np_merge(ids.numpy(), d.numpy())
    assert np.array_equal(mi.cpu().numpy(), wi) and np.array_equal(md.cpu().numpy(), wd)
    # fewer results than K in all: the empty places stay last
    ids1 = ids[:2, :, :].clone()
    d1 = d[:2, :, :].clone()
    dade.merge_shards(ids1.cuda(), d1.cuda(), mi, md)
    torch.cuda.synchronize()
    assert (mi[:, 3] == -1).all() and torch.isinf(md[:, 3]).all()
