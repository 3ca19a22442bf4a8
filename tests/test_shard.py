"""The index split by inverted lists, on the CPU (no GPU).

* dade_shard_lists (host code of the library): every list dealt once,
  deterministic, balanced by rows (greedy longest-first: no shard exceeds
  the mean load by more than the longest list).
* Two gloo ranks run the sharded search with the oracle as each rank's
  search (the rows of the rank's lists, ids mapped back), exchange their
  [nq, K] results with the product's all-gather (``shard.gather_results``)
  and keep the K nearest.  In FD mode the sharded result equals the
  unsharded oracle's exactly.  In DADE mode a shard's threshold is never
  below the unsharded one at the same point of the scan (its tiles are a
  subsequence of the unsharded tiles), so it prunes no more: every position
  of the merged result is at least as near as the unsharded result's.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2411_17229_gb300 import dade, synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_2411_17229_gb300 import build
    build.build()
    return dade.lib()


def test_shard_lists_deals_every_list_once_balanced(lib):
    rng = np.random.default_rng(5)
    rows = np.minimum(rng.zipf(1.3, 2000), 50000).astype(np.int64)
    for g in (1, 2, 3, 8):
        owner = dade.shard_lists(rows, g)
        assert owner.min() >= 0 and owner.max() < g
        load = np.bincount(owner, weights=rows, minlength=g)
        assert load.sum() == rows.sum()
        assert load.max() <= rows.sum() / g + rows.max()
        assert np.array_equal(owner, dade.shard_lists(rows, g))   # every rank gets the same partition


def test_shard_lists_greedy_order_and_ties(lib):
    # longest first, ties by list id; each to the lightest shard, ties by shard id
    owner = dade.shard_lists([5, 7, 5, 1, 0, 7], 2)
    # order: list 1 (7) -> 0, list 5 (7) -> 1, list 0 (5) -> 0, list 2 (5) -> 1, list 3 (1) -> 0, list 4 (0) -> 1
    assert owner.tolist() == [0, 0, 1, 0, 1, 1]


def test_shard_lists_rejects_bad_arguments(lib):
    with pytest.raises(dade.DadeError):
        dade.shard_lists([3, -1], 2)
    with pytest.raises(dade.DadeError):
        dade.shard_lists([3, 1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    w = synth.Workload("shard64", 3000, 64, 40, 1.0, 8, 0.0, 2.0, 1.0, False, False, 8, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    assign = synth.component_lists(labels, 24)
    pairs = synth.eps_pairs(w.n, 2000)
    return base, queries, assign, pairs


def _shard_search(orc, Qr, rows, prune, K, nprobe, eps):
    """The oracle's IVF search over the rows of one shard's lists (global list
    ids, global centroids), ids mapped back to base ids."""
    ids, d, _, _ = orc.o.search(orc.Xr[rows], orc.assign[rows], orc.cent, orc.lam, Qr, K, nprobe, 16,
                                eps if prune else None, oracle.TILE, 32)
    return np.where(ids >= 0, rows[np.maximum(ids, 0)], -1), d


def _merge(ids, d, K):
    """The K nearest by (distance, id) of the shards' results [G, nq, K]."""
    g, nq, _ = ids.shape
    out_i, out_d = np.empty((nq, K), np.int64), np.empty((nq, K))
    for q in range(nq):
        keys = sorted(zip(d[:, q].ravel().tolist(), ids[:, q].ravel().tolist()),
                      key=lambda t: (t[0], t[1] if t[1] >= 0 else 1 << 62))
        out_d[q] = [t[0] for t in keys[:K]]
        out_i[q] = [t[1] for t in keys[:K]]
    return out_i, out_d


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2411_17229_gb300 import shard
    base, queries, assign, pairs = _case()
    orc = oracle.Index(base, 24, assign=assign, pairs=pairs)
    Qr = orc.rotate(queries)
    owner = dade.shard_lists(np.bincount(assign, minlength=24), world)
    rows = np.flatnonzero(owner[assign] == rank)
    K, nprobe = 10, 6
    eps = orc.eps(0.1, 16)
    res = {}
    for mode, prune in (("fd", False), ("dade", True)):
        li, ld = _shard_search(orc, Qr, rows, prune, K, nprobe, eps)
        gi, gd = shard.gather_results(torch.from_numpy(li), torch.from_numpy(ld))
        res[mode] = (gi.numpy(), gd.numpy())
    out[rank] = (owner, res)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sharded_search():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert np.array_equal(res[0][0], res[1][0])               # one partition on every rank
    base, queries, assign, pairs = _case()
    orc = oracle.Index(base, 24, assign=assign, pairs=pairs)
    Qr = orc.rotate(queries)
    owner = res[0][0]
    K, nprobe = 10, 6
    eps = orc.eps(0.1, 16)
    for mode, prune in (("fd", False), ("dade", True)):
        gi, gd = res[0][1][mode]
        assert np.array_equal(gi, res[1][1][mode][0]) and np.array_equal(gd, res[1][1][mode][1])
        # rank order of the gather: rank g's slice is its own shard's search
        for g in range(world):
            li, ld = _shard_search(orc, Qr, np.flatnonzero(owner[assign] == g), prune, K, nprobe, eps)
            assert np.array_equal(gi[g], li) and np.array_equal(gd[g], ld)
        mi, md = _merge(gi, gd, K)
        ui, ud, _, _ = orc.o.search(orc.Xr, orc.assign, orc.cent, orc.lam, Qr, K, nprobe, 16,
                                    eps if prune else None, oracle.TILE, 32)
        if mode == "fd":
            assert np.array_equal(mi, ui) and np.array_equal(md, ud)
        else:
            assert np.all(md <= ud)                   # equal or nearer, position by position
