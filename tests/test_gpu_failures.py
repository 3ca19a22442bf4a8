"""Failure paths on the GPU, made without a fault (GPU only).

A search option sets the limit of every bounded device-side wait of the
scan kernels.  At 1 ns a wait gives up at its first poll whenever the copy it
waits for has not landed yet, which happens on the tile kernel's first tile
(the copy was issued a moment before): the thread block records
DADE_ETIMEOUT, lets its copies in flight land (bounded), and leaves.
dade_sync must report the timeout, and the same index must then answer a
normal search with the results it gave before.  The list-major kernels wait
for copies issued a tile earlier, so there the limit may or may not run out;
either way the index must still answer.  An allocation hook that refuses a
device allocation in the middle of a build gives DADE_ENOMEM, and a build
without it succeeds.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HOOK = C.CFUNCTYPE(C.c_int, C.c_size_t, C.c_void_p)


@pytest.fixture(scope="module")
def index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()
    w = synth.Workload("fail160", 12000, 160, 300, 1.0, 12, 0.0, 2.0, 1.0, False, False, 12, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    ix = dade.Index(torch.from_numpy(base).cuda(), 12, assign=labels, eps_pairs=3000)
    q = torch.from_numpy(queries).cuda()
    qr = torch.empty_like(q)
    ix.rotate(q, qr)
    pr = torch.empty(q.shape[0], 6, dtype=torch.int32, device="cuda")
    ix.probe(qr, 6, pr)
    ix.sync()
    return ix, qr, pr


def _scan(ix, qr, pr, **kw):
    ids = torch.empty(qr.shape[0], 10, dtype=torch.int64, device="cuda")
    d = torch.empty(qr.shape[0], 10, dtype=torch.float32, device="cuda")
    ix.scan(qr, pr, 10, 0.1, 32, ids, d, **kw)
    return ids, d


POINTS = [dict(schedule=dade.SCHED_TILE, tile=128),
          dict(schedule=dade.SCHED_TILE, tile=64, flags=dade.FLAG_GENERIC_KERNEL),
          dict(schedule=dade.SCHED_SEEDED, seed_lists=2, tile=128),
          dict(schedule=dade.SCHED_ROUNDS, tile=32),
          dict(schedule=dade.SCHED_ROUNDS, tile=32, flags=dade.FLAG_TC_PREFILTER)]


@pytest.mark.parametrize("kw", POINTS, ids=["tile", "generic", "seeded", "rounds", "rounds-tc"])
def test_wait_limit_runs_out_and_the_index_still_answers(index, kw):
    ix, qr, pr = index
    ref = _scan(ix, qr, pr, **kw)
    ix.sync()
    ref = (ref[0].cpu().numpy(), ref[1].cpu().numpy())
    _scan(ix, qr, pr, wait_ns=1, **kw)
    timed_out = False
    try:
        ix.sync()
    except dade.DadeError as e:
        assert e.status == dade.ETIMEOUT, e
        timed_out = True
    if kw["schedule"] != dade.SCHED_ROUNDS:   # the first tile's wait starts right after its copy is issued
        assert timed_out
    again = _scan(ix, qr, pr, **kw)
    ix.sync()
    assert np.array_equal(again[0].cpu().numpy(), ref[0])
    assert np.array_equal(again[1].cpu().numpy().view(np.uint32), ref[1].view(np.uint32))


def test_refused_allocation_mid_build(index):
    calls = []

    @HOOK
    def refuse_third(nbytes, user):
        calls.append(int(nbytes))
        return 1 if len(calls) == 3 else 0

    base = np.random.default_rng(3).standard_normal((4000, 64)).astype(np.float32)
    lib = dade.lib()
    lib.dade_set_alloc_hook(C.cast(refuse_third, C.c_void_p), None)
    try:
        with pytest.raises(dade.DadeError) as e:
            dade.Index(torch.from_numpy(base).cuda(), 16, eps_pairs=1000)
    finally:
        lib.dade_set_alloc_hook(None, None)
    assert e.value.status == dade.ENOMEM and len(calls) == 3
    ix = dade.Index(torch.from_numpy(base).cuda(), 16, eps_pairs=1000)   # the same build, no hook
    assert ix.info.n == 4000
    ix.close()
