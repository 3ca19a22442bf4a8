"""Failure paths on the GPU, made without a fault (GPU only).

A search option sets the limit of every bounded device-side wait of the
scan kernels, and DADE_FLAG_CHECK_TIMEOUT makes the first wait on a copy of
every thread block wait on a device word that nothing sets instead: it runs
out after that limit with the block's first copies in flight.  Every kernel
family (the tile kernel, the kernels specialised for D <= 128, the generic
tile kernel, the seeded passes, the list-major rounds with and without the
tensor-core prefilter) must then record DADE_ETIMEOUT, let its copies land
and leave; dade_sync reports the timeout, and the same index must answer
the next normal search with the results it gave before.  A limit of 1 ns on
real copies (a single poll) may or may not run out; either way the index
still answers.  An allocation hook that refuses a device allocation in the
middle of a build gives DADE_ENOMEM, and a build without it succeeds.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HOOK = C.CFUNCTYPE(C.c_int, C.c_size_t, C.c_void_p)


def _index(name, d):
    w = synth.Workload(name, 12000, d, 300, 1.0, 12, 0.0, 2.0, 1.0, False, False, 12, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    ix = dade.Index(torch.from_numpy(base).cuda(), 12, assign=labels, eps_pairs=3000)
    q = torch.from_numpy(queries).cuda()
    qr = torch.empty_like(q)
    ix.rotate(q, qr)
    pr = torch.empty(q.shape[0], 6, dtype=torch.int32, device="cuda")
    ix.probe(qr, 6, pr)
    ix.sync()
    return ix, qr, pr


@pytest.fixture(scope="module")
def indexes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()
    return {160: _index("fail160", 160), 96: _index("fail96", 96)}


@pytest.fixture(scope="module")
def index(indexes):
    return indexes[160]


def _scan(ix, qr, pr, **kw):
    ids = torch.empty(qr.shape[0], 10, dtype=torch.int64, device="cuda")
    d = torch.empty(qr.shape[0], 10, dtype=torch.float32, device="cuda")
    ix.scan(qr, pr, 10, 0.1, 32, ids, d, **kw)
    return ids, d


POINTS = [(160, dict(schedule=dade.SCHED_TILE, tile=128)),
          (96, dict(schedule=dade.SCHED_TILE, tile=128)),
          (96, dict(schedule=dade.SCHED_TILE, tile=64, flags=dade.FLAG_GENERIC_KERNEL)),
          (160, dict(schedule=dade.SCHED_TILE, tile=64, mode=dade.MODE_FD)),
          (160, dict(schedule=dade.SCHED_PIPELINED, tile=64)),
          (160, dict(schedule=dade.SCHED_SEEDED, seed_lists=2, tile=128)),
          (160, dict(schedule=dade.SCHED_ROUNDS, tile=32)),
          (160, dict(schedule=dade.SCHED_ROUNDS, tile=32, flags=dade.FLAG_TC_PREFILTER))]
NAMES = ["tile", "fast", "generic", "fd", "pipelined", "seeded", "rounds", "rounds-tc"]


def _ref(ix, qr, pr, kw):
    ref = _scan(ix, qr, pr, **kw)
    ix.sync()
    return ref[0].cpu().numpy(), ref[1].cpu().numpy()


def _answers_as_before(ix, qr, pr, kw, ref):
    again = _scan(ix, qr, pr, **kw)
    ix.sync()
    assert np.array_equal(again[0].cpu().numpy(), ref[0])
    assert np.array_equal(again[1].cpu().numpy().view(np.uint32), ref[1].view(np.uint32))


@pytest.mark.parametrize("point", POINTS, ids=NAMES)
def test_wait_on_a_word_nothing_sets_times_out(indexes, point):
    ix, qr, pr = indexes[point[0]]
    kw = point[1]
    ref = _ref(ix, qr, pr, kw)
    _scan(ix, qr, pr, wait_ns=200_000, **dict(kw, flags=kw.get("flags", 0) | dade.FLAG_CHECK_TIMEOUT))
    with pytest.raises(dade.DadeError) as e:
        ix.sync()
    assert e.value.status == dade.ETIMEOUT
    ix.sync()                                      # the error word was cleared
    _answers_as_before(ix, qr, pr, kw, ref)


@pytest.mark.parametrize("point", POINTS, ids=NAMES)
def test_single_poll_limit_leaves_the_index_usable(indexes, point):
    ix, qr, pr = indexes[point[0]]
    kw = point[1]
    ref = _ref(ix, qr, pr, kw)
    _scan(ix, qr, pr, wait_ns=1, **kw)
    try:
        ix.sync()
    except dade.DadeError as e:
        assert e.status == dade.ETIMEOUT, e
    _answers_as_before(ix, qr, pr, kw, ref)
    ids, d = _scan(ix, qr, pr, wait_ns=50_000_000, **kw)   # a limit that does not run out: same bits
    ix.sync()
    assert np.array_equal(ids.cpu().numpy(), ref[0])
    assert np.array_equal(d.cpu().numpy().view(np.uint32), ref[1].view(np.uint32))


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
