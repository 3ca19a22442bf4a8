"""dade_probe_noalloc against dade_probe (GPU only; collected last on purpose).

dade_probe_noalloc serves callers that must not allocate device memory (for
example a serving path that must not block on or fail in the allocator in the
middle of a request, or a process whose device memory is owned by another
framework's allocator).  It must give exactly the lists dade_probe gives, call
after call, although every call reuses the same fixed scratch array, and also
where two lists are tied for a query (both probes compute the same bits, so
they break the tie alike).  This file builds what it needs, so it
passes alone in a fresh process as well as after the other tests.
"""
import ctypes as C

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
    base, queries, _ = synth.make("c1_gauss_10k_d128", n=6000, nq=96)
    assign = synth.zipf_assign(6000, 48, s=0.9)
    ix = dade.Index(torch.from_numpy(base).cuda(), 48, assign=assign, eps_pairs=2000)
    q = torch.from_numpy(queries).cuda()
    q_rot = torch.empty_like(q)
    ix.rotate(q, q_rot)
    return ix, q_rot


def _noalloc(ix, q_rot, nprobe, out):
    stream = torch.cuda.current_stream().cuda_stream
    return dade.lib().dade_probe_noalloc(ix.handle, q_rot.data_ptr(), q_rot.shape[0], nprobe, out.data_ptr(), stream)


def test_noalloc_probe_matches_probe_twice(index):
    ix, q_rot = index
    # two calls in a row with different batches: the second must not see the
    # first call's leftovers in the shared scratch array
    for rows, nprobe in ((slice(0, 96), 12), (slice(20, 70), 5)):
        q = q_rot[rows].contiguous()
        expected = torch.empty(q.shape[0], nprobe, dtype=torch.int32, device="cuda")
        ix.probe(q, nprobe, expected)
        got = torch.full((q.shape[0], nprobe), -7, dtype=torch.int32, device="cuda")
        assert _noalloc(ix, q, nprobe, got) == dade.OK, dade.lib().dade_last_error()
        ix.sync()
        assert torch.equal(got, expected)


def test_noalloc_probe_planted_ties(index):
    """Queries placed exactly between two centroids, on a centroid, and at the
    origin: every distance pair that rounds to a tie must be ordered the same
    way (by list id) by both probes."""
    ix, q_rot = index
    cent = torch.from_numpy(ix.export(dade.FIELD_CENTROIDS).reshape(ix.n_clusters, ix.d)).cuda()
    rows = [0.5 * (cent[a] + cent[b]) for a, b in ((0, 1), (3, 7), (10, 11), (20, 40), (5, 6))]
    rows += [cent[2].clone(), cent[9].clone(), torch.zeros(ix.d, device="cuda")]
    q = torch.stack(rows).contiguous()
    for nprobe in (1, 2, 7):
        expected = torch.empty(q.shape[0], nprobe, dtype=torch.int32, device="cuda")
        ix.probe(q, nprobe, expected)
        got = torch.full((q.shape[0], nprobe), -7, dtype=torch.int32, device="cuda")
        assert _noalloc(ix, q, nprobe, got) == dade.OK, dade.lib().dade_last_error()
        ix.sync()
        assert torch.equal(got, expected)


def test_noalloc_probe_limits(index):
    ix, q_rot = index
    too_many = dade.PROBE_NOALLOC_MAX // ix.n_clusters + 1
    big = torch.zeros(too_many, ix.d, device="cuda")
    out = torch.empty(too_many, 4, dtype=torch.int32, device="cuda")
    assert _noalloc(ix, big, 4, out) == dade.EINVAL
    assert b"DADE_PROBE_NOALLOC_MAX" in dade.lib().dade_last_error()
    host_q = np.zeros((4, ix.d), np.float32)
    host_out = np.zeros((4, 4), np.int32)
    rc = dade.lib().dade_probe_noalloc(ix.handle, host_q.ctypes.data, 4, 4, host_out.ctypes.data,
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == dade.EINVAL
