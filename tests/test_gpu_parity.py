"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Each test builds the same seeded inputs for both sides; the oracle never sees
anything the CUDA path produced.  Inverted lists are fixed by a seeded input
assignment (uneven random lists, or mixture labels), so both sides scan the
same lists; k-means itself is compared separately (test_kmeans_parity).
Tolerances are those of tests/parity.py.
"""
import itertools

import numpy as np
import pytest

import oracle
import parity
from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()
    dade.lib()


class Case:
    """A workload built on both sides with the same lists and eps pairs."""

    def __init__(self, base, queries, assign, n_clusters, n_pairs=20000, seed=4):
        self.base, self.queries = base, queries
        self.assign = np.ascontiguousarray(assign, np.int32)
        self.nc = n_clusters
        self.pairs = synth.eps_pairs(base.shape[0], n_pairs, seed=seed)
        self.orc = oracle.Index(base, n_clusters=n_clusters, assign=self.assign, pairs=self.pairs)
        self.gpu = dade.Index(torch.from_numpy(base).cuda(), n_clusters, assign=self.assign, pairs=self.pairs)
        self.q_dev = torch.from_numpy(queries).cuda()
        self.q_rot = torch.empty_like(self.q_dev)
        self.gpu.rotate(self.q_dev, self.q_rot)
        self.Qr = self.orc.rotate(queries)
        self.scale = float(np.mean((self.orc.Xr ** 2).sum(1)))

    def gpu_search(self, k, nprobe, alpha, delta_d, mode=dade.MODE_DADE, tile=128, stats=False,
                   schedule=dade.SCHED_TILE, threads=0, flags=0, seed_lists=0):
        nq = self.queries.shape[0]
        ids = torch.empty(nq, k, dtype=torch.int64, device="cuda")
        d = torch.empty(nq, k, dtype=torch.float32, device="cuda")
        st = torch.zeros(nq, 4, dtype=torch.int64, device="cuda") if stats else None
        self.gpu.search(self.q_rot, k, nprobe, alpha, delta_d, ids, d, mode=mode, tile=tile, stats=st,
                        schedule=schedule, threads=threads, flags=flags, seed_lists=seed_lists)
        self.gpu.sync()
        out = ids.cpu().numpy(), d.cpu().numpy()
        return out + ((st.cpu().numpy(),) if stats else ())

    def oracle_search(self, k, nprobe, alpha, delta_d, fd=False, tile=128, schedule=dade.SCHED_TILE, seed=0):
        """The oracle's bracketed search (parity.compare's input) in the GPU schedule's epochs."""
        eps = None if fd else self.orc.eps(np.float32(alpha), delta_d)
        if schedule == dade.SCHED_ROUNDS:
            o = self.orc.o.search_bracket(self.orc.Xr, self.assign, self.orc.cent, self.orc.lam, self.Qr, k,
                                          nprobe, delta_d if not fd else 64, eps, schedule=oracle.ROW_ROUNDS,
                                          tile=tile)
        else:
            lag = 0 if fd else dade.schedule_lag(self.base.shape[1], delta_d, schedule)
            o = self.orc.o.search_bracket(self.orc.Xr, self.assign, self.orc.cent, self.orc.lam, self.Qr, k, nprobe,
                                          delta_d if not fd else 64, eps, schedule=oracle.TILE, tile=tile, lag=lag,
                                          seed=seed)
        return o + (self.same_probe(nprobe),)

    def same_probe(self, nprobe):
        """Queries whose GPU probe lists (dade_probe, as inside the search) are the oracle's, in order."""
        pg = torch.empty(self.queries.shape[0], nprobe, dtype=torch.int32, device="cuda")
        self.gpu.probe(self.q_rot, nprobe, pg)
        self.gpu.sync()
        po, _ = self.orc.o.probe(self.Qr, self.orc.cent, nprobe)
        return (pg.cpu().numpy() == po).all(1)

    def exact_d(self, q, ids):
        return ((self.orc.Xr[ids] - self.Qr[q]) ** 2).sum(1)


@pytest.fixture(scope="module")
def c1():
    """10,000 x 128 Gaussian, lambda_i ~ i^-1.2, 100 queries, 64 uneven lists."""
    base, queries, _ = synth.make("c1_gauss_10k_d128")
    assign = synth.zipf_assign(base.shape[0], 64, s=0.6)
    return Case(base, queries, assign, 64)


@pytest.fixture(scope="module")
def mix():
    """20,000 x 64 mixture of 24 anisotropic Gaussians, lists = components."""
    w = synth.Workload("mix_test", 20000, 64, 120, 1.0, 24, 0.0, 3.0, 1.0, False, False, 24, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    return Case(base, queries, labels, 24)


def test_pca_parity(c1):
    g, o = c1.gpu, c1.orc
    assert np.allclose(g.export(dade.FIELD_MEAN), o.mu, rtol=0, atol=1e-12 * np.abs(o.mu).max() + 1e-15)
    lam = g.export(dade.FIELD_EIGVAL)
    assert np.max(np.abs(lam - o.lam) / o.lam[0]) < 1e-9
    W = g.export(dade.FIELD_BASIS)
    M = W.T @ o.W
    assert np.allclose(np.abs(np.diag(M)), 1.0, atol=1e-6)   # same eigenvectors up to sign


def _signs(c):
    """Eigenvectors are defined up to sign; align the GPU basis to the oracle's."""
    W = c.gpu.export(dade.FIELD_BASIS)
    return np.sign(np.einsum("jk,jk->k", W, c.orc.W))


def test_rotation_parity(c1):
    sg = _signs(c1)
    Xg = c1.gpu.export(dade.FIELD_ROTATED).astype(np.float64) * sg
    # every rotated vector within ROT_TOL of the exact one, relative to its own norm
    # (the FP32 error the parity tolerances and the oracle's decision bracket assume)
    err = np.linalg.norm(Xg - c1.orc.Xr, axis=1) / np.linalg.norm(c1.orc.Xr, axis=1)
    assert err.max() < parity.ROT_TOL, err.max()
    Qg = c1.q_rot.cpu().numpy().astype(np.float64) * sg
    err = np.linalg.norm(Qg - c1.Qr, axis=1) / np.linalg.norm(c1.Qr, axis=1)
    assert err.max() < parity.ROT_TOL, err.max()
    # host buffers in, host buffers out give the same bits
    qh = np.empty_like(c1.queries)
    c1.gpu.rotate(c1.queries, qh)
    assert np.array_equal(qh, c1.q_rot.cpu().numpy())


def test_assignment_and_centroids(c1):
    assert np.array_equal(c1.gpu.export(dade.FIELD_ASSIGN), c1.assign)
    cg = c1.gpu.export(dade.FIELD_CENTROIDS).astype(np.float64) * _signs(c1)
    err = np.linalg.norm(cg - c1.orc.cent, axis=1) / np.linalg.norm(c1.orc.cent, axis=1)
    assert err.max() < parity.ROT_TOL, err.max()


def test_eps_parity(c1):
    rho_g = c1.gpu.export(dade.FIELD_RHO)
    dl = c1.orc.dlist
    assert rho_g.shape == (len(dl), c1.orc.rho.shape[1])
    assert np.abs(rho_g - c1.orc.rho).max() < 1e-5
    for alpha in (0.05, 0.1, 0.3):
        for dd in (16, 32, 64):
            eg, cg = c1.gpu.eps_table(alpha, dd)
            eo = c1.orc.eps(np.float32(alpha), dd)
            for d in oracle.increments(128, dd):
                assert abs(eg[d] - eo[d]) < 2e-5, (alpha, dd, d)
                lam = c1.orc.lam
                coef = (1 + eo[d]) ** 2 * lam[:d].sum() / lam.sum()
                assert abs(cg[d] - coef) < 1e-4 * coef


@pytest.mark.parametrize("nprobe", [1, 8, 64])
def test_probe_parity(c1, mix, nprobe):
    for case in (c1, mix):
        if nprobe > case.nc:
            continue
        pg = np.empty((case.queries.shape[0], nprobe), np.int32)
        pg_dev = torch.empty(case.queries.shape[0], nprobe, dtype=torch.int32, device="cuda")
        case.gpu.probe(case.q_rot, nprobe, pg_dev)
        case.gpu.sync()
        pg = pg_dev.cpu().numpy()
        po, tie = case.orc.o.probe(case.Qr, case.orc.cent, nprobe)
        ok = np.all(pg == po, axis=1)
        assert np.all(ok | (tie != 0)), np.nonzero(~ok & (tie == 0))


@pytest.mark.parametrize("k,nprobe,alpha,delta_d,tile", [
    (10, 8, 0.05, 32, 128),      # the 10k x 128 configuration
    (10, 8, 0.1, 16, 128),
    (10, 8, 0.3, 64, 64),
    (1, 4, 0.05, 32, 32),
    (100, 16, 0.05, 32, 256),
    (256, 8, 0.2, 32, 96),
])
@pytest.mark.parametrize("schedule,threads,flags", [(dade.SCHED_TILE, 128, 0), (dade.SCHED_TILE, 256, 0),
                                                    (dade.SCHED_TILE, 128, dade.FLAG_GENERIC_KERNEL),
                                                    (dade.SCHED_PIPELINED, 128, 0), (dade.SCHED_PIPELINED, 256, 0)])
def test_search_parity_c1(c1, k, nprobe, alpha, delta_d, tile, schedule, threads, flags):
    g_ids, g_d, g_st = c1.gpu_search(k, nprobe, alpha, delta_d, tile=tile, stats=True, schedule=schedule,
                                     threads=threads, flags=flags)
    o = c1.oracle_search(k, nprobe, alpha, delta_d, tile=tile, schedule=schedule)
    parity.compare(g_ids, g_d, o, c1.exact_d)
    # the work done is the same: candidates exactly, the rest where the bracket counts the same
    parity.compare_stats(g_st, o)
    if schedule == dade.SCHED_TILE:   # a deep pipeline on a short scan may never refresh its threshold
        assert np.all(g_st[:, 1] < g_st[:, 0] * 128)   # DADE used fewer dimensions than FDScanning


@pytest.mark.parametrize("k,nprobe,alpha,delta_d", [(10, 4, 0.1, 16), (10, 2, 0.05, 32), (50, 6, 0.2, 64)])
@pytest.mark.parametrize("schedule", [dade.SCHED_TILE, dade.SCHED_PIPELINED])
def test_search_parity_mixture(mix, k, nprobe, alpha, delta_d, schedule):
    g_ids, g_d = mix.gpu_search(k, nprobe, alpha, delta_d, schedule=schedule)
    o = mix.oracle_search(k, nprobe, alpha, delta_d, schedule=schedule)
    parity.compare(g_ids, g_d, o, mix.exact_d)


@pytest.mark.parametrize("k,nprobe", [(10, 8), (100, 16)])
@pytest.mark.parametrize("threads,flags", [(128, 0), (256, 0), (256, dade.FLAG_GENERIC_KERNEL)])
def test_fd_parity(c1, k, nprobe, threads, flags):
    g_ids, g_d, g_st = c1.gpu_search(k, nprobe, 0.1, 32, mode=dade.MODE_FD, stats=True, threads=threads,
                                     flags=flags)
    o = c1.oracle_search(k, nprobe, 0.1, 32, fd=True)
    parity.compare(g_ids, g_d, o, c1.exact_d)
    parity.compare_stats(g_st, o)
    assert np.all(g_st[:, 1] == g_st[:, 0] * 128)


def test_host_buffers_match_device(c1):
    k, nprobe = 10, 8
    d_ids, d_d = c1.gpu_search(k, nprobe, 0.05, 32)
    ids = np.empty((c1.queries.shape[0], k), np.int64)
    dist = np.empty((c1.queries.shape[0], k), np.float32)
    c1.gpu.query(c1.queries, k, nprobe, 0.05, 32, ids, dist)
    assert np.array_equal(ids, d_ids) and np.array_equal(dist, d_d)


def test_exhaustive_fd_is_exact_knn():
    """nprobe = N_c with FDScanning is exact KNN (oracle brute force in the
    original space), including ties between duplicated vectors."""
    base, queries, _ = synth.make("c1_gauss_10k_d128", n=3000, nq=40)
    base[7] = base[1500]
    queries[5] = base[1500]
    assign = synth.zipf_assign(3000, 10, s=1.1)
    g = dade.Index(torch.from_numpy(base).cuda(), 10, assign=assign, eps_pairs=2000)
    ids = torch.empty(40, 20, dtype=torch.int64, device="cuda")
    d = torch.empty(40, 20, dtype=torch.float32, device="cuda")
    g.query(torch.from_numpy(queries).cuda(), 20, 10, 0.1, 32, ids, d, mode=dade.MODE_FD)
    g.sync()
    o_ids, o_d = oracle.get().exact_knn(base, queries, 20)
    gi = ids.cpu().numpy()
    for q in range(40):
        for a, b in parity._runs(o_d[q]):
            assert set(gi[q, a:b]) == set(o_ids[q, a:b]), q
    assert gi[5, 0] == 7 and gi[5, 1] == 1500   # equal distance 0: lower id first


@pytest.mark.parametrize("d,nlists,delta_d", [(16, 3, 16), (20, 5, 16), (40, 4, 32), (48, 6, 32), (64, 3, 64),
                                              (33, 7, 1024), (160, 5, 16)])
def test_odd_shapes(d, nlists, delta_d):
    """D not a multiple of 16 or of delta_d, delta_d >= D, empty lists, K > candidates."""
    rng = np.random.default_rng(d)
    base = (rng.standard_normal((700, d)) * np.linspace(2.0, 0.2, d)).astype(np.float32)
    queries = (rng.standard_normal((25, d)) * np.linspace(2.0, 0.2, d)).astype(np.float32)
    assign = synth.zipf_assign(700, nlists, s=1.5)
    if nlists >= 3:
        assign[assign == 1] = 2               # one empty list (its centroid is the origin)
    case = Case(base, queries, assign, nlists, n_pairs=3000)
    for k, nprobe in ((5, 1), (200, 2), (10, nlists)):
        for schedule in (dade.SCHED_TILE, dade.SCHED_PIPELINED):
            g_ids, g_d = case.gpu_search(k, nprobe, 0.1, delta_d, tile=32, schedule=schedule)
            o = case.oracle_search(k, nprobe, 0.1, delta_d, tile=32, schedule=schedule)
            parity.compare(g_ids, g_d, o, case.exact_d)


def test_empty_batch_and_invalid(c1):
    ids = torch.empty(0, 10, dtype=torch.int64, device="cuda")
    d = torch.empty(0, 10, dtype=torch.float32, device="cuda")
    c1.gpu.search(c1.q_rot[:0], 10, 8, 0.05, 32, ids, d)
    with pytest.raises(dade.DadeError) as e:
        c1.gpu.search(c1.q_rot, 10, 65, 0.05, 32, torch.empty(100, 10, dtype=torch.int64, device="cuda"),
                      torch.empty(100, 10, device="cuda"))
    assert e.value.status == dade.EINVAL
    with pytest.raises(dade.DadeError):
        c1.gpu.search(c1.q_rot, 10, 8, 0.05, 24, ids, d)
    with pytest.raises(dade.DadeError):
        c1.gpu.search(c1.q_rot, 10, 8, 1.5, 32, ids, d)


def test_kmeans_parity():
    """GPU k-means (FP32 distances, FP64 sums) vs the oracle's FP64 Lloyd
    iterations from the same initial ids: per-iteration objectives agree to
    1e-5 and the final lists agree on almost every vector."""
    base, _, _ = synth.make("c1_gauss_10k_d128", n=6000, nq=1)
    init = synth.kmeans_init(6000, 32, seed=3)
    g = dade.Index(torch.from_numpy(base).cuda(), 32, kmeans_iters=6, kmeans_init=init, eps_pairs=1000)
    o = oracle.Index(base, init=init, iters=6, pairs=synth.eps_pairs(6000, 1000))
    obj_g = g.export(dade.FIELD_KMEANS_OBJ)
    assert np.allclose(obj_g, o.kmeans_obj, rtol=1e-5)
    agree = np.mean(g.export(dade.FIELD_ASSIGN) == o.assign)
    assert agree > 0.995, agree


@pytest.mark.parametrize("mode,delta_d,flags", [(dade.MODE_DADE, 32, 0), (dade.MODE_DADE, 64, 0),
                                                (dade.MODE_FD, 32, 0),
                                                (dade.MODE_DADE, 48, dade.FLAG_GENERIC_KERNEL)])
def test_query_order_gives_same_results(c1, mode, delta_d, flags):
    """Running the queries grouped by first probed list changes only the
    order of the CTAs: ids, distance bits and statistics are unchanged."""
    a = c1.gpu_search(10, 8, 0.1, delta_d, mode=mode, stats=True, flags=flags)
    b = c1.gpu_search(10, 8, 0.1, delta_d, mode=mode, stats=True, flags=flags | dade.FLAG_QUERY_ORDER)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("tail_from,delta_d,flags", [(64, 64, 0), (32, 32, 0), (16, 16, 0), (32, 64, dade.FLAG_LEAD),
                                                     (48, 32, dade.FLAG_GENERIC_KERNEL),
                                                     (16, 16, dade.FLAG_GENERIC_KERNEL | dade.FLAG_LEAD),
                                                     (112, 64, dade.FLAG_GENERIC_KERNEL)])
def test_row_tail_gives_same_results(tail_from, delta_d, flags):
    """Survivors reading their later dims from the row-major tail copy get
    the same bits as from the dimension-blocked slabs."""
    base, queries, _ = synth.make("c1_gauss_10k_d128", n=6000, nq=80)
    assign = synth.zipf_assign(6000, 30, s=0.7)
    ix = dade.Index(torch.from_numpy(base).cuda(), 30, assign=assign, eps_pairs=3000, tail_from=tail_from,
                    lead_format=dade.LEAD_BF16, lead_dims=64)
    assert ix.info.tail_from == tail_from
    q = torch.from_numpy(queries).cuda()
    out = []
    for extra in (0, dade.FLAG_ROW_TAIL):
        ids = torch.empty(80, 20, dtype=torch.int64, device="cuda")
        d = torch.empty(80, 20, dtype=torch.float32, device="cuda")
        st = torch.zeros(80, 4, dtype=torch.int64, device="cuda")
        ix.query(q, 20, 8, 0.1, delta_d, ids, d, stats=st, flags=flags | extra)
        ix.sync()
        out.append((ids.cpu().numpy(), d.cpu().numpy(), st.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("k,nprobe,alpha,delta_d,tile,seed", [
    (10, 8, 0.05, 32, 128, 2),
    (10, 8, 0.1, 16, 64, 1),
    (100, 16, 0.3, 64, 256, 2),
    (1, 4, 0.2, 32, 32, 3),
    (256, 8, 0.1, 64, 128, 1),       # phase 1 finds fewer than K: r frozen at +inf
    (20, 12, 0.1, 128, 128, 2),      # one increment
    (10, 8, 0.1, 32, 4096, 3),       # whole-list epochs: the seed lists run list-major as rounds
    (100, 16, 0.3, 64, 4096, 1),
    (1, 6, 0.2, 16, 4096, 5),
])
@pytest.mark.parametrize("flags", [0, dade.FLAG_QUERY_ORDER, dade.FLAG_SEED_SPLIT,
                                   dade.FLAG_SEED_SPLIT | dade.FLAG_QUERY_ORDER])
def test_seeded_schedule_parity(c1, k, nprobe, alpha, delta_d, tile, seed, flags):
    g_ids, g_d, g_st = c1.gpu_search(k, nprobe, alpha, delta_d, tile=tile, stats=True, schedule=dade.SCHED_SEEDED,
                                     seed_lists=seed, flags=flags)
    o = c1.oracle_search(k, nprobe, alpha, delta_d, tile=tile, seed=seed)
    parity.compare(g_ids, g_d, o, c1.exact_d)
    parity.compare_stats(g_st, o)


@pytest.mark.parametrize("k,nprobe", [(10, 8), (100, 16)])
@pytest.mark.parametrize("tile", [128, 4096])
def test_seeded_fd_is_fd(c1, k, nprobe, tile):
    """FDScanning under the seeded schedule is exact IVF: the same results as
    the tile schedule, whatever the seed."""
    a = c1.gpu_search(k, nprobe, 0.1, 32, mode=dade.MODE_FD)
    b = c1.gpu_search(k, nprobe, 0.1, 32, mode=dade.MODE_FD, schedule=dade.SCHED_SEEDED, seed_lists=1, tile=tile)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    # split passes run the generic tile kernel, whose per-lane sums group 64 dims at a time
    g = dade.FLAG_GENERIC_KERNEL
    a = c1.gpu_search(k, nprobe, 0.1, 32, mode=dade.MODE_FD, flags=g)
    b = c1.gpu_search(k, nprobe, 0.1, 32, mode=dade.MODE_FD, schedule=dade.SCHED_SEEDED, seed_lists=1, tile=tile,
                      flags=g | dade.FLAG_SEED_SPLIT)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


def test_seeded_schedule_mixture_and_limits():
    """A 128-dim mixture whose lists are its 24 components (uneven, some
    probed by many queries), and the limits of the seed."""
    w = synth.Workload("mix128_test", 16000, 128, 90, 1.0, 24, 0.0, 3.0, 1.0, False, False, 24, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    case = Case(base, queries, labels, 24, n_pairs=8000)
    for k, nprobe, seed, dd, tile in ((10, 6, 1, 32, 128), (50, 8, 2, 16, 128), (30, 12, 3, 64, 128),
                                      (30, 12, 3, 64, 1 << 20)):
        g_ids, g_d = case.gpu_search(k, nprobe, 0.1, dd, schedule=dade.SCHED_SEEDED, seed_lists=seed, tile=tile)
        o = case.oracle_search(k, nprobe, 0.1, dd, seed=seed, tile=tile)
        parity.compare(g_ids, g_d, o, case.exact_d)
    # seed >= nprobe is the tile schedule
    a = case.gpu_search(10, 4, 0.1, 32, stats=True)
    b = case.gpu_search(10, 4, 0.1, 32, stats=True, schedule=dade.SCHED_SEEDED, seed_lists=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    # D = 64 and D = 40 (fewer than 8 blocks) are outside the list-major kernels: the
    # passes with r frozen run query-major, tile and whole-list epochs alike
    for d in (64, 40):
        small = Case(*synth.make(synth.Workload(f"mix{d}", 3000, d, 10, 1.0, 6, 0.0, 3.0, 1.0, False, False, 6, (4,),
                                                10, (16,), 0.1))[:2], synth.zipf_assign(3000, 6, s=0.5), 6,
                     n_pairs=1000)
        for tile, seed in ((64, 1), (1 << 20, 2)):
            g_ids, g_d = small.gpu_search(5, 4, 0.1, 32, schedule=dade.SCHED_SEEDED, seed_lists=seed, tile=tile)
            o = small.oracle_search(5, 4, 0.1, 32, seed=seed, tile=tile)
            parity.compare(g_ids, g_d, o, small.exact_d)


@pytest.mark.parametrize("d,delta_d,seed,tile", [(160, 16, 2, 128), (160, 32, 1, 4096), (256, 64, 2, 128),
                                                 (384, 128, 3, 128), (136, 16, 2, 128)])
def test_seeded_schedule_any_dimension(d, delta_d, seed, tile):
    """The list-major kernel for D > 128 (blocks walked in windows): parity
    with the oracle's seeded schedule, and FDScanning unchanged."""
    w = synth.Workload(f"mix{d}", 8000, d, 70, 1.0, 20, 0.0, 3.0, 1.0, False, False, 20, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    case = Case(base, queries, labels, 20, n_pairs=4000)
    for (k, nprobe), fl in itertools.product(((10, 8), (60, 12)), (0, dade.FLAG_SEED_SPLIT)):
        g_ids, g_d, g_st = case.gpu_search(k, nprobe, 0.1, delta_d, tile=tile, stats=True,
                                           schedule=dade.SCHED_SEEDED, seed_lists=seed, flags=fl)
        o = case.oracle_search(k, nprobe, 0.1, delta_d, tile=tile, seed=seed)
        parity.compare(g_ids, g_d, o, case.exact_d)
        parity.compare_stats(g_st, o)
    a = case.gpu_search(10, 8, 0.1, 32, mode=dade.MODE_FD)
    b = case.gpu_search(10, 8, 0.1, 32, mode=dade.MODE_FD, schedule=dade.SCHED_SEEDED, seed_lists=2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


@pytest.mark.parametrize("d,delta_d,stage", [(160, 16, 64), (160, 32, 160), (256, 16, 128), (128, 32, 96),
                                             (40, 16, 48)])
def test_staged_depth_gives_same_results(d, delta_d, stage):
    """Streaming several increments per tile (tested inside the staged unit)
    changes where the bytes come from, not the results: ids, distance bits
    and work counters equal the one-increment stage, and the oracle."""
    w = synth.Workload(f"stage{d}", 6000, d, 60, 1.0, 16, 0.0, 3.0, 1.0, False, False, 16, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    case = Case(base, queries, labels, 16, n_pairs=3000)
    nq = queries.shape[0]
    out = []
    for sd in (0, stage):
        ids = torch.empty(nq, 20, dtype=torch.int64, device="cuda")
        dd = torch.empty(nq, 20, dtype=torch.float32, device="cuda")
        st = torch.zeros(nq, 4, dtype=torch.int64, device="cuda")
        case.gpu.search(case.q_rot, 20, 6, 0.1, delta_d, ids, dd, tile=64, stats=st, stage_dims=sd,
                        flags=dade.FLAG_GENERIC_KERNEL)
        case.gpu.sync()
        out.append((ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))
    assert np.array_equal(out[0][2], out[1][2])
    o = case.oracle_search(20, 6, 0.1, delta_d, tile=64)
    parity.compare(out[1][0], out[1][1], o, case.exact_d)


@pytest.mark.parametrize("d,delta_d,tail_from,spec", [(160, 32, 32, 8), (256, 16, 64, 3), (200, 64, 16, 8),
                                                      (960, 32, 32, 8)])
def test_generic_kernel_row_tail_and_window(d, delta_d, tail_from, spec):
    """D > 128 on the tile kernel, with and without the row-major tail in the
    index and with several survivor window widths: same bits, same counters,
    and oracle parity."""
    n = 3000 if d > 512 else 6000
    w = synth.Workload(f"tail{d}", n, d, 50, 1.0, 16, 0.0, 3.0, 1.0, False, False, 16, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    case = Case(base, queries, labels, 16, n_pairs=3000)
    ix = dade.Index(torch.from_numpy(base).cuda(), 16, assign=case.assign, pairs=case.pairs, tail_from=tail_from)
    nq = queries.shape[0]
    q_rot = torch.empty_like(case.q_dev)
    ix.rotate(case.q_dev, q_rot)
    out = []
    for extra, sp in ((0, 8), (dade.FLAG_ROW_TAIL, 8), (dade.FLAG_ROW_TAIL, spec)):
        ids = torch.empty(nq, 20, dtype=torch.int64, device="cuda")
        dd = torch.empty(nq, 20, dtype=torch.float32, device="cuda")
        st = torch.zeros(nq, 4, dtype=torch.int64, device="cuda")
        ix.search(q_rot, 20, 6, 0.1, delta_d, ids, dd, tile=64, stats=st, spec=sp,
                  flags=dade.FLAG_GENERIC_KERNEL | extra)
        ix.sync()
        out.append((ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy()))
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0]) and np.array_equal(out[0][1].view(np.uint32), o[1].view(np.uint32))
        assert np.array_equal(out[0][2], o[2])
    o = case.oracle_search(20, 6, 0.1, delta_d, tile=64)
    parity.compare(out[0][0], out[0][1], o, case.exact_d)


@pytest.mark.parametrize("delta_d,seed,flags", [(32, 2, 0), (16, 1, dade.FLAG_QUERY_ORDER), (64, 3, 0)])
def test_seed_split_matches_list_major(c1, delta_d, seed, flags):
    """The lists after the seeds, query-major and split over thread blocks,
    against list-major: the same r, the same tests, so the same bits and
    work counters."""
    a = c1.gpu_search(50, 12, 0.1, delta_d, stats=True, schedule=dade.SCHED_SEEDED, seed_lists=seed, flags=flags)
    b = c1.gpu_search(50, 12, 0.1, delta_d, stats=True, schedule=dade.SCHED_SEEDED, seed_lists=seed,
                      flags=flags | dade.FLAG_SEED_SPLIT)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    assert np.array_equal(a[2], b[2])


def test_seed_split_with_prefilter():
    """The split later lists with the low-precision prefilter: FP32 results
    equal the FP32 path's, and the dropped-candidate counts add up over the
    seed lists and every part."""
    base, queries, _ = synth.make("c1_gauss_10k_d128", n=6000, nq=60)
    assign = synth.zipf_assign(6000, 30, s=0.7)
    ix = dade.Index(torch.from_numpy(base).cuda(), 30, assign=assign, eps_pairs=3000,
                    lead_format=dade.LEAD_BF16, lead_dims=64)
    q = torch.from_numpy(queries).cuda()
    out = []
    for fl in (dade.FLAG_SEED_SPLIT, dade.FLAG_SEED_SPLIT | dade.FLAG_LEAD):
        ids = torch.empty(60, 20, dtype=torch.int64, device="cuda")
        d = torch.empty(60, 20, dtype=torch.float32, device="cuda")
        st = torch.zeros(60, 4, dtype=torch.int64, device="cuda")
        ls = torch.zeros(60, dtype=torch.int64, device="cuda") if fl & dade.FLAG_LEAD else None
        ix.query(q, 20, 10, 0.1, 32, ids, d, stats=st, flags=fl, schedule=dade.SCHED_SEEDED, seed_lists=2,
                 tile=64, lead_stats=ls)
        ix.sync()
        out.append((ids.cpu().numpy(), d.cpu().numpy(), st.cpu().numpy(), None if ls is None else ls.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))
    assert np.array_equal(out[0][2][:, 0], out[1][2][:, 0])
    assert (out[1][3] > 0).any() and (out[1][3] <= out[1][2][:, 0]).all()


@pytest.mark.parametrize("d,delta_d,tile,seed", [(128, 32, 128, 2), (128, 16, 4096, 2), (160, 32, 128, 2),
                                                 (256, 64, 4096, 1)])
def test_list_chunks_same_results(d, delta_d, tile, seed):
    """List-major work items that cover a list in several chunks (other
    thread blocks, other times) give the same bits and counters as one item
    per list: r is frozen in those passes."""
    w = synth.Workload(f"chunk{d}", 12000, d, 60, 1.0, 8, 0.0, 3.0, 1.0, False, False, 8, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    case = Case(base, queries, labels, 8, n_pairs=3000)    # 8 lists of ~1,500 rows
    out = []
    for chunk in (0, 64, 192):
        nq = queries.shape[0]
        ids = torch.empty(nq, 20, dtype=torch.int64, device="cuda")
        dd = torch.empty(nq, 20, dtype=torch.float32, device="cuda")
        st = torch.zeros(nq, 4, dtype=torch.int64, device="cuda")
        case.gpu.search(case.q_rot, 20, 5, 0.1, delta_d, ids, dd, tile=tile, stats=st,
                        schedule=dade.SCHED_SEEDED, seed_lists=seed, list_chunk=chunk)
        case.gpu.sync()
        out.append((ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy()))
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0]) and np.array_equal(out[0][1].view(np.uint32), o[1].view(np.uint32))
        assert np.array_equal(out[0][2], o[2])
    o = case.oracle_search(20, 5, 0.1, delta_d, tile=tile, seed=seed)
    parity.compare(out[1][0], out[1][1], o, case.exact_d)


def test_accept_buffer_overflow_is_reported():
    """A pass with r = +inf over a list longer than the accept buffer
    (65,536 entries per query) reports DADE_ENOMEM at the next sync instead
    of returning partial results silently; the index stays usable."""
    n, d = 70000, 16
    rng = np.random.default_rng(5)
    base = rng.standard_normal((n, d)).astype(np.float32)
    assign = np.zeros(n, np.int32)
    assign[:8] = 1                                            # list 0: 69,992 rows; list 1: 8, far away
    base[:8, 0] += 100.0
    ix = dade.Index(torch.from_numpy(base).cuda(), 2, assign=assign, eps_pairs=2000)
    q = torch.from_numpy(base[8:12].copy()).cuda()            # list 0 is probed first
    ids = torch.empty(4, 5, dtype=torch.int64, device="cuda")
    dd = torch.empty(4, 5, dtype=torch.float32, device="cuda")
    with pytest.raises(dade.DadeError) as e:
        ix.query(q, 5, 2, 0.1, 16, ids, dd, schedule=dade.SCHED_SEEDED, seed_lists=1, tile=1 << 20,
                 flags=dade.FLAG_SEED_SPLIT | dade.FLAG_GENERIC_KERNEL)
        ix.sync()
    assert e.value.status == dade.ENOMEM
    ix.query(q, 5, 2, 0.1, 16, ids, dd)                      # the tile schedule still answers
    ix.sync()
    assert (ids.cpu().numpy()[:, 0] == np.arange(8, 12)).all()


def test_kbest_staging_bounds_a_loose_threshold():
    """A list-major pass with r = +inf over a 70,000-row list (whole-list
    seed epoch, D = 144): each work item keeps only its K best accepted keys
    per query, so the pass fits the accept buffer, and the results are the
    oracle's."""
    n, d = 70000, 144
    w = synth.Workload("kbest", n, d, 6, 1.0, 1, 0.0, 0.0, 1.0, False, False, 2, (2,), 10, (16,), 0.1)
    base, queries, _ = synth.make(w)
    assign = np.zeros(n, np.int32)
    assign[:8] = 1
    base[:8, :] += 50.0                                       # list 1: 8 rows far away
    case = Case(base, queries, assign, 2, n_pairs=3000)
    for tile, seed in ((1 << 20, 1), (128, 1)):
        g_ids, g_d, g_st = case.gpu_search(10, 2, 0.1, 32, tile=tile, stats=True, schedule=dade.SCHED_SEEDED,
                                           seed_lists=seed)
        o = case.oracle_search(10, 2, 0.1, 32, tile=tile, seed=seed)
        parity.compare(g_ids, g_d, o, case.exact_d)
        parity.compare_stats(g_st, o)


@pytest.mark.parametrize("d,ring,flags", [(160, 4, 0), (128, 3, dade.FLAG_GENERIC_KERNEL), (256, 8, 0),
                                          (128, 4, dade.FLAG_GENERIC_KERNEL | dade.FLAG_LEAD)])
def test_stage_ring_gives_same_results(d, ring, flags):
    """More staged tiles in flight per thread block changes when bytes
    arrive, not the results."""
    w = synth.Workload(f"ring{d}", 6000, d, 50, 1.0, 16, 0.0, 3.0, 1.0, False, False, 16, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    ix = dade.Index(torch.from_numpy(base).cuda(), 16, assign=labels, eps_pairs=3000,
                    lead_format=dade.LEAD_BF16, lead_dims=64)
    q = torch.from_numpy(queries).cuda()
    out = []
    for r in (0, ring):
        ids = torch.empty(q.shape[0], 20, dtype=torch.int64, device="cuda")
        dd = torch.empty(q.shape[0], 20, dtype=torch.float32, device="cuda")
        st = torch.zeros(q.shape[0], 4, dtype=torch.int64, device="cuda")
        ix.query(q, 20, 6, 0.1, 32, ids, dd, tile=64, stats=st, flags=flags, stage_ring=r)
        ix.sync()
        out.append((ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))
    assert np.array_equal(out[0][2], out[1][2])


def test_flat_index_is_a_linear_scan():
    """One list holding every vector (a flat index, Section 5's linear-scan
    setting): DADE against the oracle for several delta_d and alpha, and
    FDScanning against the oracle's (itself pinned to brute force)."""
    base, queries, _ = synth.make("c1_gauss_10k_d128", n=6000, nq=30)
    case = Case(base, queries, np.zeros(6000, np.int32), 1, n_pairs=4000)
    for dd, alpha in ((16, 0.05), (32, 0.1), (64, 0.3)):
        g_ids, g_d, g_st = case.gpu_search(10, 1, alpha, dd, tile=256, stats=True)
        o = case.oracle_search(10, 1, alpha, dd, tile=256)
        parity.compare(g_ids, g_d, o, case.exact_d)
        parity.compare_stats(g_st, o)
    f_ids, f_d = case.gpu_search(10, 1, 0.1, 32, mode=dade.MODE_FD)
    o = case.oracle_search(10, 1, 0.1, 32, fd=True)
    parity.compare(f_ids, f_d, o, case.exact_d)


@pytest.mark.parametrize("d,schedule,seed", [(128, dade.SCHED_TILE, 0), (128, dade.SCHED_SEEDED, 2),
                                             (160, dade.SCHED_SEEDED, 2)])
def test_tune_keeps_results_and_caches(d, schedule, seed):
    """dade_tune picks among options that leave results unchanged: the tuned
    options give the base options' bits and counters, and a repeated shape
    returns the cached choice."""
    w = synth.Workload(f"tune{d}", 8000, d, 64, 1.0, 16, 0.0, 3.0, 1.0, False, False, 16, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    ix = dade.Index(torch.from_numpy(base).cuda(), 16, assign=labels, eps_pairs=3000, tail_from=32)
    q = torch.from_numpy(queries).cuda()
    qr = torch.empty_like(q)
    ix.rotate(q, qr)
    pr = torch.empty(q.shape[0], 10, dtype=torch.int32, device="cuda")
    ix.probe(qr, 10, pr)
    ids = torch.empty(q.shape[0], 20, dtype=torch.int64, device="cuda")
    dd = torch.empty(q.shape[0], 20, dtype=torch.float32, device="cuda")
    opts = dict(tile=128, threads=128, schedule=schedule, seed_lists=seed, flags=0)
    tuned = ix.tune(qr, pr, 20, 10, 0.1, 32, ids, dd, **opts)
    assert tuned["threads"] in (128, 256) and tuned["flags"] & ~(dade.FLAG_QUERY_ORDER | dade.FLAG_ROW_TAIL |
                                                                 dade.FLAG_SEED_SPLIT) == 0
    assert ix.tune(qr, pr, 20, 10, 0.1, 32, ids, dd, **opts) == tuned
    out = []
    for o in (opts, dict(opts, **tuned)):
        st = torch.zeros(q.shape[0], 4, dtype=torch.int64, device="cuda")
        ix.scan(qr, pr, 20, 0.1, 32, ids, dd, stats=st, **o)
        ix.sync()
        out.append((ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))
    assert np.array_equal(out[0][2], out[1][2])
    # every candidate the tuner may choose gives the same bits (not only the winner)
    for nt in (128, 256):
        for fl in (dade.FLAG_QUERY_ORDER | dade.FLAG_ROW_TAIL,
                   dade.FLAG_SEED_SPLIT if schedule == dade.SCHED_SEEDED else dade.FLAG_ROW_TAIL):
            ix.scan(qr, pr, 20, 0.1, 32, ids, dd, **dict(opts, threads=nt, flags=fl))
            ix.sync()
            assert np.array_equal(out[0][0], ids.cpu().numpy())
            assert np.array_equal(out[0][1].view(np.uint32), dd.cpu().numpy().view(np.uint32))


# ---- the row-rounds schedule -------------------------------------------------------

@pytest.mark.parametrize("k,nprobe,alpha,delta_d,r1", [
    (10, 8, 0.05, 32, 64), (10, 8, 0.1, 16, 1), (100, 16, 0.3, 64, 32), (1, 4, 0.2, 32, 7),
    (256, 8, 0.1, 64, 64),          # round 0 finds fewer than K: the next round runs with r = +inf
    (20, 12, 0.1, 128, 100),        # one increment
    (10, 8, 0.1, 32, 4096),         # one round holds every row: exact
])
@pytest.mark.parametrize("flags", [0, dade.FLAG_QUERY_ORDER, dade.FLAG_SEED_SPLIT])
def test_rounds_schedule_parity(c1, k, nprobe, alpha, delta_d, r1, flags):
    g_ids, g_d, g_st = c1.gpu_search(k, nprobe, alpha, delta_d, tile=r1, stats=True, schedule=dade.SCHED_ROUNDS,
                                     flags=flags)
    o = c1.oracle_search(k, nprobe, alpha, delta_d, tile=r1, schedule=dade.SCHED_ROUNDS)
    parity.compare(g_ids, g_d, o, c1.exact_d)
    parity.compare_stats(g_st, o)


@pytest.mark.parametrize("d,delta_d,r1", [(160, 16, 64), (256, 64, 16), (384, 128, 64), (136, 32, 1), (64, 32, 16),
                                          (40, 16, 8)])
def test_rounds_schedule_any_dimension(d, delta_d, r1):
    """List-major rounds for D > 112 (blocks walked in windows), query-major
    split rounds below: parity with the oracle's row rounds, the split form
    equal to the list-major one bit for bit, FDScanning unchanged."""
    w = synth.Workload(f"mix{d}", 8000, d, 70, 1.0, 20, 0.0, 3.0, 1.0, False, False, 20, (4,), 10, (16,), 0.1)
    base, queries, labels = synth.make(w)
    case = Case(base, queries, labels, 20, n_pairs=4000)
    for k, nprobe in ((10, 8), (60, 12)):
        outs = []
        for fl in (0, dade.FLAG_SEED_SPLIT):
            outs.append(case.gpu_search(k, nprobe, 0.1, delta_d, tile=r1, stats=True, schedule=dade.SCHED_ROUNDS,
                                        flags=fl))
        o = case.oracle_search(k, nprobe, 0.1, delta_d, tile=r1, schedule=dade.SCHED_ROUNDS)
        parity.compare(outs[0][0], outs[0][1], o, case.exact_d)
        parity.compare_stats(outs[0][2], o)
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][2], outs[1][2])
        assert np.array_equal(outs[0][1].view(np.uint32), outs[1][1].view(np.uint32))
    # FDScanning: exact whatever the rounds (the list-major kernel sums its dims in
    # another grouping than the tile kernel, so distances agree to rounding)
    b = case.gpu_search(10, 8, 0.1, 32, mode=dade.MODE_FD, schedule=dade.SCHED_ROUNDS, tile=16)
    o = case.oracle_search(10, 8, 0.1, 32, fd=True)
    parity.compare(b[0], b[1], o, case.exact_d)


def test_rounds_schedule_dominant_list():
    """Zipf(1.1) list sizes over 64 lists of a 60,000 x 192 mixture (the
    largest list holds about a fifth of the data): rounds of doubling row
    windows cut it into chunks over many thread blocks; any chunk size gives
    the same bits and counters, and the oracle's results."""
    w = synth.Workload("zipf192", 60000, 192, 80, 1.5, 64, 0.0, 2.0, 1.0, False, True, 64, (4,), 10, (32,), 0.1,
                       comp_zipf=1.1, lists_are_components=True)
    base, queries, labels = synth.make(w)
    case = Case(base, queries, labels, 64, n_pairs=4000)
    assert np.bincount(labels).max() > 0.15 * base.shape[0]
    out = []
    for chunk in (0, 64, 256):
        nq = queries.shape[0]
        ids = torch.empty(nq, 10, dtype=torch.int64, device="cuda")
        dd = torch.empty(nq, 10, dtype=torch.float32, device="cuda")
        st = torch.zeros(nq, 4, dtype=torch.int64, device="cuda")
        case.gpu.search(case.q_rot, 10, 6, 0.1, 32, ids, dd, tile=64, stats=st, schedule=dade.SCHED_ROUNDS,
                        list_chunk=chunk)
        case.gpu.sync()
        out.append((ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy()))
    for o2 in out[1:]:
        assert np.array_equal(out[0][0], o2[0]) and np.array_equal(out[0][1].view(np.uint32), o2[1].view(np.uint32))
        assert np.array_equal(out[0][2], o2[2])
    o = case.oracle_search(10, 6, 0.1, 32, tile=64, schedule=dade.SCHED_ROUNDS)
    parity.compare(out[0][0], out[0][1], o, case.exact_d)
    parity.compare_stats(out[0][2], o)


def test_rounds_schedule_with_prefilter():
    """Row rounds with the low-precision prefilter (query-major rounds): the
    FP32 path's bits and counters."""
    base, queries, _ = synth.make("c1_gauss_10k_d128", n=6000, nq=60)
    assign = synth.zipf_assign(6000, 30, s=1.0)
    ix = dade.Index(torch.from_numpy(base).cuda(), 30, assign=assign, eps_pairs=3000,
                    lead_format=dade.LEAD_FP8, lead_dims=64)
    q = torch.from_numpy(queries).cuda()
    out = []
    for fl in (dade.FLAG_SEED_SPLIT, dade.FLAG_LEAD):
        ids = torch.empty(60, 20, dtype=torch.int64, device="cuda")
        d = torch.empty(60, 20, dtype=torch.float32, device="cuda")
        st = torch.zeros(60, 4, dtype=torch.int64, device="cuda")
        ix.query(q, 20, 10, 0.1, 32, ids, d, stats=st, flags=fl, schedule=dade.SCHED_ROUNDS, tile=32)
        ix.sync()
        out.append((ids.cpu().numpy(), d.cpu().numpy(), st.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))
    assert np.array_equal(out[0][2], out[1][2])


# ---- the tensor-core prefilter of the list-major passes -----------------------------

@pytest.mark.parametrize("d,delta_d,schedule,tile", [(128, 32, dade.SCHED_ROUNDS, 32), (128, 64, dade.SCHED_SEEDED, 128),
                                                     (160, 16, dade.SCHED_ROUNDS, 64), (256, 64, dade.SCHED_ROUNDS, 7),
                                                     (384, 32, dade.SCHED_SEEDED, 128), (768, 32, dade.SCHED_ROUNDS, 64)])
def test_tensor_core_prefilter_equals_fp32(d, delta_d, schedule, tile):
    """List-major passes with the first increment's inner products on the
    tensor cores (FP32 rows read as TF32, certified bound): ids, distance bits
    and work counters equal the FP32 list-major path, the bound drops most
    candidates, and the results match the oracle."""
    n = 12000 if d <= 256 else 6000
    w = synth.Workload(f"tc{d}", n, d, 60, 1.2, 12, 0.0, 2.0, 1.0, False, True, 12, (4,), 10, (16,), 0.1,
                       comp_zipf=1.1, lists_are_components=True)
    base, queries, labels = synth.make(w)
    case = Case(base, queries, labels, 12, n_pairs=3000)
    nq = queries.shape[0]
    out = []
    for fl in (0, dade.FLAG_TC_PREFILTER):
        ids = torch.empty(nq, 10, dtype=torch.int64, device="cuda")
        dd = torch.empty(nq, 10, dtype=torch.float32, device="cuda")
        st = torch.zeros(nq, 4, dtype=torch.int64, device="cuda")
        ls = torch.full((nq,), -1, dtype=torch.int64, device="cuda") if fl else None
        case.gpu.search(case.q_rot, 10, 5, 0.1, delta_d, ids, dd, tile=tile, stats=st, schedule=schedule,
                        seed_lists=2, flags=fl, lead_stats=ls, list_chunk=256)
        case.gpu.sync()
        out.append((ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy(), None if ls is None else ls.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1].view(np.uint32), out[1][1].view(np.uint32))
    assert np.array_equal(out[0][2], out[1][2])
    assert (out[1][3] >= 0).all() and (out[1][3] <= out[1][2][:, 3]).all()
    assert out[1][3].sum() > 0.3 * out[1][2][:, 3].sum(), (out[1][3].sum(), out[1][2][:, 3].sum())
    sched = dade.SCHED_ROUNDS if schedule == dade.SCHED_ROUNDS else dade.SCHED_SEEDED
    o = case.oracle_search(10, 5, 0.1, delta_d, tile=tile, schedule=sched, seed=2 if sched == dade.SCHED_SEEDED else 0)
    parity.compare(out[1][0], out[1][1], o, case.exact_d)


def test_tensor_core_prefilter_integer_data_and_large_k():
    """The bound on 1M-style integer data far from the origin (large norms,
    small distances: the hardest case for the expanded form) and K = 100
    (accepted keys appended directly): the FP32 path's bits and counters."""
    w = synth.Workload("tcint", 20000, 128, 50, 1.0, 16, 40.0, 25.0, 20.0, True, False, 16, (4,), 100, (16,), 0.1)
    base, queries, labels = synth.make(w)
    ix = dade.Index(torch.from_numpy(base).cuda(), 16, assign=labels, eps_pairs=3000)
    q = torch.from_numpy(queries).cuda()
    out = []
    for fl in (0, dade.FLAG_TC_PREFILTER):
        for schedule in (dade.SCHED_SEEDED, dade.SCHED_ROUNDS):
            ids = torch.empty(50, 100, dtype=torch.int64, device="cuda")
            dd = torch.empty(50, 100, dtype=torch.float32, device="cuda")
            st = torch.zeros(50, 4, dtype=torch.int64, device="cuda")
            ix.query(q, 100, 6, 0.3, 64, ids, dd, stats=st, flags=fl, schedule=schedule, seed_lists=2, tile=128)
            ix.sync()
            out.append((ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy()))
    for a_, b_ in ((out[0], out[2]), (out[1], out[3])):
        assert np.array_equal(a_[0], b_[0]) and np.array_equal(a_[1].view(np.uint32), b_[1].view(np.uint32))
        assert np.array_equal(a_[2], b_[2])
