"""The ADSampling comparator (GPU only): an index over a random orthogonal
basis and the sqrt(D/d) estimate with the eps0 test, against the oracle run
with a uniform spectrum and eps_d = eps0 / sqrt(d) over the same basis."""
import numpy as np
import pytest

import oracle
import parity
from paper_2411_17229_gb300 import dade, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_17229_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def case():
    base, queries, _ = synth.make("c1_gauss_10k_d128")
    W = synth.haar(128, np.random.default_rng(123))
    assign = np.ascontiguousarray(synth.zipf_assign(base.shape[0], 64, s=0.6), np.int32)
    g = dade.Index(torch.from_numpy(base).cuda(), 64, assign=assign, eps_pairs=2000, basis=W)
    o = oracle.get()
    mu, _ = o.mean_cov(base)
    Xr = o.rotate(base, mu, W)
    Qr = o.rotate(queries, mu, W)
    cent = o.list_means(Xr, assign, 64)
    q_rot = torch.empty(queries.shape[0], 128, device="cuda")
    g.rotate(torch.from_numpy(queries).cuda(), q_rot)
    scale = float(np.mean((Xr ** 2).sum(1)))
    return dict(g=g, o=o, W=W, Xr=Xr, Qr=Qr, cent=cent, assign=assign, q_rot=q_rot, scale=scale, base=base)


def test_given_basis_is_kept(case):
    W = case["g"].export(dade.FIELD_BASIS)
    assert np.abs(W - case["W"]).max() < 1e-12
    lam = case["g"].export(dade.FIELD_EIGVAL)
    _, C = case["o"].mean_cov(case["base"])
    ref = np.einsum("jk,ji,ik->k", case["W"], C, case["W"])
    assert np.allclose(lam, ref, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("k,nprobe,eps0,delta_d", [(10, 8, 2.1, 32), (10, 8, 1.0, 16), (100, 16, 3.0, 64)])
@pytest.mark.parametrize("schedule,seed", [(dade.SCHED_TILE, 0), (dade.SCHED_SEEDED, 2)])
def test_adsampling_parity(case, k, nprobe, eps0, delta_d, schedule, seed):
    c = case
    nq = c["Qr"].shape[0]
    ids = torch.empty(nq, k, dtype=torch.int64, device="cuda")
    d = torch.empty(nq, k, dtype=torch.float32, device="cuda")
    st = torch.zeros(nq, 4, dtype=torch.int64, device="cuda")
    c["g"].search(c["q_rot"], k, nprobe, 0.5, delta_d, ids, d, stats=st, estimator=dade.ESTIMATOR_ADSAMPLING,
                  eps0=eps0, schedule=schedule, seed_lists=seed)
    c["g"].sync()
    eps = np.full(129, np.nan)
    for dd in oracle.increments(128, delta_d):
        eps[dd] = np.float32(eps0) / np.sqrt(dd)
    o = c["o"].search_bracket(c["Xr"], c["assign"], c["cent"], np.ones(128), c["Qr"], k, nprobe,
                              delta_d, eps, schedule=oracle.TILE, tile=128, seed=seed)
    exact = lambda q, sel: ((c["Xr"][sel] - c["Qr"][q]) ** 2).sum(1)
    pg = torch.empty(nq, nprobe, dtype=torch.int32, device="cuda")
    c["g"].probe(c["q_rot"], nprobe, pg)
    c["g"].sync()
    po, _ = c["o"].probe(c["Qr"], c["cent"], nprobe)
    parity.compare(ids.cpu().numpy(), d.cpu().numpy(), o, exact, same_probe=(pg.cpu().numpy() == po).all(1))
    g_st = st.cpu().numpy()
    parity.compare_stats(g_st, o)
    assert g_st[:, 3].sum() > 0   # the test prunes


def test_random_transform_is_orthonormal():
    base, _, _ = synth.make("c1_gauss_10k_d128", n=3000, nq=1)
    g = dade.Index(torch.from_numpy(base).cuda(), 8, kmeans_iters=1, eps_pairs=500, transform=dade.TRANSFORM_RANDOM,
                   seed=9)
    W = g.export(dade.FIELD_BASIS)
    assert np.abs(W.T @ W - np.eye(128)).max() < 1e-12
    g2 = dade.Index(torch.from_numpy(base).cuda(), 8, kmeans_iters=1, eps_pairs=500, transform=dade.TRANSFORM_RANDOM,
                    seed=9)
    assert np.array_equal(W, g2.export(dade.FIELD_BASIS))   # seeded
    with pytest.raises(dade.DadeError) as e:
        dade.Index(torch.from_numpy(base).cuda(), 8, kmeans_iters=1, eps_pairs=500, basis=np.ones((128, 128)))
    assert e.value.status == dade.EINVAL
