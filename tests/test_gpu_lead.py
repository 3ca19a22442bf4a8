"""Low-precision leading blocks (BF16 / FP8-e4m3 prefilter), GPU only.

The index may hold a BF16 or FP8 copy of the residuals o' - c' over its
leading dims, with per-vector error norms.  Two kinds of check:

* the build step against plain numpy definitions: BF16 codes are the
  round-to-nearest-even of the FP32 residual; FP8 scales are max|r| / 448 per
  (list, 16-dim block) and codes the nearest e4m3 value of r / s (ties to
  even, saturating at 448); every stored error norm bounds the true FP64
  error from above and is tight to FP32 rounding;
* the search: a search with the prefilter must return exactly what the FP32
  path returns (same ids, same distance bits, same per-query statistics) and
  match the FP64 oracle (tests/parity.py), while the prefilter actually drops
  candidates.
"""
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


def e4m3_grid():
    """Nonnegative finite e4m3 values, indexed by code 0..126 (bias 7, 3-bit
    mantissa, subnormals at exponent field 0; code 127 is NaN)."""
    v = []
    for code in range(127):
        e, m = code >> 3, code & 7
        v.append((m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(v)


def e4m3_round(x):
    """Nearest e4m3 value of float32 x, ties to the even code, |x| > 448 saturating."""
    g = e4m3_grid()
    ax = np.minimum(np.abs(x.astype(np.float64)), 448.0)
    hi = np.clip(np.searchsorted(g, ax), 1, len(g) - 1)
    lo = hi - 1
    dlo, dhi = ax - g[lo], g[hi] - ax
    pick = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(lo % 2 == 0, lo, hi)))
    return np.sign(x) * g[pick]


def bf16_round(x):
    """Round-to-nearest-even of float32 x to bfloat16, returned as float32."""
    b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


class LeadCase:
    def __init__(self, base, queries, assign, n_clusters, lead_format, lead_dims, n_pairs=20000):
        self.base, self.queries = base, queries
        self.assign = np.ascontiguousarray(assign, np.int32)
        self.nc = n_clusters
        self.pairs = synth.eps_pairs(base.shape[0], n_pairs, seed=4)
        self.orc = oracle.Index(base, n_clusters=n_clusters, assign=self.assign, pairs=self.pairs)
        self.gpu = dade.Index(torch.from_numpy(base).cuda(), n_clusters, assign=self.assign, pairs=self.pairs,
                              lead_format=lead_format, lead_dims=lead_dims)
        q = torch.from_numpy(queries).cuda()
        self.q_rot = torch.empty_like(q)
        self.gpu.rotate(q, self.q_rot)
        self.Qr = self.orc.rotate(queries)
        self.scale = float(np.mean((self.orc.Xr ** 2).sum(1)))

    def search(self, k, nprobe, alpha, delta_d, tile=128, flags=0, threads=0):
        nq = self.queries.shape[0]
        ids = torch.empty(nq, k, dtype=torch.int64, device="cuda")
        d = torch.empty(nq, k, dtype=torch.float32, device="cuda")
        st = torch.zeros(nq, 4, dtype=torch.int64, device="cuda")
        lead = torch.full((nq,), -1, dtype=torch.int64, device="cuda") if flags & dade.FLAG_LEAD else None
        self.gpu.search(self.q_rot, k, nprobe, alpha, delta_d, ids, d, tile=tile, stats=st, flags=flags,
                        threads=threads, lead_stats=lead)
        self.gpu.sync()
        return (ids.cpu().numpy(), d.cpu().numpy(), st.cpu().numpy(),
                lead.cpu().numpy() if lead is not None else None)

    def oracle_search(self, k, nprobe, alpha, delta_d, tile=128):
        eps = self.orc.eps(np.float32(alpha), delta_d)
        o = self.orc.o.search_bracket(self.orc.Xr, self.assign, self.orc.cent, self.orc.lam, self.Qr, k, nprobe,
                                      delta_d, eps, schedule=oracle.TILE, tile=tile, lag=0)
        pg = torch.empty(self.queries.shape[0], nprobe, dtype=torch.int32, device="cuda")
        self.gpu.probe(self.q_rot, nprobe, pg)
        self.gpu.sync()
        po, _ = self.orc.o.probe(self.Qr, self.orc.cent, nprobe)
        return o + ((pg.cpu().numpy() == po).all(1),)

    def exact_d(self, q, ids):
        return ((self.orc.Xr[ids] - self.Qr[q]) ** 2).sum(1)


_CASES = {}


def lead_case(name):
    """Shared, lazily built workloads: 10,000 x 128 Gaussian (specialised
    kernels) and 4,000 x 160 (generic kernel), each in BF16 and FP8."""
    if name not in _CASES:
        shape, fmt = name.split("-")
        lf = {"bf16": dade.LEAD_BF16, "fp8": dade.LEAD_FP8}[fmt]
        if shape == "d128":
            base, queries, _ = synth.make("c1_gauss_10k_d128")
            assign = synth.zipf_assign(base.shape[0], 64, s=0.6)
            _CASES[name] = LeadCase(base, queries, assign, 64, lf, 64)
        else:
            rng = np.random.default_rng(160)
            sd = np.arange(1, 161) ** -0.5
            base = (rng.standard_normal((4000, 160)) * sd).astype(np.float32)
            queries = (rng.standard_normal((60, 160)) * sd).astype(np.float32)
            assign = synth.zipf_assign(4000, 12, s=0.8)
            _CASES[name] = LeadCase(base, queries, assign, 12, lf, 48, n_pairs=5000)
    return _CASES[name]


@pytest.mark.parametrize("name", ["d128-bf16", "d128-fp8", "d160-bf16", "d160-fp8"])
def test_lead_codes_and_error_norms(name):
    c = lead_case(name)
    g = c.gpu
    info = g.info
    ld, nb = info.lead_dims, info.lead_dims // 16
    X = g.export(dade.FIELD_ROTATED)[:, :ld]
    C = g.export(dade.FIELD_CENTROIDS)[:, :ld]
    asg = g.export(dade.FIELD_ASSIGN)
    deq = g.export(dade.FIELD_LEAD_DEQ)
    err = g.export(dade.FIELD_LEAD_ERR)
    scale = g.export(dade.FIELD_LEAD_SCALE)
    r32 = X - C[asg]                                          # FP32 residual (one rounding)
    if info.lead_format == dade.LEAD_BF16:
        assert np.all(scale == 1.0)
        assert np.array_equal(deq, bf16_round(r32))
    else:
        amax = np.abs(r32).reshape(-1, nb, 16).max(2)
        exp_scale = np.ones((c.nc, nb), np.float32)
        for lst in range(c.nc):
            m = asg == lst
            if m.any():
                a = amax[m].max(0)
                exp_scale[lst] = np.where(a > 0, a / np.float32(448.0), np.float32(1.0))
        assert np.array_equal(scale, exp_scale)
        s = np.repeat(scale[asg], 16, axis=1)                 # per dim
        x = (r32 / s).astype(np.float32)
        assert np.array_equal(deq, (s * e4m3_round(x).astype(np.float32)).astype(np.float32))
    # error norms: cumulative over blocks, an upper bound, tight to FP32 rounding
    e = (X.astype(np.float64) - C[asg].astype(np.float64)) - deq.astype(np.float64)
    true = np.sqrt(np.cumsum((e ** 2).reshape(-1, nb, 16).sum(2), axis=1)).T   # [nb][n]
    assert np.all(err.astype(np.float64) >= true * (1 - 1e-12))
    assert np.all(err.astype(np.float64) <= true * (1 + 2.0 ** -22) + 1e-37)
    # the quantisation is tight enough for a useful prefilter
    rn = np.sqrt((r32.astype(np.float64) ** 2).sum(1))
    ratio = np.median(err[-1] / np.maximum(rn, 1e-30))
    assert ratio < (5e-3 if info.lead_format == dade.LEAD_BF16 else 0.1), ratio


@pytest.mark.parametrize("name", ["d128-bf16", "d128-fp8", "d160-bf16", "d160-fp8"])
@pytest.mark.parametrize("k,nprobe,alpha,delta_d,tile", [
    (10, 8, 0.05, 32, 128),
    (10, 8, 0.1, 16, 256),
    (100, 16, 0.2, 32, 64),
    (1, 4, 0.3, 48, 32),      # three blocks per increment: the generic kernel even at D = 128
    (20, 8, 0.1, 64, 128),
])
@pytest.mark.parametrize("threads,generic", [(128, False), (256, False), (128, True)])
def test_lead_search_equals_fp32_and_oracle(name, k, nprobe, alpha, delta_d, tile, threads, generic):
    c = lead_case(name)
    if delta_d > c.gpu.info.lead_dims or nprobe > c.nc:
        pytest.skip("configuration outside this index's lead copy")
    base_flags = dade.FLAG_GENERIC_KERNEL if generic else 0
    f_ids, f_d, f_st, _ = c.search(k, nprobe, alpha, delta_d, tile=tile, flags=base_flags, threads=threads)
    l_ids, l_d, l_st, l_lead = c.search(k, nprobe, alpha, delta_d, tile=tile, flags=base_flags | dade.FLAG_LEAD,
                                        threads=threads)
    # identical to the FP32 path: ids, distance bits and the work counted
    assert np.array_equal(l_ids, f_ids)
    assert np.array_equal(l_d.view(np.uint32), f_d.view(np.uint32))
    assert np.array_equal(l_st, f_st)
    # the prefilter drops only candidates the exact first test prunes, and some
    n_inc = -(-c.gpu.info.d_pad // delta_d)
    assert np.all(l_lead >= 0)
    if n_inc > 1:
        assert np.all(l_lead <= l_st[:, 3])
    assert l_lead.sum() > 0.05 * l_st[:, 0].sum()
    # and parity with the FP64 oracle
    o = c.oracle_search(k, nprobe, alpha, delta_d, tile=tile)
    parity.compare(l_ids, l_d, o, c.exact_d)
    parity.compare_stats(l_st, o)


def test_lead_whole_vector_single_increment():
    """delta_d >= D: one increment, the prefilter bounds the full distance
    against r^2 itself; survivors get the exact compare."""
    c = lead_case("d160-bf16")
    # lead_dims 48 < D: a single increment needs the whole vector, so it is refused
    with pytest.raises(dade.DadeError) as e:
        c.search(10, 4, 0.1, 1024, flags=dade.FLAG_LEAD)
    assert e.value.status == dade.EINVAL
    rng = np.random.default_rng(7)
    base = (rng.standard_normal((3000, 40)) * np.linspace(2.0, 0.3, 40)).astype(np.float32)
    queries = (rng.standard_normal((30, 40)) * np.linspace(2.0, 0.3, 40)).astype(np.float32)
    assign = synth.zipf_assign(3000, 6, s=0.5)
    case = LeadCase(base, queries, assign, 6, dade.LEAD_BF16, 48, n_pairs=3000)
    for k, nprobe in ((10, 2), (50, 6)):
        f = case.search(k, nprobe, 0.1, 1024)
        l = case.search(k, nprobe, 0.1, 1024, flags=dade.FLAG_LEAD)
        assert np.array_equal(l[0], f[0]) and np.array_equal(l[1].view(np.uint32), f[1].view(np.uint32))
        assert np.array_equal(l[2], f[2])
        assert l[3].sum() > 0
        o = case.oracle_search(k, nprobe, 0.1, 1024)
        parity.compare(l[0], l[1], o, case.exact_d)


def test_lead_invalid_requests():
    c = lead_case("d128-bf16")
    nq = c.queries.shape[0]
    ids = torch.empty(nq, 10, dtype=torch.int64, device="cuda")
    d = torch.empty(nq, 10, dtype=torch.float32, device="cuda")
    bad = [
        dict(delta_d=128, flags=dade.FLAG_LEAD),                                    # beyond lead_dims = 64
        dict(delta_d=32, flags=dade.FLAG_LEAD, schedule=dade.SCHED_PIPELINED),
        dict(delta_d=32, flags=dade.FLAG_LEAD, mode=dade.MODE_FD),
        dict(delta_d=32, flags=0, lead_stats=torch.zeros(nq, dtype=torch.int64, device="cuda")),
        dict(delta_d=32, flags=8),
    ]
    for kw in bad:
        dd = kw.pop("delta_d")
        with pytest.raises(dade.DadeError) as e:
            c.gpu.search(c.q_rot, 10, 8, 0.1, dd, ids, d, **kw)
        assert e.value.status == dade.EINVAL, kw
    # an index without a lead copy refuses the flag
    g = dade.Index(torch.from_numpy(c.base).cuda(), c.nc, assign=c.assign, eps_pairs=1000)
    with pytest.raises(dade.DadeError) as e:
        g.search(c.q_rot, 10, 8, 0.1, 32, ids, d, flags=dade.FLAG_LEAD)
    assert e.value.status == dade.EINVAL
