"""The certified margin of the low-precision prefilter (lead_prunes), on the CPU.

The prefilter drops a candidate at the first increment when

    L = sqrtf(p_lead) (1 - 2^-16) - e - 2^-20 qcn   and   L^2 > thr (1 + 2^-15),

where p_lead is the FP32 sum of squares of (q' - c') - dequant(code) over the
increment's n dims, e the stored error norm ||(o' - c') - dequant|| (FP64 from
exact differences, rounded up), qcn = sqrtf(FP32 ||q' - c'||^2) and thr the
FP32 threshold coef_d r^2 of the Section 3.3 test.  It must drop only
candidates whose FP32 partial distance P (the exact path's own sum) exceeds
thr, so that results stay those of the FP32 path.  With u = 2^-24 and every
FP32 sum of the kernels taking at most m = n/16 + 6 roundings along any path
(4 in a lane's 4-term FMA chain, one per 16-dim block added, two shuffle
adds), the three constants are safe when (gamma_k = k u / (1 - k u)):

  R1  2^-16 >= 3u + gamma_{m+2} / 2 + 2^-42     (sqrtf, the FP32 sum of p_lead,
        the rounding of (q' - c') - dequant, the FP64 accumulation of e)
  R2  2^-20 >= u (1 + 2u + gamma_m)              (the rounding of q' - c')
  R3  2^-15 >= 8u + gamma_{m+2}                  (forming L and L^2, rounding
        thr (1 + 2^-15), and the FP32 path's own sum P >= (1 - 2u - gamma_{m+2}) P_exact)

This file checks R1-R3 in exact rational arithmetic for every n = 16 ..
1024 (the largest increment), and then runs the kernel's arithmetic,
operation by operation, in FP32 on random and near-threshold candidates at
scales 2^-20 .. 2^20: every candidate the emulated prefilter drops is pruned
by the emulated FP32 test.
"""
from fractions import Fraction as F

import numpy as np
import pytest

U = F(1, 2 ** 24)


def gamma(k):
    return k * U / (1 - k * U)


@pytest.mark.parametrize("n", list(range(16, 1025, 16)))
def test_margin_inequalities(n):
    m = n // 16 + 6
    assert F(1, 2 ** 16) >= 3 * U + gamma(m + 2) / 2 + F(1, 2 ** 42), n
    assert F(1, 2 ** 20) >= U * (1 + 2 * U + gamma(m)), n
    assert F(1, 2 ** 15) >= 8 * U + gamma(m + 2), n


# ---- FP32 emulation of the kernel arithmetic ------------------------------------------
f32 = np.float32


def _fma(a, b, c):
    """fmaf: one rounding of a b + c (a b is exact in FP64; the FP64 sum
    rounds at most once more, far below the margins tested)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def _lane_quad_sum(x):
    """The kernels' sum of squares of x [..., n] (n a multiple of 16): lane lq
    takes dims 16 b + 4 lq .. + 3 of every block b, each block as
    fma(a, a, fma(b, b, fma(c, c, e e))), blocks added in order; then the two
    shuffle adds (lanes 0+1, 2+3, then both)."""
    n = x.shape[-1]
    lanes = []
    for lq in range(4):
        p = np.zeros(x.shape[:-1], f32)
        for b in range(n // 16):
            v = x[..., 16 * b + 4 * lq: 16 * b + 4 * lq + 4]
            s = (v[..., 3] * v[..., 3]).astype(f32)
            s = _fma(v[..., 2], v[..., 2], s)
            s = _fma(v[..., 1], v[..., 1], s)
            s = _fma(v[..., 0], v[..., 0], s)
            p = (p + s).astype(f32)
        lanes.append(p)
    return ((lanes[0] + lanes[1]).astype(f32) + (lanes[2] + lanes[3]).astype(f32)).astype(f32)


def _qn_sum(v):
    """qn of the tile kernel: per lane fma(x, x, fma(y, y, fma(z, z, fma(w, w, qn)))) over the blocks."""
    n = v.shape[-1]
    lanes = []
    for lq in range(4):
        qn = np.zeros(v.shape[:-1], f32)
        for b in range(n // 16):
            w4 = v[..., 16 * b + 4 * lq: 16 * b + 4 * lq + 4]
            qn = _fma(w4[..., 3], w4[..., 3], qn)
            qn = _fma(w4[..., 2], w4[..., 2], qn)
            qn = _fma(w4[..., 1], w4[..., 1], qn)
            qn = _fma(w4[..., 0], w4[..., 0], qn)
        lanes.append(qn)
    return ((lanes[0] + lanes[1]).astype(f32) + (lanes[2] + lanes[3]).astype(f32)).astype(f32)


def _bf16(x):
    """Round-to-nearest-even to bfloat16, returned as float32 (exact widening)."""
    b = x.astype(f32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(f32)


def _lead_prunes(p, e, qcn, thr, contract):
    s = np.sqrt(p.astype(np.float64)).astype(f32)                  # sqrtf, correctly rounded
    c = f32(1.0 - 2.0 ** -16)
    a = _fma(s, np.full_like(s, c), -e) if contract else ((s * c).astype(f32) - e).astype(f32)
    L = (a - (qcn * f32(2.0 ** -20)).astype(f32)).astype(f32)
    lb = np.where(L > 0, (L * L).astype(f32), f32(0))
    return lb > (thr * f32(1.0 + 2.0 ** -15)).astype(f32)


@pytest.mark.parametrize("n", [16, 32, 64, 256, 1024])
@pytest.mark.parametrize("scale_exp", [-20, 0, 20])
@pytest.mark.parametrize("contract", [False, True])
def test_prefilter_drops_only_what_fp32_prunes(n, scale_exp, contract):
    rng = np.random.default_rng(n * 7 + scale_exp + 100 * contract)
    s = 2.0 ** scale_exp
    cnt = 4000
    cen = (rng.standard_normal(n) * s).astype(f32)
    q = (cen + rng.standard_normal(n) * s * 0.5).astype(f32)
    o = (cen[None, :] + rng.standard_normal((cnt, n)) * s * rng.uniform(0.05, 1.0, (cnt, 1))).astype(f32)
    # the FP32 path: P = sum of fl(q' - o')^2 in the kernels' order
    P = _lane_quad_sum((q[None, :] - o).astype(f32))
    # the prefilter: BF16 residual codes, exact error norm rounded up
    r = (o - cen[None, :]).astype(f32)
    rq = _bf16(r)
    err = ((o.astype(np.float64) - cen.astype(np.float64)) - rq.astype(np.float64))
    e = np.nextafter(np.sqrt((err ** 2).sum(1)).astype(f32), f32(np.inf))
    qc = (q - cen).astype(f32)
    p_lead = _lane_quad_sum((qc[None, :] - rq).astype(f32))
    qcn = np.sqrt(_qn_sum(qc[None, :]).astype(np.float64)).astype(f32)
    # thresholds: every candidate once just below its own P (the hardest case), and a spread
    for thr in (np.nextafter(P, f32(0)), (P * f32(1.0 - 2.0 ** -13)).astype(f32),
                (P * rng.uniform(0.5, 1.5, cnt)).astype(f32)):
        drop = _lead_prunes(p_lead, e, qcn, thr, contract)
        assert not np.any(drop & ~(P > thr)), "the prefilter dropped a candidate the FP32 test keeps"
    # and it is not vacuous: far above the threshold it drops
    drop = _lead_prunes(p_lead, e, qcn, (P * f32(0.5)).astype(f32), contract)
    assert drop.mean() > 0.9
