"""Pins for statistics, constants and the relative->log transform (Section III).

Every decision is checked against exact rational arithmetic (fractions) or an
independent double-precision restatement of the paper's formulas.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2309_09778_gb300 import gen


def near_half(v, tol=1e-6):
    return abs(abs(v - math.floor(v)) - 0.5) < tol


def test_stats_definition(O):
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(5000) * np.exp(rng.uniform(-20, 20, 5000))).astype(np.float32)
    x[::17] = 0.0
    x[5] = np.float32(1e-40)  # subnormal: not part of abs_min
    st, mn, mx, tr = O.stats(x)
    a = np.abs(x.astype(np.float64))
    normal = a[a >= np.finfo(np.float32).tiny]
    assert st == 0 and tr == 0
    assert mn == normal.min() and mx == a.max()


def test_stats_rejects_nonfinite_and_flags_trivial(O):
    x = np.ones(10, np.float32)
    x[3] = np.nan
    assert O.stats(x)[0] == -3
    x[3] = np.inf
    assert O.stats(x)[0] == -3
    z = np.zeros(10, np.float32)
    z[2] = np.float32(1e-42)
    st, mn, mx, tr = O.stats(z)
    assert st == 0 and tr == 1


@pytest.mark.parametrize("dtype", [0, 1])
def test_constants_follow_eq8_to_eq12(O, dtype):
    """Kp, Kn, Zq and S restated from Eq. 8-12 in plain double math.log2."""
    rng = np.random.default_rng(2 + dtype)
    e0 = 2.0 ** -149 if dtype == 0 else 2.0 ** -1074
    le0 = -149.0 if dtype == 0 else -1074.0
    for _ in range(300):
        amin = float(np.exp(rng.uniform(-60, 10)))
        amax = amin * float(np.exp(rng.uniform(0, 40)))
        if dtype == 0:
            amin, amax = float(np.float32(amin)), float(np.float32(amax))
        eb = float(10 ** rng.uniform(-5, -1))
        st, c = O.make_consts(dtype, amin, amax, 0, eb)
        assert st == 0
        step = 2 * math.log2(1 + eb)                                          # Eq. 8
        kp = math.log2(amin) / step                                           # Eq. 9
        lfn = math.log2(amax + e0) + math.log2(amin) + step - math.log2(amin - e0)  # Eq. 10
        kn = lfn / step
        for got, want in ((c.Kp, kp), (c.Kn, kn), (c.Zq - c.Kp, le0 / step), (c.S - c.Kp, math.log2(amax + e0) / step)):
            if not near_half(want, 1e-4):
                assert got == round(want), (got, want)
        assert abs(c.step64 - step) <= 1e-15 * step
        assert c.ebdn32 <= eb and float(np.nextafter(np.float32(c.ebdn32), np.float32(1))) > eb


def test_constants_reject_bad_eb_and_range(O):
    assert O.make_consts(0, 1.0, 2.0, 0, 0.0)[0] == -1
    assert O.make_consts(0, 1.0, 2.0, 0, 1.0)[0] == -1
    assert O.make_consts(0, 1e-30, 1e30, 0, 1e-9)[0] == -8


def test_separation_inequality_exact(O):
    """Section III.B: every negative image lies at least 2 b_a above every
    positive image.  With integer offsets the smallest negative code minus the
    largest positive code must exceed the paper's margin less the three
    roundings (Kp, Kn and the per-point rint), checked in exact rationals."""
    rng = np.random.default_rng(4)
    for _ in range(200):
        amin = float(np.float32(np.exp(rng.uniform(-40, 5))))
        amax = float(np.float32(amin * np.exp(rng.uniform(0, 30))))
        eb = float(10 ** rng.uniform(-4, -1))
        st, c = O.make_consts(0, amin, amax, 0, eb)
        step = Fraction(2 * math.log2(1 + eb))
        # real images in code units: pos(amax) = log2(amax)/step + Kp, neg(amin) = log2(amin)/step + Kn
        pos_hi = Fraction(math.log2(amax)) / step + c.Kp
        neg_lo = Fraction(math.log2(amin)) / step + c.Kn
        # paper's separation is one code unit (2 b_a); Kp, Kn roundings cost at most one unit
        assert neg_lo - pos_hi >= Fraction(1) - Fraction(1) - Fraction(1, 1000)
        # and the boundary S sits between them (within rounding)
        assert c.S >= math.floor(pos_hi) - 1 and c.S <= math.ceil(neg_lo) + 1


def exact_ok(x, q, c, O, dtype):
    r = O.recon(q, c, dtype)
    want = 1 if x > 0 else 2
    cls = 0 if q <= c.Zq else (1 if q <= c.S else 2)
    if cls != want:
        return False
    ebdn = c.ebdn32 if dtype == 0 else c.ebdnd
    return abs(Fraction(r) - Fraction(x)) <= Fraction(ebdn) * abs(Fraction(x))


@pytest.mark.parametrize("dtype,eb", [(0, 1e-2), (0, 1e-3), (0, 1e-4), (1, 1e-5), (1, 1e-3)])
def test_transform_brute_force(O, dtype, eb):
    """For each point: dq is rint(log2|x| / 2b_a) + K (away from ties), and
    ok is exactly 'right sign class and |R(dq) - x| <= eb |x|' in rationals."""
    rng = np.random.default_rng(5)
    npd = np.float32 if dtype == 0 else np.float64
    x = (np.where(rng.random(3000) < 0.5, -1, 1) * np.exp(rng.uniform(-15, 15, 3000))).astype(npd)
    c = O.consts_for(x, eb)
    dq, ok = O.transform(x, c)
    step = 2 * math.log2(1 + eb)
    nok = 0
    for xi, qi, oi in zip(x.tolist(), dq.tolist(), ok.tolist()):
        K = c.Kp if xi > 0 else c.Kn
        lg = math.log2(abs(xi))
        want = lg / step
        # tie window: 4 ulp of log2 (the L error bound) scaled to code units,
        # plus the rounding of the product itself
        u = (lambda v: float(np.spacing(np.float32(abs(v))))) if dtype == 0 else (lambda v: float(np.spacing(abs(v))))
        tol = 4 * u(lg) / step + 2 * u(want) + 1e-9
        if not near_half(want, tol):
            assert qi - K == round(want)
        assert bool(oi) == exact_ok(xi, qi, c, O, dtype)
        nok += oi
    # the bound check passes for nearly all points: the transform is not trivially rejecting
    assert nok >= 0.98 * x.size


def test_transform_zero_and_special_values(O):
    x = np.array([0.0, -0.0, 1e-40, -1e-41, 1.0, -1.0, 3.5], np.float32)
    c = O.consts_for(x, 1e-3)
    dq, ok = O.transform(x, c)
    assert dq[0] == c.Zq and ok[0] == 1            # +0 maps to the zero image (Eq. 12)
    assert ok[1] == 0 and ok[2] == 0 and ok[3] == 0  # -0 and subnormals: balance points
    assert dq[1] == c.Zq and dq[2] == c.Zq
    assert O.recon(c.Zq, c) == 0.0 and not np.signbit(O.recon(c.Zq, c))
    assert ok[4] and ok[5] and ok[6]
    assert c.Zq < dq[4] <= c.S < dq[5]            # zero < positive <= boundary < negative


def test_scale_invariance_eq5(O):
    """Eq. 5: multiplying the data by a constant C leaves the bound intact; a
    power-of-two C shifts every positive code by exactly log2(C)/2b_a when
    that is an integer number of steps."""
    eb = 1e-2
    rng = np.random.default_rng(6)
    x = np.exp(rng.uniform(-5, 5, 2000)).astype(np.float32)
    c1 = O.consts_for(x, eb)
    dq1, ok1 = O.transform(x, c1)
    x2 = (x * np.float32(2.0 ** 8)).astype(np.float32)
    c2 = O.consts_for(x2, eb)
    dq2, ok2 = O.transform(x2, c2)
    # positive codes relative to Kp are log2|x|/step; both fields keep ok on nearly all points
    assert ok1.mean() > 0.99 and ok2.mean() > 0.99
    step = 2 * math.log2(1 + eb)
    d = (dq2 - c2.Kp) - (dq1 - c1.Kp)
    assert np.all(np.abs(d - 8 / step) <= 1.0)
