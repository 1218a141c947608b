"""Pins for the oracle's fixed-point (BF16) perceptron form.

The form: weights are integers |W| <= 255 times 2^-e per layer (exact bf16
values), stencil inputs integers clamped to +-(2^16 - 1), hidden activations
integers clamped to +-(2^15 - 1) after a leaky ReLU (slope 2^-4) and a
round-half-up shift by t >= 0, prediction = rne(A_out 2^-F) with
F = sum e - sum t.  These tests hold the oracle to
  - the exactness claim behind the tensor-core evaluation: splitting inputs
    and activations into signed 8-bit limbs keeps every FP32 partial sum of
    limb products exact, in any order;
  - the rational value of the network when quantization loses nothing
    (the unit bookkeeping of e, t, s_in and the biases);
  - round-half-even shifts against exact fractions;
  - the container round trip with the error bound on every point.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2309_09778_gb300 import gen


def limbs(v, base=256):
    """8-bit limbs: v = base * hi + lo with 0 <= lo < base (floor division)."""
    v = np.asarray(v, np.int64)
    return v // base, v % base


def f32_sum(products, rng):
    """Sum float32 products in a random order with float32 rounding."""
    p = np.asarray(products, np.float32)[rng.permutation(len(products))]
    s = np.float32(0)
    for t in p:
        s = np.float32(s + t)
    return s


@pytest.mark.parametrize("K,lim", [(7, 65535), (13, 65535), (16, 32767), (32, 32767)])
def test_limb_products_accumulate_exactly_in_fp32(K, lim):
    """Each limb's products are bf16 x bf16 (exact in FP32) and their sums stay
    below 2^24, so any FP32 accumulation order gives the exact integer."""
    rng = np.random.default_rng(K)
    for _ in range(300):
        w = rng.integers(-255, 256, K)
        x = rng.integers(-lim, lim + 1, K)
        x[rng.random(K) < 0.2] = lim * rng.choice([-1, 1])
        hi, lo = limbs(x)
        assert np.all(np.abs(hi) <= 256) and np.all((lo >= 0) & (lo <= 255))
        s_hi = f32_sum(w * hi, rng)
        s_lo = f32_sum(w * lo, rng)
        assert abs(float(s_hi)) < 2 ** 24 and abs(float(s_lo)) < 2 ** 24
        assert 256 * int(s_hi) + int(s_lo) == int(np.dot(w, x))


def rhu_shift(x: int, s: int) -> int:
    """floor(x 2^-s + 1/2)"""
    f = Fraction(x, 2 ** s) + Fraction(1, 2)
    return f.numerator // f.denominator


def rne_shift(x: int, s: int) -> int:
    f = Fraction(x, 2 ** s) if s >= 0 else Fraction(x * 2 ** (-s))
    fl = f.numerator // f.denominator
    r = f - fl
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return int(fl)


def test_quantized_net_equals_rational_value_when_lossless(O):
    """One hidden layer whose weights and biases are exactly representable,
    pre-activations multiples of 16 (so the leaky slope 1/16 is exact) and
    inputs small enough that the chosen shift t1 = 0: no step loses
    information, so the fixed-point prediction is the round-half-even of the
    FP32 network's exact value.  This pins the units of e, t, s_in, the
    biases and F."""
    rng = np.random.default_rng(3)
    k, h1, h2 = 7, 16, 0
    nw = O.mlp_nweights(k, h1, h2)
    checked = 0
    for trial in range(40):
        s_in = int(rng.integers(0, 4))
        W1 = rng.integers(-8, 9, (h1, k)).astype(np.float64) / 8       # max |W1| = 1 -> e1 = 7
        W1[0, 0] = 1.0
        b1 = 16 * rng.integers(-20, 21, h1).astype(np.float64) / 2 ** (7 + s_in)
        Wo = rng.integers(-8, 9, h1).astype(np.float64) / 4             # max |Wo| = 2 -> e2 = 6
        Wo[0] = 2.0
        bo = float(rng.integers(-20, 21)) / 4
        w = np.concatenate([W1.ravel(), b1, Wo, [bo]]).astype(np.float32)
        assert w.size == nw
        tin = rng.integers(-2, 3, (100, k)).astype(np.int32)
        q = O.qnet_build(w, k, h1, h2, s_in, tin, np.ones(100, np.uint8))
        assert (int(q[4]), int(q[5])) == (7, 6)
        if int(q[7]) != 0:
            continue
        for v in tin[:30]:
            u = [Fraction(int(a), 2 ** s_in) for a in v]
            a1 = [sum(Fraction(W1[j, i]) * u[i] for i in range(k)) + Fraction(b1[j]) for j in range(h1)]
            a1 = [a if a >= 0 else a / 16 for a in a1]
            out = (sum(Fraction(Wo[j]) * a1[j] for j in range(h1)) + Fraction(bo)) * 2 ** s_in
            fl = out.numerator // out.denominator
            r = out - fl
            want = fl + (1 if (r > Fraction(1, 2) or (r == Fraction(1, 2) and fl % 2)) else 0)
            assert O.mlp_pred_q(q, v) == want, (trial, int(q[7]))
            checked += 1
    assert checked >= 300


def test_rne_shift_matches_fractions(O):
    """The prediction's final shift: a one-weight network passes A through."""
    rng = np.random.default_rng(4)
    k, h1, h2 = 7, 2, 0
    n = O.qnet_len(k, h1, h2)
    for _ in range(400):
        q = np.zeros(n, np.int64)
        q[:9] = [k, h1, h2, 0, 0, 0, 0, 0, 0]
        F = int(rng.integers(-3, 12))
        # e1 + e2 - t1 = F with t1 = 0
        q[4], q[5] = F, 0
        # unit 0 passes input 0 through (weight 1), output weight 1, bias 0
        q[9 + 0] = 1
        q[9 + h1 * k + h1 + 0] = 1
        v = np.zeros(k, np.int32)
        x = int(rng.integers(0, 30000))
        v[0] = x
        want = rne_shift(x, F)
        want = max(min(want, 2 ** 30), -2 ** 30)
        assert O.mlp_pred_q(q, v) == want, (x, F)


def test_leaky_requant_uses_slope_and_rounds_half_up(O):
    """Negative pre-activations are divided by 16 before the shift; halves round up."""
    k, h1, h2 = 7, 2, 0
    n = O.qnet_len(k, h1, h2)
    for x in (-1, -8, -24, -40, -1000, 8, 24, 37, -7, -9):
        for t in (0, 1, 3):
            q = np.zeros(n, np.int64)
            q[:9] = [k, h1, h2, 0, 0, t, 0, t, 0]   # e1 = 0, e2 = t, t1 = t: F = 0
            q[9] = 1                                 # unit 0 = input 0
            q[9 + h1 * k + h1] = 1                   # output = unit 0
            v = np.zeros(k, np.int32); v[0] = x
            h = rhu_shift(x, t) if x >= 0 else rhu_shift(x, t + 4)
            h = max(min(h, 32767), -32767)
            assert O.mlp_pred_q(q, v) == h, (x, t)


def test_input_and_activation_clamps(O):
    k, h1, h2 = 7, 2, 0
    q = np.zeros(O.qnet_len(k, h1, h2), np.int64)
    q[:9] = [k, h1, h2, 0, 0, 0, 0, 0, 0]
    q[9] = 1
    q[9 + h1 * k + h1] = 1
    v = np.zeros(k, np.int32)
    v[0] = 10 ** 6                  # input clamp 65535, then activation clamp 32767
    assert O.mlp_pred_q(q, v) == 32767
    v[0] = -10 ** 6                 # -65535 / 16 = -4095.9375, half up -> -4096
    assert O.mlp_pred_q(q, v) == -4096


def test_quantized_prediction_close_to_fp32(O):
    """On a trained network the fixed-point prediction stays near the FP32 one."""
    x = gen.positive_lognormal((24, 40, 40), 3.0, 5, 1.5)
    best, W, s_in, costs = O.train(x, 1e-3, block=(8, 8, 8), k=7, h1=16, h2=16, seed=0)
    w = W[best if best >= 0 else 0]
    q = O.quantize(x, 1e-3, w, s_in)
    rng = np.random.default_rng(5)
    diffs = []
    for _ in range(400):
        v = rng.integers(-300, 300, 7).astype(np.int32)
        diffs.append(abs(O.mlp_pred_q(q, v) - O.mlp_pred32(w, 7, 16, 16, s_in, v)))
    diffs = np.array(diffs)
    assert np.median(diffs) <= 1 and diffs.max() <= 8


def test_fixed_point_container_round_trip(O):
    x = gen.signed_lognormal((20, 21, 22), 3.5, 11, 2.5, 0.05)
    best, W, s_in, _ = O.train(x, 1e-2, block=(8, 8, 8), k=7, h1=16, h2=16, seed=1)
    w = W[best if best >= 0 else 0]
    q = O.quantize(x, 1e-2, w, s_in, seed=1)
    st, blob, d = O.compress(x, 1e-2, qnet=q, s_in=s_in, dump=True)
    assert st == 0
    st, y = O.decompress(blob)
    assert st == 0
    xd = x.astype(np.float64)
    assert np.all(np.abs(y.astype(np.float64) - xd) <= 1e-2 * np.abs(xd))
    assert np.array_equal(np.signbit(x), np.signbit(y))


def test_fixed_point_container_rejects_bad_network(O):
    x = gen.positive_lognormal((16, 16, 16), 3.0, 2, 1.0)
    best, W, s_in, _ = O.train(x, 1e-2, block=(8, 8, 8), k=7, h1=16, h2=16, seed=2)
    q = O.quantize(x, 1e-2, W[max(best, 0)], s_in, seed=2)
    st, blob = O.compress(x, 1e-2, qnet=q, s_in=s_in)
    assert st == 0
    import struct
    off_w = struct.unpack_from("<Q", blob, 168)[0]
    bad = bytearray(blob)
    struct.pack_into("<q", bad, off_w + 8 * 9, 300)      # |W| > 255
    assert O.decompress(bytes(bad))[0] == -5
    bad = bytearray(blob)
    struct.pack_into("<q", bad, off_w + 8 * 7, 99)       # shift out of range
    assert O.decompress(bytes(bad))[0] == -5
