"""Pins for the FP64 reporting predictor (the same FP32 weights evaluated in
double precision) and the prediction-error report built on it.

The FP64 form is held to an independent float64 evaluation written here with
numpy (no fused multiply-add: the two may differ by a few ulp of double, far
below the rounding to an integer code), to the Lorenzo-equal initialisation,
and to the container round trip with the bound on every point.  The report is
held to counts and sums recomputed from the oracle's own per-point
predictions on a small field, and to the special case of a network that
predicts like Lorenzo.
"""
import numpy as np
import pytest

from paper_2309_09778_gb300 import gen


def np_mlp64(w, k, h1, h2, s_in, v):
    w = w.astype(np.float64)
    u = v.astype(np.float64) * 2.0 ** -s_in
    p = 0
    W1 = w[p:p + h1 * k].reshape(h1, k); p += h1 * k
    b1 = w[p:p + h1]; p += h1
    a = W1 @ u + b1
    a = np.where(a >= 0, a, a * 0.0625)
    if h2:
        W2 = w[p:p + h2 * h1].reshape(h2, h1); p += h2 * h1
        b2 = w[p:p + h2]; p += h2
        a = W2 @ a + b2
        a = np.where(a >= 0, a, a * 0.0625)
    hl = h2 if h2 else h1
    return float((w[p:p + hl] @ a + w[p + hl]) * 2.0 ** s_in)


@pytest.mark.parametrize("k,h1,h2", [(7, 16, 16), (13, 32, 32), (7, 2, 0)])
def test_fp64_forward_matches_numpy(O, k, h1, h2):
    rng = np.random.default_rng(k * 7 + h1)
    nw = O.mlp_nweights(k, h1, h2)
    for _ in range(200):
        w = (rng.standard_normal(nw) * 0.3).astype(np.float32)
        s_in = int(rng.integers(0, 8))
        v = rng.integers(-5000, 5000, k).astype(np.int32)
        got = O.mlp_fwd64(w, k, h1, h2, s_in, v)
        want = np_mlp64(w, k, h1, h2, s_in, v)
        assert abs(got - want) <= 1e-12 * (1.0 + abs(want)) * 2.0 ** s_in * (1 + np.abs(v).max())
        # the FP32 form differs from it only by single-precision rounding
        got32 = O.mlp_fwd32(w, k, h1, h2, s_in, v)
        assert abs(got32 - want) <= 1e-4 * (1.0 + abs(want)) * (1 + np.abs(v).max() * 2.0 ** -s_in)


@pytest.mark.parametrize("k,h1,h2", [(7, 16, 16), (13, 32, 32)])
def test_fp64_initial_network_is_lorenzo(O, k, h1, h2):
    rng = np.random.default_rng(5)
    w = O.init_weights(k, h1, h2, seed=9)
    lzw = np.array([O.lz_weight(k, i) for i in range(k)])
    for _ in range(300):
        v = rng.integers(-(2 ** 18), 2 ** 18, k).astype(np.int32)
        assert O.mlp_pred64(w, k, h1, h2, int(rng.integers(0, 10)), v) == int((lzw * v.astype(np.int64)).sum())


def test_fp64_container_round_trip(O):
    x = gen.signed_lognormal((20, 24, 28), 3.0, 2, 2.0, 0.05)
    best, W, s_in, _ = O.train(x, 1e-2, k=7, h1=16, h2=16, seed=1)
    w = W[best if best >= 0 else 0]
    st, blob = O.compress(x, 1e-2, weights=w, s_in=s_in, fp64=True)
    assert st == 0
    assert int(np.frombuffer(blob, "<u4", 1, 12)[0]) == 3  # predictor field: FP64 form
    st, y = O.decompress(blob)
    assert st == 0
    xd = x.astype(np.float64)
    assert np.all(np.abs(y.astype(np.float64) - xd) <= 1e-2 * np.abs(xd))
    st32, b32 = O.compress(x, 1e-2, weights=w, s_in=s_in)
    # same weights, same selection rule: sizes agree to within a small fraction
    assert abs(len(blob) - len(b32)) <= 0.02 * len(b32)


def test_pred_report_counts_and_lorenzo_case(O):
    x = gen.positive_lognormal((16, 16, 24), 3.0, 4, 1.5)
    eb = 1e-2
    w = O.init_weights(7, 16, 16, seed=2)          # predicts exactly like Lorenzo
    r = O.pred_report(x, eb, w, 3, k=7, h1=16, h2=16)
    nblocks = 2 * 2 * 3
    assert r["points"] == x.size - nblocks
    assert r["rms_residual"]["fp64"] == pytest.approx(r["rms_residual"]["lorenzo"], rel=0, abs=0)
    assert r["rms_residual"]["fp32"] == r["rms_residual"]["lorenzo"]
    assert r["rms_vs_fp64"]["fp32"] == 0.0 and r["frac_differs_from_fp64"]["fp32"] == 0.0
    assert r["bits_proxy_per_point"]["fp64"] == r["bits_proxy_per_point"]["lorenzo"]


def test_pred_report_matches_dumped_codes(O):
    """With m = 16 and no residual reaching R, the report's Lorenzo bits equal the
    bit lengths of the Lorenzo residuals the compressor stores (Lorenzo-only run)."""
    x = gen.positive_lognormal((16, 16, 16), 3.0, 6, 1.0)
    eb = 1e-2
    w = O.init_weights(7, 16, 16, seed=2)
    r = O.pred_report(x, eb, w, 3, k=7, h1=16, h2=16)
    st, blob, d = O.compress(x, eb, dump=True)
    assert st == 0
    codes = d["codes"].reshape(-1, 512)[:, 1:].astype(np.int64)
    assert np.all(codes > 0)  # no balance point besides the anchors on this smooth positive field
    k = codes - 32768
    bits = np.array([int(abs(int(a))).bit_length() for a in k.reshape(-1)])
    assert r["bits_proxy_per_point"]["lorenzo"] * r["points"] == pytest.approx(bits.sum())
    assert r["rms_residual"]["lorenzo"] == pytest.approx(np.sqrt((k.astype(np.float64) ** 2).mean()))
