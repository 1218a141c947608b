"""Pins for the paper-literal data selection (Section IV.D), the experimental
mode that predicts every point from the TRUE values of its neighbours while
the decoder can only use its own reconstructions, so errors drift until a
stored balance point ("equilibrium point") resets them.

Closed forms on 1-D blocks (a 1 x 1 x N field in 1 x 8 x 8 blocks is a row of
8-point blocks, where the Lorenzo stencil reduces to the previous value):
  - a geometric ramp rising 0.3 quantization steps per point: every true-value
    residual rounds to 0, so every code is the zero residual and the decoder
    repeats the anchor's level over the whole block (drift of 0.3 steps per
    point), whereas the bound-safe reading codes the ramp and holds the bound;
  - with every second point stored, each coded point is predicted from an
    exact neighbour, so its error stays within half a step, i.e. the bound;
  - values the bound-safe transform cannot code (zeros, subnormals) are
    stored and come back exactly; blocks stay independent.
"""
import struct

import numpy as np
import pytest

from paper_2309_09778_gb300 import gen


def ramp(n, eb, slope, x0=3.0):
    step = 2.0 * np.log2(1.0 + eb)
    return (x0 * np.exp2(slope * step * np.arange(n))).astype(np.float32).reshape(1, 1, n)


def rel_err(x, y):
    return np.abs(y.astype(np.float64) - x) / np.abs(x.astype(np.float64))


def test_ramp_codes_zero_residual_and_decodes_the_anchor_level(O):
    eb = 1e-3
    x = ramp(64, eb, 0.3)
    st, blob, d = O.compress(x, eb, block=(1, 8, 8), literal=True, dump=True)
    assert st == 0
    assert struct.unpack_from("<I", blob, 228)[0] == 4  # the literal flag
    codes = d["codes"].reshape(-1, 64)[:, :8]  # 1 x 8 x 8 blocks: the first row holds the 8 points
    R = 1 << 15
    assert np.all(codes[:, 1:] == R)          # every residual rint(0.3) = 0
    st, y = O.decompress(blob)
    assert st == 0
    yb = y.reshape(-1, 8)
    xb = x.reshape(-1, 8)
    assert np.array_equal(yb[:, 0], xb[:, 0])  # anchors stored
    for r in yb:
        assert np.all(r[1:] == r[1])           # the anchor's level repeated (no feedback from the codes)
    e = rel_err(xb[:, 1:], yb[:, 1:])
    assert e[:, 0].max() <= eb and e[:, -1].min() > eb  # 0.3 steps fine, 2.1 steps far out
    # the bound-safe reading codes the same ramp without drift
    st, safe = O.compress(x, eb, block=(1, 8, 8))
    st, ys = O.decompress(safe)
    assert rel_err(x, ys).max() <= eb


def test_every_second_point_stored_keeps_the_bound(O):
    eb = 1e-3
    x = ramp(64, eb, 0.8)
    st, blob = O.compress(x, eb, block=(1, 8, 8), literal=True, eq_period=2)
    assert st == 0
    assert struct.unpack_from("<I", blob, 232)[0] == 2
    st, y = O.decompress(blob)
    xb, yb = x.reshape(-1, 8), y.reshape(-1, 8)
    assert np.array_equal(yb[:, 0::2], xb[:, 0::2])              # stored: exact
    assert rel_err(xb[:, 1::2], yb[:, 1::2]).max() <= eb * 1.001  # half a step from an exact neighbour
    # without the equilibrium points the same ramp drifts past the bound
    st, blob0 = O.compress(x, eb, block=(1, 8, 8), literal=True)
    st, y0 = O.decompress(blob0)
    assert rel_err(x, y0).max() > 2 * eb


def test_uncodable_values_are_stored(O):
    x = np.zeros((1, 4, 24), np.float32)
    x[0, 1, ::3] = np.float32(1e-40)   # subnormal
    x[0, 2, :] = -0.0
    x[0, 3, :] = np.linspace(1, 2, 24, dtype=np.float32)
    st, blob, d = O.compress(x, 1e-2, block=(1, 8, 8), literal=True, dump=True)
    assert st == 0
    st, y = O.decompress(blob)
    keep = (x == 0) | (np.abs(x) < np.float32(2.0 ** -126))
    assert np.array_equal(y[keep].view(np.uint32), x[keep].view(np.uint32))


def test_blocks_drift_independently(O):
    x = gen.positive_lognormal((16, 16, 24), 3.0, 2, 1.0)
    st, a = O.compress(x, 1e-3, literal=True)
    x2 = x.copy()
    x2[3, 4, 5] *= np.float32(1.5)      # block (0, 0, 0)
    st, b = O.compress(x2, 1e-3, literal=True)
    st, ya = O.decompress(a)
    st, yb = O.decompress(b)
    same = ya.view(np.uint32) == yb.view(np.uint32)
    inside = np.zeros(x.shape, bool)
    inside[:8, :8, :8] = True
    assert same[~inside].all() and not same[inside].all()


def test_perceptron_literal_round_trip_of_stored_points(O):
    x = gen.positive_lognormal((16, 16, 16), 3.0, 3, 1.0)
    w = O.init_weights(7, 8, 8, seed=1)
    # every point stored: the container carries the flag and the weights, and decodes exactly
    st, blob = O.compress(x, 1e-3, weights=w, stencil=7, h1=8, h2=8, s_in=4, literal=True, eq_period=1)
    assert st == 0
    st, y = O.decompress(blob)
    assert np.array_equal(y.view(np.uint32), x.view(np.uint32))
    # float64 fields and the fixed-point form are refused
    assert O.compress(x.astype(np.float64), 1e-3, literal=True)[0] == -1
