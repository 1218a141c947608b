"""Pins for blocks, the data-selection rule, Lorenzo and the perceptron.

Lorenzo (Section IV.A) with out-of-block neighbours reading the anchor value is
exactly the backward mixed third difference of the anchor-centred codes
extended by zeros: a closed form that catches a dropped term, a wrong sign,
a wrong index or a flipped residual sign.
"""
import numpy as np
import pytest

from paper_2309_09778_gb300 import gen

R = 1 << 15


def block_iter(shape, block):
    nb = [(shape[i] + block[i] - 1) // block[i] for i in range(3)]
    b = 0
    for bz in range(nb[0]):
        for by in range(nb[1]):
            for bx in range(nb[2]):
                o = (bz * block[0], by * block[1], bx * block[2])
                e = tuple(min(block[i], shape[i] - o[i]) for i in range(3))
                yield b, o, e
                b += 1


def mixed_third_difference(v):
    """Delta_z Delta_y Delta_x of v with v = 0 at index -1 on every axis."""
    p = np.zeros((v.shape[0] + 1, v.shape[1] + 1, v.shape[2] + 1), np.int64)
    p[1:, 1:, 1:] = v
    d = p[1:] - p[:-1]
    d = d[:, 1:] - d[:, :-1]
    d = d[:, :, 1:] - d[:, :, :-1]
    return d


@pytest.mark.parametrize("shape,block", [((20, 21, 22), (8, 8, 8)), ((9, 30, 17), (4, 4, 4)),
                                         ((1, 50, 61), (1, 16, 32)), ((13, 11, 40), (16, 16, 16))])
def test_lorenzo_is_mixed_third_difference(O, shape, block):
    x = gen.signed_lognormal(shape, 3.0, 7, 2.0, 0.05)
    st, blob, d = O.compress(x, 1e-2, block=block, dump=True)
    assert st == 0
    dq = d["dq"].reshape(shape).astype(np.int64)
    ok = d["ok"].reshape(shape)
    bvol = block[0] * block[1] * block[2]
    checked = 0
    for b, o, e in block_iter(shape, block):
        sub = dq[o[0]:o[0] + e[0], o[1]:o[1] + e[1], o[2]:o[2] + e[2]]
        v = sub - sub[0, 0, 0]
        vc = np.clip(v, -(2 ** 24 - 1), 2 ** 24 - 1)
        k = v - (vc - mixed_third_difference(vc))   # residual = v - Lorenzo(v)
        codes = d["codes"][b * bvol:b * bvol + e[0] * e[1] * e[2]].reshape(e).astype(np.int64)
        okb = ok[o[0]:o[0] + e[0], o[1]:o[1] + e[1], o[2]:o[2] + e[2]]
        want = np.where((np.abs(k) <= R - 1) & (okb == 1), k + R, 0)
        want[0, 0, 0] = 0
        assert np.array_equal(codes, want), b
        checked += codes.size
    assert checked == x.size
    # histogram counts every non-anchor code
    nblocks = sum(1 for _ in block_iter(shape, block))
    assert d["hist"].sum() == x.size - nblocks


def test_linear_codes_give_zero_residual(O):
    """A field whose codes are affine in (i, j, k) has zero Lorenzo residual
    wherever all seven neighbours are inside the block."""
    shape = (16, 16, 16)
    eb = 1e-2
    step = 2 * np.log2(1 + eb)
    i, j, kk = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    n = 3 * i - 2 * j + 5 * kk + 100
    x = np.exp2((n * step)).astype(np.float32)
    st, blob, d = O.compress(x, eb, block=(8, 8, 8), dump=True)
    dq = d["dq"].reshape(shape)
    c = O.consts_for(x, eb)
    assert np.array_equal(dq - c.Kp, n)   # exact codes of exact powers of 2^step? (checked)
    for b, o, e in block_iter(shape, (8, 8, 8)):
        codes = d["codes"][b * 512:(b + 1) * 512].reshape(e)
        assert np.all(codes[1:, 1:, 1:] == R)


def np_mlp(w, k, h1, h2, s_in, v):
    """Independent float64 restatement of the perceptron forward."""
    w = w.astype(np.float64)
    u = np.asarray(v, np.float64) * 2.0 ** -s_in
    W1 = w[:h1 * k].reshape(h1, k); p = h1 * k
    b1 = w[p:p + h1]; p += h1
    a = W1 @ u + b1
    a = np.where(a >= 0, a, a * 0.0625)
    if h2 > 0:
        W2 = w[p:p + h2 * h1].reshape(h2, h1); p += h2 * h1
        b2 = w[p:p + h2]; p += h2
        a = W2 @ a + b2
        a = np.where(a >= 0, a, a * 0.0625)
    hl = h2 if h2 > 0 else h1
    W3 = w[p:p + hl]; b3 = w[p + hl]
    assert p + hl + 1 == w.size
    return (W3 @ a + b3) * 2.0 ** s_in


@pytest.mark.parametrize("k,h1,h2", [(7, 16, 16), (13, 32, 32), (7, 2, 0), (13, 8, 0)])
def test_mlp_forward_matches_float64(O, k, h1, h2):
    rng = np.random.default_rng(k * 100 + h1)
    nw = O.mlp_nweights(k, h1, h2)
    assert nw == h1 * k + h1 + (h2 * h1 + h2 if h2 else 0) + (h2 if h2 else h1) + 1
    for _ in range(200):
        w = (rng.standard_normal(nw) * 0.3).astype(np.float32)
        s_in = int(rng.integers(0, 12))
        v = rng.integers(-3000, 3000, k).astype(np.int32)
        got = O.mlp_fwd32(w, k, h1, h2, s_in, v)
        want = np_mlp(w, k, h1, h2, s_in, v)
        scale = 2.0 ** s_in * (1 + np.abs(v).max() * 2.0 ** -s_in) * (1 + np.abs(w).sum())
        assert abs(got - want) <= 1e-5 * scale, (got, want)


@pytest.mark.parametrize("k,h1,h2", [(7, 16, 16), (13, 32, 32), (7, 2, 0), (13, 4, 0), (7, 16, 4)])
def test_initial_perceptron_equals_lorenzo(O, k, h1, h2):
    """Section IV.B init: the untrained network reproduces the Lorenzo predictor.
    The output weight c = RN(1/(1+alpha)^L) carries a relative error below
    2^-23, so rint recovers the exact integer while |Lorenzo| < 2^21."""
    rng = np.random.default_rng(3)
    w = O.init_weights(k, h1, h2, seed=99)
    lzw = np.array([O.lz_weight(k, i) for i in range(k)])
    # the Lorenzo weights on the stencil are the SZ formula's signs
    assert np.count_nonzero(lzw) == 7 and lzw.sum() == 1
    for _ in range(400):
        s_in = int(rng.integers(0, 10))
        v = rng.integers(-(2 ** 18), 2 ** 18, k).astype(np.int32)
        assert O.mlp_pred32(w, k, h1, h2, s_in, v) == int((lzw * v.astype(np.int64)).sum())


def test_block_selection_prefers_cheaper_predictor(O):
    """a7: a block uses the perceptron only when its residual cost is strictly
    lower; the Lorenzo-equal initial network therefore never gets picked."""
    x = gen.signed_lognormal((16, 16, 16), 3.0, 1, 2.0, 0.0)
    w = O.init_weights(7, 16, 16, seed=1)
    st, blob, d = O.compress(x, 1e-2, weights=w, dump=True)
    assert st == 0 and d["nnflag"].sum() == 0
    st2, blob2, d2 = O.compress(x, 1e-2, dump=True)
    assert np.array_equal(d["codes"], d2["codes"])
