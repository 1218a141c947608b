"""Pins for the training phase (Section IV.C).

Gradients are held to torch.autograd in float64 (an independent backprop);
the sampling rule to its stated rates; the update to its formula; and the
whole phase to its purpose: the chosen network must cost fewer residual bits
than Lorenzo on a field where Lorenzo is not the best linear predictor.
"""
import numpy as np
import pytest
import torch

from paper_2309_09778_gb300 import gen


def torch_loss(w, k, h1, h2, s_in, inp, tg, use):
    wt = torch.tensor(w.astype(np.float64), requires_grad=True)
    u = torch.tensor(inp.astype(np.float64)) * 2.0 ** -s_in
    t = torch.tensor(tg.astype(np.float64)) * 2.0 ** -s_in
    p = 0
    W1 = wt[p:p + h1 * k].reshape(h1, k); p += h1 * k
    b1 = wt[p:p + h1]; p += h1
    a = torch.nn.functional.leaky_relu(u @ W1.T + b1, 0.0625)
    if h2:
        W2 = wt[p:p + h2 * h1].reshape(h2, h1); p += h2 * h1
        b2 = wt[p:p + h2]; p += h2
        a = torch.nn.functional.leaky_relu(a @ W2.T + b2, 0.0625)
    hl = h2 if h2 else h1
    W3 = wt[p:p + hl]; b3 = wt[p + hl]
    o = a @ W3 + b3
    m = torch.tensor(use.astype(np.float64))
    loss = ((o - t) ** 2 * m).sum() / len(tg)
    loss.backward()
    return wt.grad.numpy()


@pytest.mark.parametrize("k,h1,h2", [(7, 16, 16), (13, 32, 32), (7, 2, 0), (7, 8, 4)])
def test_gradient_matches_autograd(O, k, h1, h2):
    rng = np.random.default_rng(k + h1)
    nw = O.mlp_nweights(k, h1, h2)
    for B in (256, 37):
        w = (rng.standard_normal(nw) * 0.4).astype(np.float32)
        inp = rng.integers(-500, 500, (B, k)).astype(np.int32)
        tg = rng.integers(-500, 500, B).astype(np.int32)
        use = (rng.random(B) < 0.8).astype(np.uint8)
        s_in = 8
        g = O.batch_grad(w, k, h1, h2, s_in, inp, tg, use)
        gt = torch_loss(w, k, h1, h2, s_in, inp, tg, use)
        scale = np.abs(gt).max()
        assert np.allclose(g, gt, rtol=1e-4, atol=1e-5 * scale), np.abs(g - gt).max() / scale


def test_sgd_update_rule(O):
    k, h1, h2 = 7, 4, 0
    nw = O.mlp_nweights(k, h1, h2)
    rng = np.random.default_rng(1)
    w = rng.standard_normal(nw).astype(np.float32)
    g = rng.standard_normal(nw).astype(np.float32)
    lr, lam = np.float32(0.01), np.float32(0.1)
    w2 = O.sgd_update(w, g, k, h1, h2, lr, lam)
    is_bias = np.zeros(nw, bool)
    is_bias[h1 * k:h1 * k + h1] = True
    is_bias[-1] = True
    want = np.where(is_bias, w - lr * g, w - lr * (g + 2 * lam * w))
    assert np.allclose(w2, want, rtol=1e-6, atol=1e-7)


def test_sampling_rates(O):
    shape, block = (40, 40, 40), (8, 8, 8)
    thr = int(0.1 * 2 ** 32)
    nt, nv = O.count_samples(shape, block, 5, thr)
    nonanchor = 40 ** 3 - 125
    assert abs((nt + nv) / nonanchor - 0.1) < 0.01       # 10% sample (Section IV.C)
    assert abs(nv / (nt + nv) - 0.2) < 0.03               # 8:2 split
    # selection is exactly the hash rule
    cnt = 0
    for z in range(40):
        for y in range(40):
            for x in range(40):
                if z % 8 == 0 and y % 8 == 0 and x % 8 == 0:
                    continue
                h = O.mix64(5, (z * 40 + y) * 40 + x)
                cnt += (h >> 32) < thr
    assert cnt == nt + nv


def test_samples_match_compression_inputs(O):
    """Training inputs are exactly the stencils the compressor feeds the
    network, rebuilt here from the compressor's own codes, in list order."""
    x = gen.signed_lognormal((16, 16, 16), 5.0, 2, 1.0, 0.0)
    thr = int(0.3 * 2 ** 32)
    (ti, tt, tu), (vi, vt, vu) = O.gather_samples(x, 1e-2, (8, 8, 8), 13, 3, thr)
    st, blob, d = O.compress(x, 1e-2, dump=True)
    c = O.consts_for(x, 1e-2)
    dq = d["dq"].reshape(x.shape).astype(np.int64)
    cls = np.where(dq <= c.Zq, 0, np.where(dq <= c.S, 1, 2))
    offs = [(a, b, e) for a in (-1, 0, 1) for b in (-1, 0, 1) for e in (-1, 0, 1)][:13]
    want_t, want_v = [], []
    for bz in range(2):
        for by in range(2):
            for bx in range(2):
                o = (8 * bz, 8 * by, 8 * bx)
                da = dq[o]
                for lz in range(8):
                    for ly in range(8):
                        for lx in range(8):
                            if lz == ly == lx == 0:
                                continue
                            p = (o[0] + lz, o[1] + ly, o[2] + lx)
                            h = O.mix64(3, (p[0] * 16 + p[1]) * 16 + p[2])
                            if (h >> 32) >= thr:
                                continue
                            ins, use = [], cls[p] != 0 and cls[p] == cls[o]
                            for (a, b, e) in offs:
                                q = (lz + a, ly + b, lx + e)
                                if min(q) >= 0 and max(q) < 8:
                                    g = (o[0] + q[0], o[1] + q[1], o[2] + q[2])
                                    ins.append(int(np.clip(dq[g] - da, -(2 ** 24 - 1), 2 ** 24 - 1)))
                                    use = use and cls[g] == cls[p]
                                else:
                                    ins.append(0)
                            rec = (ins, int(dq[p] - da), int(use))
                            (want_v if (h & 0xFFFFFFFF) % 10 < 2 else want_t).append(rec)
    for got, want in (((ti, tt, tu), want_t), ((vi, vt, vu), want_v)):
        assert len(want) == got[1].size > 0
        assert np.array_equal(got[0], np.array([w[0] for w in want]))
        assert np.array_equal(got[1], np.array([w[1] for w in want]))
        assert np.array_equal(got[2], np.array([w[2] for w in want]))


def test_input_shift_definition(O):
    tg = np.array([3, -4, 0, 100000], np.int32)
    use = np.array([1, 1, 1, 0], np.uint8)
    s = O.input_shift(tg, use)
    # rms of used targets = sqrt(25/3) ~ 2.9 -> smallest s with (sum >> 2s) < n
    assert s == 2
    assert O.input_shift(tg, np.zeros(4, np.uint8)) == 0


def test_training_beats_lorenzo_on_rough_field(O):
    """The learned part gains: on a rough positive log-normal field (power
    spectrum k^-3, density-like) the best linear predictor averages
    neighbours rather than extrapolating, so the chosen network's validation
    cost and the compressed size must both be clearly below Lorenzo's."""
    x = gen.positive_lognormal((48, 48, 48), 3.0, 0, 1.5)
    lrs = np.array([3e-2, 1e-1], np.float32)
    lams = np.array([0.0, 1e-4], np.float32)
    best, W, s_in, costs = O.train(x, 1e-2, k=7, h1=8, h2=8, seed=1, thr32=int(0.5 * 2 ** 32),
                                   lrs=lrs, lams=lams)
    assert best >= 0
    assert costs[best] < 0.96 * costs[-1], costs
    st1, b1 = O.compress(x, 1e-2, weights=W[best], h1=8, h2=8, s_in=s_in)
    st0, b0 = O.compress(x, 1e-2)
    assert len(b1) < 0.97 * len(b0), (len(b1), len(b0))
    st, y = O.decompress(b1)
    assert st == 0 and np.all(np.abs(y.astype(np.float64) - x) <= 1e-2 * np.abs(x.astype(np.float64)))
