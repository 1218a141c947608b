"""Device training (Section IV.C) against the oracle.

The GPU samples, gathers, scales, initialises and trains with the same
operations in the same order as the oracle (gradients as pairwise tree sums
over the 256 rows), so every trained weight, the input scale, the validation
costs and the chosen model must match bit for bit.  The chosen model must
also compress better than Lorenzo on a field where averaging beats
extrapolation.
"""
import numpy as np
import pytest
import torch

from paper_2309_09778_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_09778_gb300.pc as pcm
    return pcm


def gpu_train(pc, x, eb, block, k, h, seed, thr32, lrs, lams):
    p = pc.make_params(eb, block, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=h)
    ws = torch.empty(pc.pc_train_workspace_size(x.shape, pc.PC_F32 if x.dtype == np.float32 else pc.PC_F64, p,
                                                thr32, len(lrs)), dtype=torch.uint8, device="cuda")
    return pc.pc_train(torch.from_numpy(x).cuda(), p, seed, thr32, lrs, lams, ws)


@pytest.mark.parametrize("shape,block,k,h", [
    ((24, 32, 40), (8, 8, 8), 7, (8, 8)),
    ((20, 28, 33), (8, 8, 8), 7, (16, 16)),
    ((17, 24, 30), (4, 4, 4), 13, (16, 16)),
    ((12, 20, 26), (8, 8, 8), 13, (32, 32)),
    ((30, 30, 30), (8, 8, 8), 7, (2, 0)),
])
def test_training_matches_oracle(pc, O, shape, block, k, h):
    x = gen.positive_lognormal(shape, 3.0, 3, 1.5)
    lrs = np.array([3e-2, 1e-1, 1e-2], np.float32)
    lams = np.array([0.0, 1e-4, 1e-3], np.float32)
    thr = int(0.5 * 2 ** 32)
    W, s_in, chosen, costs = gpu_train(pc, x, 1e-2, block, k, h, 5, thr, lrs, lams)
    best, Wo, s_o, costs_o = O.train(x, 1e-2, block=block, k=k, h1=h[0], h2=h[1], seed=5, thr32=thr,
                                     lrs=lrs, lams=lams)
    assert s_in == s_o
    assert np.array_equal(costs, costs_o), (costs, costs_o)
    assert chosen == best
    assert np.array_equal(W.view(np.uint32), Wo.view(np.uint32))


def test_trained_model_beats_lorenzo(pc, O):
    x = gen.positive_lognormal((48, 48, 48), 3.0, 0, 1.5)
    lrs = np.array([3e-2, 1e-1], np.float32)
    lams = np.array([0.0, 1e-4], np.float32)
    W, s_in, chosen, costs = gpu_train(pc, x, 1e-2, (8, 8, 8), 7, (8, 8), 1, int(0.5 * 2 ** 32), lrs, lams)
    assert chosen >= 0 and costs[chosen] < 0.96 * costs[-1]
    d = torch.from_numpy(x).cuda()
    nn = pc.compress(d, pc.make_params(1e-2, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(8, 8),
                                       s_in=s_in, weights=W[chosen]))
    lz = pc.compress(d, pc.make_params(1e-2, (8, 8, 8)))
    assert nn.numel() < 0.97 * lz.numel()
    y = pc.decompress(nn).cpu().numpy()
    assert np.all(np.abs(y.astype(np.float64) - x) <= 1e-2 * np.abs(x.astype(np.float64)))


@pytest.mark.parametrize("pred,k,h,samples", [("fp32", 7, (16, 16), 0), ("bf16", 7, (16, 16), 0),
                                              ("bf16", 13, (32, 32), 20000)])
def test_compress_trains_when_no_weights_are_given(pc, O, pred, k, h, samples):
    """pc_compress with a perceptron form and no weights runs the training phase
    (and, for the fixed-point form, the quantization) on the device itself; the
    container equals the oracle's, trained with the same seed, rate and grid."""
    x = gen.positive_lognormal((24, 40, 48), 3.0, 7, 1.5)
    eb, seed = 1e-2, 11
    form = pc.PC_PRED_MLP_FP32 if pred == "fp32" else pc.PC_PRED_MLP_BF16
    p = pc.make_params(eb, (8, 8, 8), pred=form, stencil=k, hidden=h, seed=seed, train_samples=samples, ndims=3)
    blob = pc.compress(torch.from_numpy(x).cuda(), p).cpu().numpy().tobytes()
    n = x.size - (x.shape[0] // 8) * (x.shape[1] // 8) * (x.shape[2] // 8)
    thr = int(0.1 * 2 ** 32) if samples == 0 else int(samples / n * 2 ** 32)
    best, W, s_in, _ = O.train(x, eb, k=k, h1=h[0], h2=h[1], seed=seed, thr32=thr)
    if best < 0:
        st, want = O.compress(x, eb)
    elif pred == "fp32":
        st, want = O.compress(x, eb, weights=W[best], stencil=k, h1=h[0], h2=h[1], s_in=s_in)
    else:
        q = O.quantize(x, eb, W[best], s_in, k=k, h1=h[0], h2=h[1], seed=seed, thr32=thr)
        st, want = O.compress(x, eb, qnet=q, stencil=k, h1=h[0], h2=h[1], s_in=s_in)
    assert st == 0 and blob == want


def test_params_ndims_checked(pc):
    p = pc.make_params(1e-2, (1, 16, 32), ndims=2)
    assert pc.pc_compress_bound((1, 40, 50), pc.PC_F32, p) > 0
    assert pc.pc_compress_bound((3, 40, 50), pc.PC_F32, p) == 0


@pytest.mark.parametrize("shape,k,h,eb,dt", [((24, 32, 40), 7, (8, 8), 1e-2, np.float32),
                                             ((20, 24, 40), 13, (16, 16), 1e-3, np.float32),
                                             ((16, 24, 24), 7, (16, 16), 1e-4, np.float64)])
def test_selection_by_simulated_compression_matches_oracle(pc, O, shape, k, h, eb, dt):
    """Section IV.C selection: simulated sizes of every model and Lorenzo, the
    choice and the coverage-chosen m equal the oracle's."""
    x = gen.positive_lognormal(shape, 3.0, 3, 1.5).astype(dt)
    lrs = np.array([3e-2, 1e-1, 1e-2, 0.0], np.float32)
    lams = np.array([0.0, 1e-4, 1e-3, 0.0], np.float32)
    thr = int(0.5 * 2 ** 32)
    p = pc.make_params(eb, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=h)
    ws = torch.empty(pc.pc_train_workspace_size(shape, pc.PC_F32 if dt == np.float32 else pc.PC_F64, p, thr, 4),
                     dtype=torch.uint8, device="cuda")
    W, s_in, chosen, sizes, m = pc.pc_train_select(torch.from_numpy(x).cuda(), p, 5, thr, lrs, lams, ws)
    best, Wo, s_o, sizes_o, m_o = O.train_select(x, eb, k=k, h1=h[0], h2=h[1], seed=5, thr32=thr, lrs=lrs, lams=lams)
    assert s_in == s_o
    assert np.array_equal(W.view(np.uint32), Wo.view(np.uint32))
    assert np.array_equal(sizes, sizes_o), (sizes, sizes_o)
    assert chosen == best and m == m_o
    assert sizes[3] == sizes[4]  # the learning-rate-0 model is Lorenzo
