"""GPU parity of the paper-literal data selection (Section IV.D, experimental)
through the C ABI: containers equal the oracle's byte for byte and the
drifting decoder's output equals the oracle's bit for bit, for Lorenzo and the
FP32 perceptron, with and without deliberate equilibrium points, across block
shape families and ragged edges.  The bound is not asserted (the mode drifts by
design); the drift statistics are the bench's business.
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
    assert torch.cuda.is_available()
    return pcm


CASES = [
    # shape, block, eb, predictor (k, h), eq_period
    ((20, 27, 35), (8, 8, 8), 1e-3, None, 0),
    ((20, 27, 35), (8, 8, 8), 1e-3, None, 16),
    ((19, 23, 29), (8, 8, 8), 1e-3, (7, (16, 16)), 0),
    ((19, 23, 29), (8, 8, 8), 1e-2, (13, (32, 32)), 32),
    ((9, 30, 17), (4, 4, 4), 1e-3, (7, (8, 8)), 5),
    ((13, 11, 40), (16, 16, 16), 1e-2, None, 64),
    ((1, 50, 61), (1, 16, 32), 1e-3, (7, (16, 16)), 0),
    ((1, 1, 300), (1, 8, 8), 1e-3, None, 0),
]


@pytest.mark.parametrize("shape,block,eb,net,eq", CASES)
def test_literal_matches_oracle(pc, O, shape, block, eb, net, eq):
    x = gen.signed_lognormal(shape, 3.0, 13, 2.0, 0.03)
    w, s_in, k, h = None, 0, 7, (16, 16)
    if net is not None:
        k, h = net
        best, W, s_in, _ = O.train(x, eb, block=block, k=k, h1=h[0], h2=h[1], seed=2)
        w = W[max(best, 0)]
    st, want = O.compress(x, eb, block=block, weights=w, stencil=k, h1=h[0], h2=h[1], s_in=s_in, literal=True,
                          eq_period=eq)
    assert st == 0
    p = pc.make_params(eb, block, pred=pc.PC_PRED_MLP_FP32 if w is not None else pc.PC_PRED_LORENZO, stencil=k,
                       hidden=h, s_in=s_in, weights=w, literal=True, eq_period=eq)
    blob = pc.compress(torch.from_numpy(x).cuda(), p)
    got = blob.cpu().numpy().tobytes()
    assert len(got) == len(want)
    diff = np.flatnonzero(np.frombuffer(got, np.uint8) != np.frombuffer(want, np.uint8))
    assert diff.size == 0, f"{diff.size} bytes differ, first at {diff[0]}"
    y = pc.decompress(blob).cpu().numpy()
    st, yo = O.decompress(want)
    assert st == 0
    assert np.array_equal(y.view(np.uint32), yo.view(np.uint32))


def test_literal_refusals(pc):
    x = torch.from_numpy(gen.positive_lognormal((8, 8, 8), 3.0, 1, 1.0)).cuda()
    for kw in (dict(pred=pc.PC_PRED_MLP_BF16), dict(pred=pc.PC_PRED_MLP_FP32)):  # fixed point; no weights
        with pytest.raises(pc.PcError):
            pc.compress(x, pc.make_params(1e-3, (8, 8, 8), literal=True, **kw))
    with pytest.raises(pc.PcError):
        pc.compress(x.double(), pc.make_params(1e-3, (8, 8, 8), literal=True))
    with pytest.raises(pc.PcError):
        pc.compress(x, pc.make_params(1e-3, (8, 8, 8), eq_period=4))  # a period without the literal mode
