"""Parity at the benchmark's full size, in the benchmark's launch configuration.

The field is the benchmark's: 100 x 500 x 500 single precision, signed
log-normal, relative bound 1e-3, 8^3 blocks, 7-point stencil, 16/16
perceptron trained on the device with 10% of the points drawn.  The device
runs the same entry points the benchmark times (pc_compress / pc_decompress
with caller workspaces, on the current stream).

For both predictor forms the oracle compresses the same field with the same
network; the containers must be equal byte for byte.  The oracle's decode of
its container must equal the device decode bit for bit, and every point must
hold the bound.  The fixed-point network itself must equal the oracle's
quantization of the trained weights.  The oracle needs tens of seconds per
pass at this size.
"""
import numpy as np
import pytest
import torch

from paper_2309_09778_gb300 import gen

pytestmark = pytest.mark.gpu

SHAPE = (100, 500, 500)
EB = 1e-3
THR32 = int(0.1 * 2 ** 32)


@pytest.fixture(scope="module")
def pc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_09778_gb300.pc as pcm
    assert torch.cuda.is_available()
    return pcm


@pytest.fixture(scope="module")
def field(pc):
    x = gen.signed_lognormal(SHAPE, 11.0 / 3.0, 0, 2.0, 0.02)
    d = torch.from_numpy(x).cuda()
    tp = pc.make_params(EB, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(16, 16))
    lrs, lams = pc.default_grid()
    ws = torch.empty(pc.pc_train_workspace_size(SHAPE, pc.PC_F32, tp, THR32, lrs.size), dtype=torch.uint8,
                     device="cuda")
    W, s_in, chosen, _ = pc.pc_train(d, tp, 0, THR32, lrs, lams, ws)
    assert chosen >= 0, "the perceptron should win on this field"
    w = W[chosen]
    p32 = pc.make_params(EB, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(16, 16), s_in=s_in, weights=w)
    q = pc.pc_quantize(d, p32, 0, THR32, ws)
    del ws
    return x, d, w, s_in, q


def device_round_trip(pc, d, params):
    stream = torch.cuda.current_stream()
    out = torch.empty(pc.pc_compress_bound(SHAPE, pc.PC_F32, params), dtype=torch.uint8, device="cuda")
    wsc = torch.empty(pc.pc_compress_workspace_size(SHAPE, pc.PC_F32, params), dtype=torch.uint8, device="cuda")
    sz = pc.pc_compress(d, params, out, wsc, stream)
    blob = out[:sz].cpu().numpy().tobytes()
    _, _, wsb = pc.pc_header_info(blob[:256])
    wsd = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(d)
    pc.pc_decompress(out, sz, y, wsd, stream)
    torch.cuda.synchronize()
    return blob, y.cpu().numpy()


def check_against_oracle(O, x, blob, y, want):
    assert blob == want, "containers differ"
    st, yo = O.decompress(want)
    assert st == 0
    assert np.array_equal(y.view(np.uint32), yo.reshape(SHAPE).view(np.uint32))
    xd = x.astype(np.float64)
    assert np.all(np.abs(y.astype(np.float64) - xd) <= EB * np.abs(xd))
    assert np.array_equal(np.signbit(x), np.signbit(y))


def test_fp32_form_full_size(pc, O, field):
    x, d, w, s_in, _ = field
    p = pc.make_params(EB, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(16, 16), s_in=s_in, weights=w)
    blob, y = device_round_trip(pc, d, p)
    st, want = O.compress(x, EB, weights=w, s_in=s_in)
    assert st == 0
    check_against_oracle(O, x, blob, y, want)


def test_bf16_form_full_size(pc, O, field):
    x, d, w, s_in, q = field
    q_o = O.quantize(x, EB, w, s_in, seed=0)
    assert np.array_equal(q, q_o)
    p = pc.make_params(EB, (8, 8, 8), pred=pc.PC_PRED_MLP_BF16, stencil=7, hidden=(16, 16), s_in=s_in, qnet=q_o)
    blob, y = device_round_trip(pc, d, p)
    st, want = O.compress(x, EB, qnet=q_o, s_in=s_in)
    assert st == 0
    check_against_oracle(O, x, blob, y, want)
