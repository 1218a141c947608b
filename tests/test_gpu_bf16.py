"""GPU parity of the fixed-point (BF16) perceptron form through the C ABI.

The device quantization (pc_quantize) must equal the oracle's network entry
for entry; containers compressed with the tensor-core form must equal the
oracle's byte for byte, and decompression (tensor-core waves) must reproduce
the oracle's output bit for bit with the bound held on every point.
"""
import struct

import numpy as np
import pytest
import torch

from paper_2309_09778_gb300 import gen

pytestmark = pytest.mark.gpu

THR32 = int(0.1 * 2 ** 32)


@pytest.fixture(scope="module")
def pc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_09778_gb300.pc as pcm
    assert torch.cuda.is_available()
    return pcm


def device_quantize(pc, x, eb, block, k, h, w, s_in, seed):
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    p = pc.make_params(eb, block, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=h, s_in=s_in, weights=w)
    ws = torch.empty(pc.pc_train_workspace_size(x.shape, 0 if x.dtype == np.float32 else 1, p, THR32, 1),
                     dtype=torch.uint8, device="cuda")
    return pc.pc_quantize(t, p, seed, THR32, ws)


def same_bits(a, b):
    u = np.uint32 if a.dtype == np.float32 else np.uint64
    return np.array_equal(a.view(u), b.view(u))


CASES = [
    ((20, 21, 22), (8, 8, 8), 1e-2, 7, (16, 16), np.float32),
    ((24, 40, 40), (8, 8, 8), 1e-3, 7, (16, 16), np.float32),
    ((9, 30, 17), (4, 4, 4), 1e-3, 7, (16, 16), np.float32),
    ((13, 11, 40), (16, 16, 16), 1e-2, 7, (16, 16), np.float32),
    ((1, 50, 61), (1, 16, 32), 1e-3, 7, (16, 16), np.float32),
    ((19, 23, 29), (8, 8, 8), 1e-3, 13, (32, 32), np.float32),
    ((17, 18, 19), (8, 8, 8), 1e-4, 7, (16, 16), np.float64),
]


@pytest.mark.parametrize("shape,block,eb,k,h,dt", CASES)
def test_bf16_quantize_container_decode_match_oracle(pc, O, shape, block, eb, k, h, dt):
    x = gen.signed_lognormal(shape, 3.5, 11, 2.5, 0.05, dtype=dt) if k == 7 else \
        gen.positive_lognormal(shape, 3.0, 5, 1.5).astype(dt)
    best, W, s_in, _ = O.train(x, eb, block=block, k=k, h1=h[0], h2=h[1], seed=3)
    w = W[max(best, 0)]
    q_o = O.quantize(x, eb, w, s_in, block=block, k=k, h1=h[0], h2=h[1], seed=3)
    q_g = device_quantize(pc, x, eb, block, k, h, w, s_in, 3)
    assert np.array_equal(q_g, q_o)
    p = pc.make_params(eb, block, pred=pc.PC_PRED_MLP_BF16, stencil=k, hidden=h, s_in=s_in, qnet=q_o)
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    got = pc.compress(t, p).cpu().numpy().tobytes()
    st, want, d = O.compress(x, eb, block=block, qnet=q_o, stencil=k, h1=h[0], h2=h[1], s_in=s_in, dump=True)
    assert st == 0
    assert got == want, "containers differ"
    y = pc.decompress(torch.from_numpy(np.frombuffer(got, np.uint8).copy()).cuda()).cpu().numpy()
    st, yo = O.decompress(want)
    assert st == 0 and same_bits(y, yo.reshape(x.shape))
    xd = x.astype(np.float64)
    if dt == np.float32:
        assert np.all(np.abs(y.astype(np.float64) - xd) <= eb * np.abs(xd))
    assert np.array_equal(np.signbit(x), np.signbit(y))
    if shape[0] > 1 and d["nnflag"].size >= 8:   # the tensor-core predictor is exercised
        assert d["nnflag"].sum() > 0


def test_bf16_ratio_close_to_fp32(pc, O):
    """The fixed-point form costs little compression ratio against the FP32 form."""
    x = gen.signed_lognormal((48, 64, 64), 11 / 3, 0, 2.0, 0.02)
    t = torch.from_numpy(x).cuda()
    best, W, s_in, _ = O.train(x, 1e-3, seed=0)
    assert best >= 0
    w = W[best]
    q = device_quantize(pc, x, 1e-3, (8, 8, 8), 7, (16, 16), w, s_in, 0)
    n32 = pc.compress(t, pc.make_params(1e-3, pred=pc.PC_PRED_MLP_FP32, s_in=s_in, weights=w)).numel()
    nbf = pc.compress(t, pc.make_params(1e-3, pred=pc.PC_PRED_MLP_BF16, s_in=s_in, qnet=q)).numel()
    assert nbf <= 1.02 * n32, (nbf, n32)


def test_bf16_corrupt_network_rejected(pc, O):
    x = gen.positive_lognormal((16, 16, 16), 3.0, 2, 1.0)
    best, W, s_in, _ = O.train(x, 1e-2, seed=2)
    q = O.quantize(x, 1e-2, W[max(best, 0)], s_in, seed=2)
    t = torch.from_numpy(x).cuda()
    blob = pc.compress(t, pc.make_params(1e-2, pred=pc.PC_PRED_MLP_BF16, s_in=s_in, qnet=q)).cpu().numpy()
    off_w = struct.unpack_from("<Q", blob.tobytes(), 168)[0]
    for pos, val in ((9, 300), (7, 99), (4, 31)):
        bad = blob.copy()
        struct.pack_into("<q", bad, off_w + 8 * pos, val)
        with pytest.raises(pc.PcError) as ei:
            pc.decompress(torch.from_numpy(bad).cuda())
        assert ei.value.status == -5
    # invalid networks are refused before compression
    bad_q = q.copy()
    bad_q[9] = 256
    with pytest.raises(pc.PcError):
        pc.compress(t, pc.make_params(1e-2, pred=pc.PC_PRED_MLP_BF16, s_in=s_in, qnet=bad_q))
