"""GPU parity of the lossless back-end stage (Section IV.A's fourth SZ stage)
through the C ABI: containers with the stage equal the oracle's byte for byte
(coded and stored chunks, several chunks with a short last one), decode bit
for bit like the plain container, and a damaged section is refused without a
fault.
"""
import struct

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
    # shape, eb, muted share, dtype, predictor
    ((40, 48, 64), 1e-2, 0.6, np.float32, False),
    ((64, 96, 96), 1e-4, 0.3, np.float32, False),
    ((24, 40, 40), 1e-3, 0.05, np.float64, False),
    ((19, 23, 29), 1e-3, 0.5, np.float32, True),
    ((1, 1, 9), 1e-2, 0.0, np.float32, False),
]


@pytest.mark.parametrize("shape,eb,zf,dt,nn", CASES)
def test_lossless_matches_oracle(pc, O, shape, eb, zf, dt, nn):
    x = gen.signed_lognormal(shape, 11 / 3, 4, 2.0, zf, dtype=dt)
    w, s_in = None, 0
    if nn:
        best, W, s_in, _ = O.train(x, eb, k=7, h1=16, h2=16, seed=1)
        w = W[max(best, 0)]
    st, want = O.compress(x, eb, weights=w, s_in=s_in, lossless=True)
    assert st == 0
    p = pc.make_params(eb, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32 if nn else pc.PC_PRED_LORENZO, s_in=s_in, weights=w,
                       lossless=True)
    t = torch.from_numpy(x).cuda()
    blob = pc.compress(t, p)
    got = blob.cpu().numpy().tobytes()
    assert len(got) == len(want)
    diff = np.flatnonzero(np.frombuffer(got, np.uint8) != np.frombuffer(want, np.uint8))
    assert diff.size == 0, f"{diff.size} bytes differ, first at {diff[0]}"
    y = pc.decompress(blob).cpu().numpy()
    y0 = pc.decompress(pc.compress(t, pc.make_params(eb, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32 if nn else
                                                     pc.PC_PRED_LORENZO, s_in=s_in, weights=w))).cpu().numpy()
    u = np.uint32 if dt == np.float32 else np.uint64
    assert np.array_equal(y.view(u), y0.view(u))


def test_damaged_section_is_refused(pc, O):
    x = gen.signed_lognormal((40, 48, 64), 11 / 3, 4, 2.0, 0.6)
    blob = pc.compress(torch.from_numpy(x).cuda(), pc.make_params(1e-2, (8, 8, 8), lossless=True))
    h = blob.cpu().numpy()
    off_st = struct.unpack_from("<Q", h.tobytes(), 208)[0]
    sizes = np.frombuffer(h.tobytes(), "<u4", struct.unpack_from("<I", h.tobytes(), off_st)[0], off_st + 16)
    coded = np.flatnonzero((sizes >> 31) == 0)
    assert coded.size > 0
    bad = h.copy()
    # the first coded chunk's first control byte becomes a far match
    nch = sizes.size
    first = off_st + ((16 + 4 * nch + 15) // 16) * 16 + int(sum(int(v) & 0x7FFFFFFF for v in sizes[: coded[0]]))
    bad[first] = 0xFF
    bad[first + 1] = 0xFF
    bad[first + 2] = 0x3F
    with pytest.raises(pc.PcError):
        pc.decompress(torch.from_numpy(bad).cuda())
