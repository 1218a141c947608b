"""Parity at the full sizes of the 512^3 and the float64 workloads, by sampling.

The oracle cannot compress a 134-million-point field in a test's time, so at
full size every check is either a sample the oracle computes one block at a
time, or a property that holds at any size:
  - the fixed-point network the device builds equals the oracle's
    quantization of the device-trained weights, entry for entry;
  - the header constants equal the oracle's (abs_min, abs_max, Kp, Kn, Zq, S,
    step) for the whole field;
  - sampled blocks: the device's stored codes and perceptron flags equal the
    oracle's for the same block (orc_block_codes, with the field's constants);
  - the stored histogram counts the device's codes exactly, the codebook
    equals the oracle's Huffman construction on that histogram, the block
    table carries each block's bit and balance-point counts;
  - the decoded field holds the bound on every point, and on the sampled
    blocks equals the oracle's value point by point (the stored value for a
    balance point, the reconstruction of its code otherwise).
Workloads: one 512^3 float32 density field (exp(1.5 G), G ~ k^-2), eb_rel 1e-4,
13-point 32/32 network trained on 2^20 sampled stencils; one 256 x 384 x 384
float64 field spanning 1e-8 .. 1e8 with 1% zeros, eb_rel 1e-5, 7-point 16/16
network; both in the fixed-point tensor-core form.
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
    return pcm


CASES = {
    "density512": dict(shape=(512, 512, 512), eb=1e-4, k=13, h=32, samples=1 << 20),
    "wide384_f64": dict(shape=(256, 384, 384), eb=1e-5, k=7, h=16, samples=0),
}


def make_field(name):
    dev = torch.device("cuda")
    if name == "density512":
        return torch.exp(1.5 * gen.grf_device((512, 512, 512), 2.0, 0, dev)).to(torch.float32)
    return gen.wide_range_device((256, 384, 384), 3.0, 0, dev, 8.0, 0.01)


@pytest.mark.parametrize("name", sorted(CASES))
def test_full_size_sampled_parity(pc, O, name):
    cfg = CASES[name]
    shape, eb, k, h = cfg["shape"], cfg["eb"], cfg["k"], cfg["h"]
    d = make_field(name)
    dt = pc.PC_F32 if d.dtype == torch.float32 else pc.PC_F64
    n = d.numel()
    nblocks = n // 512
    thr = int(0.1 * 2 ** 32) if not cfg["samples"] else int(round(cfg["samples"] / (n - nblocks) * 2 ** 32))
    tp = pc.make_params(eb, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h, h))
    lrs, lams = pc.default_grid()
    ws = torch.empty(pc.pc_train_workspace_size(shape, dt, tp, thr, lrs.size), dtype=torch.uint8, device="cuda")
    W, s_in, chosen, _ = pc.pc_train(d, tp, 0, thr, lrs, lams, ws)
    assert chosen >= 0
    w = W[chosen]
    p32 = pc.make_params(eb, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h, h), s_in=s_in, weights=w)
    q = pc.pc_quantize(d, p32, 0, thr, ws)
    del ws
    x = d.cpu().numpy()
    # the fixed-point network
    q_o = O.quantize(x, eb, w, s_in, k=k, h1=h, h2=h, seed=0, thr32=thr)
    assert np.array_equal(q, q_o)
    p = pc.make_params(eb, (8, 8, 8), pred=pc.PC_PRED_MLP_BF16, stencil=k, hidden=(h, h), s_in=s_in, qnet=q)
    out = torch.empty(pc.pc_compress_bound(shape, dt, p), dtype=torch.uint8, device="cuda")
    wsc = torch.empty(pc.pc_compress_workspace_size(shape, dt, p), dtype=torch.uint8, device="cuda")
    sz = pc.pc_compress(d, p, out, wsc)
    off_codes, off_nn, off_hist = pc.pc_compress_workspace_layout(shape, dt, p)
    codes = wsc[off_codes: off_codes + 2 * n].view(torch.int16).view(nblocks, 512)
    nnflag = wsc[off_nn: off_nn + nblocks]
    hist = wsc[off_hist: off_hist + 8 * 65536].view(torch.int64).cpu().numpy()
    blob = out[:sz].cpu().numpy()
    hdr = blob[:256].tobytes()
    # header constants
    c = O.consts_for(x, eb)
    Kp, Kn, Zq, S = struct.unpack_from("<4i", hdr, 100)
    assert (Kp, Kn, Zq, S) == (c.Kp, c.Kn, c.Zq, c.S)
    amin, amax = struct.unpack_from("<2d", hdr, 80)
    assert (amin, amax) == (c.abs_min, c.abs_max)
    step_bits = struct.unpack_from("<Q", hdr, 120)[0]
    want_step = np.array([c.step32], np.float32).view(np.uint32)[0] if dt == pc.PC_F32 else \
        np.array([c.stepd], np.float64).view(np.uint64)[0]
    assert step_bits == int(want_step)
    # histogram, codebook, block table (properties at full size)
    cu = codes.to(torch.int32) & 0xFFFF
    cu[:, 0] = -1  # anchors are not coded
    counts = torch.bincount(cu[:, 1:].reshape(-1), minlength=65536).cpu().numpy()
    assert np.array_equal(counts.astype(np.int64), hist)
    lens, order = O.huffman_lengths(hist.astype(np.uint64), with_order=True)
    off_cb, off_bb, off_bn = struct.unpack_from("<3Q", hdr, 176)
    n_used = struct.unpack_from("<I", hdr, 116)[0]
    cb = np.frombuffer(blob.tobytes(), "<u4", n_used, off_cb)
    assert np.array_equal(cb & 0xFFFF, order) and np.array_equal(cb >> 16, lens[order])
    lens_t = torch.from_numpy(lens.astype(np.int64)).cuda()
    bits = lens_t[cu[:, 1:].long()].sum(dim=1).cpu().numpy()
    bb = np.frombuffer(blob.tobytes(), "<u4", nblocks, off_bb)
    assert np.array_equal(bb & 0x7FFFFFFF, bits.astype(np.uint32))
    assert np.array_equal(bb >> 31, nnflag.cpu().numpy().astype(np.uint32))
    bn = np.frombuffer(blob.tobytes(), "<u2", nblocks, off_bn)
    zeros = (cu[:, 1:] == 0).sum(dim=1).cpu().numpy()
    assert np.array_equal(bn.astype(np.int64), zeros + 1)
    # sampled blocks against the oracle
    rng = np.random.default_rng(1)
    nbz, nby, nbx = (s // 8 for s in shape)
    sample = set(rng.choice(nblocks, 160, replace=False).tolist()) | {0, nblocks - 1, nbx - 1, nby * nbx - 1}
    codes_h = codes.cpu().numpy().view(np.uint16)
    nn_h = nnflag.cpu().numpy()
    for bi in sorted(sample):
        oc, usen = O.block_codes(x, c, bi, eb, stencil=k, h1=h, h2=h, s_in=s_in, qnet=q)
        assert usen == bool(nn_h[bi]), bi
        assert np.array_equal(oc[1:], codes_h[bi, 1:]), bi
    # decode: bound everywhere, the oracle's values on sampled blocks
    _, _, wsb = pc.pc_header_info(hdr)
    wsd = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(d)
    pc.pc_decompress(out, sz, y, wsd)
    torch.cuda.synchronize()
    assert bool(((y.double() - d.double()).abs() <= eb * d.double().abs()).all().item())
    assert bool((torch.signbit(y) == torch.signbit(d)).all().item())
    yh = y.cpu().numpy()
    for bi in sorted(sample)[:40]:
        bz, by, bx = bi // (nby * nbx), (bi // nbx) % nby, bi % nbx
        xb = x[8 * bz: 8 * bz + 8, 8 * by: 8 * by + 8, 8 * bx: 8 * bx + 8].reshape(-1)
        yb = yh[8 * bz: 8 * bz + 8, 8 * by: 8 * by + 8, 8 * bx: 8 * bx + 8].reshape(-1)
        dq, _ = O.transform(xb, c)
        for j in range(512):
            balance = j == 0 or codes_h[bi, j] == 0
            want = xb[j] if balance else O.recon(int(dq[j]), c, 0 if dt == pc.PC_F32 else 1)
            assert np.array_equal(np.array([yb[j]]).view(np.uint8), np.array([want], x.dtype).view(np.uint8)), (bi, j)
