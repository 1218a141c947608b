"""GPU parity of single-pass compression with a sample codebook (Section IV.C:
the training phase's Huffman code kept for compression) through the C ABI.

The device's sample codebook must equal the oracle's list entry for entry;
containers compressed in one pass (codes outside the list become balance
points, a look-back across bricks places each brick's bits, the stream
precedes the balance values) must equal the oracle's byte for byte, and
decode bit for bit with the bound held on every point.  Cases span ragged
edges, every block shape family, the three predictor forms, both dtypes,
fields of one point and of no coded bits, a field of thousands of bricks,
and the batched entry point.
"""
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


def same_bits(a, b):
    u = np.uint32 if a.dtype == np.float32 else np.uint64
    return np.array_equal(a.view(u), b.view(u))


def bound_held(x, y, eb):
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    ok = np.abs(yd - xd) <= eb * np.abs(xd)
    if x.dtype == np.float64:
        from fractions import Fraction
        for i in np.flatnonzero(~ok.ravel())[:200]:
            ok.ravel()[i] = abs(Fraction(x.ravel()[i]) - Fraction(y.ravel()[i])) <= Fraction(eb) * abs(
                Fraction(x.ravel()[i]))
    return bool(ok.all()) and np.array_equal(np.signbit(x), np.signbit(y))


def drop_one(O, cb, rank=3):
    """The list rebuilt without its rank-th entry (not symbol 0): exercises the remap."""
    syms = cb & 0xFFFF
    keep = [int(s) for s in syms]
    s = [v for v in keep if v != 0][min(rank, len(keep) - 2)]
    h = np.zeros(1 << 16, np.uint64)
    # lengths as weights: any histogram gives a valid list; this one keeps the shape of cb
    h[syms] = (1 << (25 - (cb >> 16))).astype(np.uint64)
    h[s] = 0
    return O.sample_codebook(h, m=16)


CASES = [
    # shape, block, eb, form, k, hidden, dtype
    ((20, 27, 35), (8, 8, 8), 1e-3, "lorenzo", 7, (16, 16), np.float32),
    ((37, 45, 70), (8, 8, 8), 1e-3, "fp32", 7, (16, 16), np.float32),
    ((24, 40, 40), (8, 8, 8), 1e-3, "bf16", 7, (16, 16), np.float32),
    ((19, 23, 29), (8, 8, 8), 1e-3, "bf16", 13, (32, 32), np.float32),
    ((9, 30, 17), (4, 4, 4), 1e-3, "fp32", 7, (16, 16), np.float32),
    ((13, 11, 40), (16, 16, 16), 1e-2, "lorenzo", 7, (16, 16), np.float32),
    ((1, 50, 61), (1, 16, 32), 1e-3, "bf16", 7, (16, 16), np.float32),
    ((1, 70, 130), (1, 64, 64), 1e-3, "fp32", 7, (16, 16), np.float32),
    ((1, 33, 19), (1, 8, 8), 1e-2, "lorenzo", 7, (16, 16), np.float32),
    ((17, 18, 19), (8, 8, 8), 1e-5, "fp32", 7, (16, 16), np.float64),
    ((21, 16, 24), (8, 8, 8), 1e-4, "bf16", 7, (16, 16), np.float64),
]


def field_for(shape, dt, seed):
    return gen.signed_lognormal(shape, 3.0, seed, 2.0, 0.05, dtype=dt)


def trained(O, x, eb, block, k, h):
    best, W, s_in, _ = O.train(x, eb, block=block, k=k, h1=h[0], h2=h[1], seed=3)
    return W[max(best, 0)], s_in


@pytest.mark.parametrize("shape,block,eb,form,k,h,dt", CASES)
def test_single_pass_matches_oracle(pc, O, shape, block, eb, form, k, h, dt):
    x = field_for(shape, dt, 7)
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    dtc = pc.PC_F32 if dt == np.float32 else pc.PC_F64
    w, s_in, q = None, 0, None
    if form != "lorenzo":
        w, s_in = trained(O, x, eb, block, k, h)
    # the device's sample codebook for the FP32 weights (or Lorenzo) equals the oracle's
    pp = pc.make_params(eb, block, pred=pc.PC_PRED_LORENZO if w is None else pc.PC_PRED_MLP_FP32, stencil=k,
                        hidden=h, s_in=s_in, weights=w)
    ws = torch.empty(pc.pc_train_workspace_size(shape, dtc, pp, THR32, 1), dtype=torch.uint8, device="cuda")
    for fill in (False, True):
        cb = pc.pc_sample_codebook(t, pp, 3, THR32, ws, span_fill=fill)
        cb_o = O.sample_codebook_for(x, eb, block=block, k=k, h1=h[0], h2=h[1], s_in=s_in, weights=w, seed=3,
                                     thr32=THR32, span_fill=fill)
        assert np.array_equal(cb, cb_o), fill
    if CASES.index((shape, block, eb, form, k, h, dt)) % 2:
        cb = drop_one(O, cb)  # a hole inside the span: those codes become balance points
    if form == "bf16":
        q = O.quantize(x, eb, w, s_in, block=block, k=k, h1=h[0], h2=h[1], seed=3)
        p = pc.make_params(eb, block, pred=pc.PC_PRED_MLP_BF16, stencil=k, hidden=h, s_in=s_in, qnet=q, codebook=cb)
        st, want = O.compress(x, eb, block=block, stencil=k, h1=h[0], h2=h[1], s_in=s_in, qnet=q, codebook=cb)
    else:
        p = pc.make_params(eb, block, pred=pc.PC_PRED_LORENZO if w is None else pc.PC_PRED_MLP_FP32, stencil=k,
                           hidden=h, s_in=s_in, weights=w, codebook=cb)
        st, want = O.compress(x, eb, block=block, weights=w, stencil=k, h1=h[0], h2=h[1], s_in=s_in, codebook=cb)
    assert st == 0
    blob = pc.compress(t, p)
    got = blob.cpu().numpy().tobytes()
    assert len(got) == len(want)
    a, b = np.frombuffer(got, np.uint8), np.frombuffer(want, np.uint8)
    diff = np.flatnonzero(a != b)
    assert diff.size == 0, f"{diff.size} bytes differ, first at {diff[0]}"
    y = pc.decompress(blob).cpu().numpy()
    st, yo = O.decompress(want)
    assert st == 0 and same_bits(y, yo)
    assert bound_held(x, y, eb)


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 1, 1), (5, 3, 2)])
def test_single_pass_tiny_fields(pc, O, shape):
    # one point (only an anchor, no coded bits); a few points in one brick
    x = field_for(shape, np.float32, 2)
    cb = np.array([0 | 1 << 16], np.uint32) if shape == (1, 1, 1) else \
        O.sample_codebook(np.bincount([0, 5, 5, 9], minlength=1 << 16).astype(np.uint64), m=16)
    p = pc.make_params(1e-2, (8, 8, 8), codebook=cb)
    st, want = O.compress(x, 1e-2, codebook=cb)
    assert st == 0
    blob = pc.compress(torch.from_numpy(x).cuda(), p)
    assert blob.cpu().numpy().tobytes() == want
    y = pc.decompress(blob).cpu().numpy()
    st, yo = O.decompress(want)
    assert same_bits(y, yo)


def test_single_pass_many_bricks(pc, O):
    # 4 M points, 8192 bricks: the look-back runs across many CTAs' worth of bricks
    shape = (64, 128, 512)
    x = gen.positive_lognormal(shape, 3.0, 9, 1.5)
    eb = 1e-3
    cb = O.sample_codebook_for(x, eb, seed=1, thr32=THR32)
    st, want = O.compress(x, eb, codebook=cb)
    assert st == 0
    p = pc.make_params(eb, (8, 8, 8), codebook=cb)
    t = torch.from_numpy(x).cuda()
    for _ in range(2):  # the same bytes on a second run (look-back order differs run to run)
        blob = pc.compress(t, p)
        assert blob.cpu().numpy().tobytes() == want
    y = pc.decompress(blob).cpu().numpy()
    assert bound_held(x, y, eb)


def test_single_pass_batch(pc, O):
    rng = np.random.default_rng(4)
    fields, params, wants = [], [], []
    for f in range(6):
        shape = tuple(int(v) for v in rng.integers(8, 40, 3))
        x = field_for(shape, np.float32, 20 + f)
        cb = O.sample_codebook_for(x, 1e-3, seed=f, thr32=THR32)
        if f % 2:
            cb = drop_one(O, cb, 1)
        fields.append(torch.from_numpy(x).cuda())
        params.append(pc.make_params(1e-3, (8, 8, 8), codebook=cb))
        st, want = O.compress(x, 1e-3, codebook=cb)
        assert st == 0
        wants.append(want)
    wsb, ob = pc.pc_compress_batch_workspace_size(fields, params)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    out = torch.empty(ob, dtype=torch.uint8, device="cuda")
    offs, sizes = pc.pc_compress_batch(fields, params, out, ws)
    blob = out.cpu().numpy()
    for i in range(len(fields)):
        assert blob[offs[i]: offs[i] + sizes[i]].tobytes() == wants[i]


def test_single_pass_refuses_bad_lists(pc):
    x = torch.from_numpy(field_for((8, 8, 8), np.float32, 1)).cuda()
    for cb in ([5 | 1 << 16, 0 | 1 << 16, 7 | 1 << 16],       # Kraft sum above one
               [5 | 2 << 16, 0 | 1 << 16],                    # lengths decreasing
               [5 | 1 << 16, 7 | 1 << 16]):                   # no symbol 0
        p = pc.make_params(1e-2, (8, 8, 8), codebook=np.array(cb, np.uint32))
        with pytest.raises(pc.PcError):
            pc.compress(x, p)
