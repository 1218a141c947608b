"""GPU vs oracle parity through the C ABI.

The container produced on the GPU must equal the oracle's byte for byte
(codes, balance points, histogram-derived codebook, block table and
bitstream), and decompression must reproduce the oracle's output bit for
bit, with the pointwise relative bound held on every point.
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


SECTIONS = ["header", "weights", "codebook", "block bits", "block outliers", "outliers", "stream"]


def where(blob, off):
    offs = [0, 256, *struct.unpack_from("<5Q", blob, 176)]
    name = "header"
    for nm, o in zip(SECTIONS, offs):
        if off >= o:
            name = nm
    return name


def assert_same(got: bytes, want: bytes):
    if got == want:
        return
    n = min(len(got), len(want))
    a = np.frombuffer(got[:n], np.uint8)
    b = np.frombuffer(want[:n], np.uint8)
    diff = np.flatnonzero(a != b)
    first = int(diff[0]) if diff.size else n
    raise AssertionError(f"containers differ: len {len(got)} vs {len(want)}, first diff at {first} "
                         f"({where(want, first)}), {diff.size} differing bytes")


def run_gpu(pc, x, eb, block=(8, 8, 8), weights=None, stencil=7, hidden=(16, 16), s_in=4, m=16):
    p = pc.make_params(eb, block, pred=pc.PC_PRED_MLP_FP32 if weights is not None else pc.PC_PRED_LORENZO,
                       stencil=stencil, hidden=hidden, m=m, s_in=s_in, weights=weights)
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    blob = pc.compress(t, p)
    y = pc.decompress(blob).cpu().numpy()
    return blob.cpu().numpy().tobytes(), y


def check_roundtrip(x, y, eb):
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    if x.dtype == np.float32:
        assert np.all(np.abs(yd - xd) <= eb * np.abs(xd))
    else:
        from fractions import Fraction
        bad = np.flatnonzero((np.abs(yd - xd) > eb * np.abs(xd)).ravel())
        for i in bad[:100]:
            assert abs(Fraction(x.ravel()[i]) - Fraction(y.ravel()[i])) <= Fraction(eb) * abs(Fraction(x.ravel()[i]))
    assert np.array_equal(np.signbit(x), np.signbit(y))


def same_bits(a, b):
    u = np.uint32 if a.dtype == np.float32 else np.uint64
    return np.array_equal(a.view(u), b.view(u))


CASES = [
    ((20, 21, 22), (8, 8, 8), 1e-2, np.float32),
    ((64, 64, 64), (8, 8, 8), 1e-2, np.float32),
    ((9, 30, 17), (4, 4, 4), 1e-3, np.float32),
    ((13, 11, 40), (16, 16, 16), 1e-2, np.float32),
    ((1, 50, 61), (1, 16, 32), 1e-3, np.float32),
    ((1, 70, 130), (1, 64, 64), 1e-2, np.float32),
    ((3, 40, 33), (1, 8, 8), 1e-4, np.float32),
    # rows a multiple of 16 bytes: whole bricks take the vector-load path
    ((2, 40, 128), (1, 8, 8), 1e-3, np.float32),
    ((8, 16, 64), (4, 4, 4), 1e-3, np.float32),
    ((17, 18, 19), (8, 8, 8), 1e-5, np.float64),
    ((33, 9, 70), (4, 4, 4), 1e-3, np.float64),
]


@pytest.mark.parametrize("shape,block,eb,dt", CASES)
def test_lorenzo_container_and_decode_match_oracle(pc, O, shape, block, eb, dt):
    x = gen.signed_lognormal(shape, 3.5, 11, 2.5, 0.05, dtype=dt)
    got, y = run_gpu(pc, x, eb, block)
    st, want = O.compress(x, eb, block=block)
    assert st == 0
    assert_same(got, want)
    st, yo = O.decompress(want)
    assert st == 0
    assert same_bits(y, yo.reshape(x.shape))
    check_roundtrip(x, y, eb)


@pytest.mark.parametrize("shape,block,eb,k,h", [
    ((20, 21, 22), (8, 8, 8), 1e-2, 7, (16, 16)),
    ((19, 23, 29), (8, 8, 8), 1e-3, 13, (32, 32)),
    ((9, 30, 17), (4, 4, 4), 1e-2, 7, (2, 0)),
    ((13, 11, 40), (16, 16, 16), 1e-2, 13, (8, 4)),
    ((1, 50, 61), (1, 16, 32), 1e-3, 13, (32, 32)),
    # several 16-block reconstruction bricks along x, truncated last brick
    ((9, 30, 70), (4, 4, 4), 1e-2, 7, (16, 16)),
    ((1, 40, 300), (1, 8, 8), 1e-3, 7, (16, 16)),
    ((2, 40, 600), (1, 16, 32), 1e-3, 7, (16, 16)),
    ((16, 20, 300), (8, 8, 8), 1e-3, 7, (16, 16)),
    ((17, 24, 280), (8, 8, 8), 1e-3, 13, (32, 32)),
])
def test_perceptron_container_and_decode_match_oracle(pc, O, shape, block, eb, k, h):
    x = gen.positive_lognormal(shape, 3.0, 5, 1.5)
    w = O.init_weights(k, h[0], h[1], seed=7)
    w = (w + np.random.default_rng(1).standard_normal(w.size).astype(np.float32) * np.float32(0.05)).astype(np.float32)
    got, y = run_gpu(pc, x, eb, block, weights=w, stencil=k, hidden=h, s_in=5)
    st, want, d = O.compress(x, eb, block=block, weights=w, stencil=k, h1=h[0], h2=h[1], s_in=5, dump=True)
    assert st == 0
    if shape[0] > 1 and d["nnflag"].size >= 8:   # the larger 3-D cases exercise both predictors
        assert 0 < d["nnflag"].sum() < d["nnflag"].size
    assert_same(got, want)
    st, yo = O.decompress(want)
    assert same_bits(y, yo.reshape(x.shape))
    check_roundtrip(x, y, eb)


def test_edge_fields(pc, O):
    rng = np.random.default_rng(3)
    fields = [
        np.zeros((5, 6, 7), np.float32),
        np.full((9, 9, 9), -3.25, np.float32),
        np.array([[[1.5]]], np.float32),
        np.array([1e-40, -0.0, 0.0, -1e-42, 7.0, -7.0, 3e38, -2e-38], np.float32).reshape(1, 2, 4),
        (rng.standard_normal((8, 8, 9)) * 1e30).astype(np.float32),
    ]
    z = np.zeros((10, 10, 10), np.float32)
    z[::3] = -0.0
    fields.append(z)
    for x in fields:
        for eb in (1e-2, 1e-4):
            got, y = run_gpu(pc, x, eb, (4, 4, 4))
            st, want = O.compress(x, eb, block=(4, 4, 4))
            assert st == 0
            assert_same(got, want)
            assert same_bits(y, x) or np.all(np.abs(y.astype(np.float64) - x) <= eb * np.abs(x.astype(np.float64)))
            assert np.array_equal(np.signbit(x), np.signbit(y))


def test_error_statuses(pc):
    x = torch.ones((4, 4, 4), dtype=torch.float32, device="cuda")
    x[1, 2, 3] = float("nan")
    with pytest.raises(pc.PcError) as e:
        pc.compress(x, pc.make_params(1e-2, (4, 4, 4)))
    assert e.value.status == -3
    x[1, 2, 3] = float("inf")
    with pytest.raises(pc.PcError) as e:
        pc.compress(x, pc.make_params(1e-2, (4, 4, 4)))
    assert e.value.status == -3
    y = torch.ones((4, 4, 4), dtype=torch.float32, device="cuda")
    for eb in (0.0, 1.0, -1.0):
        with pytest.raises(pc.PcError) as e:
            pc.compress(y, pc.make_params(eb, (4, 4, 4)))
        assert e.value.status == -1
    y[0, 0, 0] = 1e-30
    y[0, 0, 1] = 1e30
    with pytest.raises(pc.PcError) as e:
        pc.compress(y, pc.make_params(1e-9, (4, 4, 4)))
    assert e.value.status == -8
    with pytest.raises(pc.PcError):
        pc.compress(y, pc.make_params(1e-2, (3, 5, 7)))   # block shape without a compiled kernel
    assert pc.pc_strerror(-5) == "corrupt compressed stream"


def test_corrupt_payload_is_rejected_or_decoded(pc, O):
    x = gen.signed_lognormal((16, 16, 24), 3.0, 2, 2.0, 0.05)
    got, _ = run_gpu(pc, x, 1e-2)
    blob = bytearray(got)
    rng = np.random.default_rng(9)
    off_bb = struct.unpack_from("<Q", blob, 184)[0]
    for trial in range(25):
        bad = bytearray(blob)
        pos = int(rng.integers(off_bb, len(bad)))
        bad[pos] ^= int(rng.integers(1, 256))
        t = torch.from_numpy(np.frombuffer(bytes(bad), np.uint8).copy()).cuda()
        try:
            pc.decompress(t)
        except pc.PcError as e:
            assert e.status == -5
    # header damage is caught by the CRC
    bad = bytearray(blob)
    bad[20] ^= 1
    with pytest.raises(pc.PcError) as e:
        pc.decompress(torch.from_numpy(np.frombuffer(bytes(bad), np.uint8).copy()).cuda())
    assert e.value.status == -5
    # truncation
    with pytest.raises(pc.PcError) as e:
        pc.decompress(torch.from_numpy(np.frombuffer(bytes(blob[:-32]), np.uint8).copy()).cuda())
    assert e.value.status == -5


def test_host_buffer_entry_points(pc, O):
    x = gen.signed_lognormal((12, 40, 40), 3.0, 4, 2.0, 0.02)
    p = pc.make_params(1e-3, (8, 8, 8))
    cap = pc.pc_compress_bound(x.shape, pc.PC_F32, p)
    dfield = torch.empty(x.size, dtype=torch.float32, device="cuda")
    dout = torch.empty(cap, dtype=torch.uint8, device="cuda")
    ws = torch.empty(pc.pc_compress_workspace_size(x.shape, pc.PC_F32, p), dtype=torch.uint8, device="cuda")
    hout = np.zeros(cap, np.uint8)
    n = pc.pc_compress_host(x, p, hout, dfield, dout, ws)
    st, want = O.compress(x, 1e-3)
    assert_same(hout[:n].tobytes(), want)
    dims, dt, wsb = pc.pc_header_info(hout[:256].tobytes())
    assert dims == x.shape and dt == pc.PC_F32
    ws2 = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    hy = np.zeros(x.shape, np.float32)
    pc.pc_decompress_host(hout[:n], n, hy, dout, dfield, ws2)
    st, yo = O.decompress(want)
    assert same_bits(hy, yo.reshape(x.shape))


def lattice_field(nb, nlev, seed, eb, B=64):
    """2-D field (1, nb0*B, nb1*B) whose Lorenzo residual codes inside each
    B x B block are chosen exactly: Fibonacci counts (1, 1, 2, 3, 5, ...) for
    nlev distinct residuals, zero elsewhere.  Values sit on the quantization
    lattice 2^(d * 2 log2(1+eb)) with d the per-block 2-D prefix sums of the
    residuals (first row and column of every block zero), so the histogram
    has the Fibonacci shape that drives a Huffman tree deepest."""
    rng = np.random.default_rng(seed)
    f = [1, 1]
    while len(f) < nlev:
        f.append(f[-1] + f[-2])
    vals = np.concatenate([np.full(c, (k // 2 + 1) * (1 if k % 2 else -1)) for k, c in enumerate(f)])
    nin = nb[0] * nb[1] * (B - 1) ** 2
    r = np.concatenate([vals, np.zeros(nin - vals.size, np.int64)])
    rng.shuffle(r)
    r = r.reshape(nb[0], nb[1], B - 1, B - 1)
    d = np.zeros((nb[0], nb[1], B, B), np.int64)
    d[:, :, 1:, 1:] = r.cumsum(axis=2).cumsum(axis=3)
    d = d.transpose(0, 2, 1, 3).reshape(1, nb[0] * B, nb[1] * B)
    return np.exp2(d * 2 * np.log2(1 + eb)).astype(np.float32)


def test_length_limit_on_fibonacci_histogram(pc, O):
    """Huffman depth beyond 24 bits: the T.81 Annex K.3 limit must act the same way."""
    x = lattice_field((15, 15), 28, 5, 1e-3)
    st, want, d = O.compress(x, 1e-3, block=(1, 64, 64), dump=True)
    assert st == 0
    assert int(O.huffman_lengths(d["hist"], 64).max()) > 24 and int(d["lens"].max()) == 24
    got, y = run_gpu(pc, x, 1e-3, (1, 64, 64))
    assert_same(got, want)
    st, yo = O.decompress(want)
    assert same_bits(y, yo.reshape(x.shape))


def test_many_used_symbols(pc, O):
    """White log-normal noise: tens of thousands of used symbols, so the
    codebook sorts and merges in the workspace before shared memory."""
    rng = np.random.default_rng(3)
    x = (np.exp2(rng.normal(0, 6.4, (48, 64, 64))) * np.where(rng.random((48, 64, 64)) < 0.5, -1, 1)).astype(np.float32)
    st, want, d = O.compress(x, 1e-3, block=(8, 8, 8), dump=True)
    assert st == 0 and int((d["hist"] > 0).sum()) > 40000
    got, y = run_gpu(pc, x, 1e-3, (8, 8, 8))
    assert_same(got, want)
    st, yo = O.decompress(want)
    assert same_bits(y, yo.reshape(x.shape))
    check_roundtrip(x, y, 1e-3)
