"""Round-trip invariants and the container layout of the oracle.

The pointwise relative bound (Eq. 1) must hold on every point, zeros and signs
must come back exactly (Section III.B), balance points bit-exactly
(Section IV.D.1), and the bitstream must be the concatenation of the canonical
code words of the block codes in block order, MSB first.
"""
import struct

import numpy as np
import pytest

from paper_2309_09778_gb300 import gen

R = 1 << 15


def check_bound(x, y, eb):
    assert y.shape == x.shape and y.dtype == x.dtype
    xd = x.astype(np.float64)
    yd = y.astype(np.float64)
    if x.dtype == np.float64:
        from fractions import Fraction
        bad = np.abs(yd - xd) > eb * np.abs(xd)
        for i in np.flatnonzero(bad.ravel())[:50]:
            a, b = Fraction(x.ravel()[i]), Fraction(y.ravel()[i])
            assert abs(a - b) <= Fraction(eb) * abs(a)
    else:
        # float32 differences and products are exact in float64
        assert np.all(np.abs(yd - xd) <= eb * np.abs(xd))
    assert np.array_equal(np.signbit(x), np.signbit(y))
    assert np.array_equal(x == 0, y == 0)


@pytest.mark.parametrize("seed", range(12))
def test_invariant_sweep(O, seed):
    rng = np.random.default_rng(100 + seed)
    shape = tuple(int(s) for s in rng.integers(1, 23, 3))
    block = tuple(int(b) for b in rng.choice([1, 2, 4, 8], 3))
    if np.prod(block) < 2:
        block = (2, 2, 2)
    eb = float(10 ** rng.uniform(-4, -1))
    dt = np.float32 if seed % 3 else np.float64
    x = gen.signed_lognormal(shape, float(rng.uniform(2, 5)), seed, float(rng.uniform(0.5, 4)),
                             float(rng.uniform(0, 0.2)), dtype=dt)
    if seed % 4 == 0:
        x.ravel()[:: 7] = -0.0
    st, blob = O.compress(x, eb, block=block)
    assert st == 0
    st, y = O.decompress(blob)
    assert st == 0
    check_bound(x, y.reshape(x.shape), eb)


def test_tiny_and_degenerate_fields(O):
    for x in [np.zeros((1, 1, 1), np.float32), np.ones((1, 1, 2), np.float32),
              np.zeros((3, 3, 3), np.float32), np.full((5, 4, 3), -2.5, np.float32),
              np.array([1e-40, 0, -1e-41, 5e-42], np.float32).reshape(1, 1, 4)]:
        st, blob = O.compress(x, 1e-3, block=(2, 2, 2))
        assert st == 0
        st, y = O.decompress(blob)
        assert st == 0
        check_bound(x, y.reshape(x.shape), 1e-3)
        assert np.array_equal(x.view(np.uint32)[x == 0], y.reshape(x.shape).view(np.uint32)[x == 0])


def test_balance_points_bit_exact(O):
    x = gen.signed_lognormal((12, 12, 12), 3.0, 4, 3.0, 0.1)
    x.ravel()[::11] = -0.0
    x.ravel()[5] = np.float32(3e-39)
    st, blob, d = O.compress(x, 1e-3, dump=True)
    st, y = O.decompress(blob)
    y = y.reshape(x.shape)
    forced = d["ok"].reshape(x.shape) == 0
    assert np.array_equal(x[forced].view(np.uint32), y[forced].view(np.uint32))


def parse(blob):
    h = {}
    (h["dtype"], h["pred"]) = struct.unpack_from("<II", blob, 8)
    h["dims"] = struct.unpack_from("<3Q", blob, 16)
    h["block"] = struct.unpack_from("<3I", blob, 40)
    h["m"] = struct.unpack_from("<I", blob, 64)[0]
    h["n_used"] = struct.unpack_from("<I", blob, 116)[0]
    h["nblocks"], h["n_out"], h["swords"] = struct.unpack_from("<3Q", blob, 144)
    h["off"] = struct.unpack_from("<7Q", blob, 168)
    return h


def test_bitstream_is_concatenated_codewords(O):
    x = gen.signed_lognormal((17, 18, 19), 4.0, 9, 2.0, 0.03)
    st, blob, d = O.compress(x, 1e-2, dump=True)
    h = parse(blob)
    lens = d["lens"]
    cb = np.frombuffer(blob, np.uint32, h["n_used"], h["off"][1])
    codes_cw = O.canonical_codes(lens, cb & 0xFFFF)
    # expected bit string, written independently of the oracle's packer
    bits = []
    shape, block = x.shape, (8, 8, 8)
    nb = [(shape[i] + 7) // 8 for i in range(3)]
    b = 0
    bb = np.frombuffer(blob, np.uint32, h["nblocks"], h["off"][2])
    for bz in range(nb[0]):
        for by in range(nb[1]):
            for bx in range(nb[2]):
                e = [min(8, shape[0] - 8 * bz), min(8, shape[1] - 8 * by), min(8, shape[2] - 8 * bx)]
                npt = e[0] * e[1] * e[2]
                cs = d["codes"][b * 512 + 1:b * 512 + npt]
                s = "".join(format(int(codes_cw[c]), f"0{int(lens[c])}b") for c in cs)
                assert (int(bb[b]) & 0x7FFFFFFF) == len(s)
                bits.append(s)
                b += 1
    allbits = "".join(bits)
    words = np.frombuffer(blob, np.uint32, h["swords"], h["off"][5])
    got = "".join(format(int(w), "032b") for w in words)
    assert got[: len(allbits)] == allbits
    assert set(got[len(allbits):]) <= {"0"}
    # codebook section lists (symbol, length) in code order: most frequent first
    _, order = O.huffman_lengths(d["hist"], with_order=True)
    assert np.array_equal(cb & 0xFFFF, order)
    assert np.array_equal(cb >> 16, lens[order])
    # total size is a multiple of 16 and equals the stored size
    assert len(blob) % 16 == 0 and struct.unpack_from("<Q", blob, 216)[0] == len(blob)


def test_corrupt_streams_are_rejected(O):
    x = gen.signed_lognormal((10, 10, 10), 3.0, 2, 2.0, 0.05)
    st, blob = O.compress(x, 1e-2)
    assert O.decompress(blob[:100])[0] == -5
    for off in (0, 4, 20, 100, 200):
        bad = bytearray(blob)
        bad[off] ^= 0x40
        assert O.decompress(bytes(bad))[0] == -5
    rng = np.random.default_rng(0)
    h = parse(blob)
    for _ in range(30):
        bad = bytearray(blob)
        pos = int(rng.integers(h["off"][2], len(blob)))
        bad[pos] ^= int(rng.integers(1, 256))
        st, y = O.decompress(bytes(bad))
        assert st in (0, -5)   # never a crash; payload damage may decode to other values
    assert O.decompress(blob[: len(blob) - 16])[0] == -5


@pytest.mark.parametrize("form", ["lorenzo", "fp32", "fixed"])
def test_block_codes_equal_full_compression(O, form):
    """The per-block export (used to check sampled blocks of full-size fields)
    gives every block's stored codes and perceptron flag exactly as the full
    compressor does, truncated edge blocks included."""
    x = gen.signed_lognormal((19, 21, 26), 3.0, 8, 2.0, 0.05)
    eb = 1e-2
    kw = {}
    if form != "lorenzo":
        best, W, s_in, _ = O.train(x, eb, k=7, h1=16, h2=16, seed=2)
        w = W[best if best >= 0 else 0]
        kw = dict(weights=w, s_in=s_in) if form == "fp32" else dict(qnet=O.quantize(x, eb, w, s_in, seed=2), s_in=s_in)
    st, blob, d = O.compress(x, eb, dump=True, **kw)
    assert st == 0
    c = O.consts_for(x, eb)
    nb = 3 * 3 * 4
    for bi in range(nb):
        codes, usen = O.block_codes(x, c, bi, eb, **kw)
        assert usen == bool(d["nnflag"][bi])
        assert np.array_equal(codes[1:], d["codes"][bi * 512 + 1: bi * 512 + codes.size])
