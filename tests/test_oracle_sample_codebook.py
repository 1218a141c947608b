"""Pins for the sample codebook and the single-pass container (Section IV.C: the
Huffman code built in the training phase from the validation set's averaged
per-block code frequencies, kept for the compression phase).

What fixes the oracle here:
  - the list construction by hand on a three-symbol histogram (most frequent
    first, ties by symbol, symbol 0 forced in);
  - averaging per block (every count divided by the same block count) leaves
    the code unchanged: scaled histograms give the same list;
  - with the field's own code as the "sample" code, every section equals the
    two-pass container's (whose packing other tests pin), only the stream and
    the balance values swap places;
  - a symbol dropped from the code turns exactly its points into balance
    points, whose stored values are the originals, and changes nothing else;
  - the sample code of a predictor costs the simulated size of Section IV.C
    (pinned by hand in test_oracle_select) under its own histogram;
  - malformed lists are refused.
"""
import struct

import numpy as np
import pytest

from paper_2309_09778_gb300 import gen


def sections(blob):
    """Header fields and sections of a container, whatever its layout."""
    h = {}
    h["n_used"] = struct.unpack_from("<I", blob, 116)[0]
    h["nblocks"], h["n_out"], h["swords"] = struct.unpack_from("<3Q", blob, 144)
    off_w, off_cb, off_bb, off_bn, off_ov, off_st, total = struct.unpack_from("<7Q", blob, 168)
    h["flags"] = struct.unpack_from("<I", blob, 228)[0]
    dt = struct.unpack_from("<I", blob, 8)[0]
    ts = 8 if dt == 1 else 4
    nb, no, sw = h["nblocks"], h["n_out"], h["swords"]
    h["cb"] = np.frombuffer(blob, "<u4", h["n_used"], off_cb)
    h["bb"] = np.frombuffer(blob, "<u4", nb, off_bb)
    h["bn"] = np.frombuffer(blob, "<u2", nb, off_bn)
    h["ov"] = bytes(blob[off_ov: off_ov + ts * no])
    h["st"] = np.frombuffer(blob, "<u4", sw, off_st)
    h["off_ov"], h["off_st"], h["total"] = off_ov, off_st, total
    h["w"] = bytes(blob[off_w: off_cb])
    return h


def test_list_by_hand(O):
    # m = 3, counts {5: 3, 7: 1}, symbol 0 absent -> forced to 1.
    # Leaves ascending by (count, symbol): (1, 0), (1, 7), (3, 5).  Merge 0 and 7 (weight 2),
    # then that node with 5: lengths 5 -> 1, 0 -> 2, 7 -> 2.  The list is the leaf order
    # reversed (most frequent first): 5, 7, 0.
    h = np.zeros(8, np.uint64)
    h[5], h[7] = 3, 1
    cb = O.sample_codebook(h, m=3)
    assert cb.tolist() == [5 | 1 << 16, 7 | 2 << 16, 0 | 2 << 16]
    # symbol 0 already present keeps its count: {0: 2, 5: 3, 7: 1}: (1, 7), (2, 0), (3, 5):
    # merge 7 and 0 (3), then 5 (3, leaf first) with it: 5 -> 1, 0 -> 2, 7 -> 2; order 5, 0, 7
    h[0] = 2
    assert O.sample_codebook(h, m=3).tolist() == [5 | 1 << 16, 0 | 2 << 16, 7 | 2 << 16]
    # a histogram with nothing but balance points: one symbol of length 1
    z = np.zeros(16, np.uint64)
    assert O.sample_codebook(z, m=4).tolist() == [0 | 1 << 16]
    # span fill: {5: 3, 7: 1} and symbol 0 forced, 6 (inside the sampled span 5..7) counts once:
    # leaves (1, 0), (1, 6), (1, 7), (3, 5); merge 0 and 6 (2), then 7 (1) with that node (3),
    # then 5 (3, leaf first) with it: lengths 5 -> 1, 7 -> 2, 0 -> 3, 6 -> 3; order 5, 7, 6, 0
    h = np.zeros(8, np.uint64)
    h[5], h[7] = 3, 1
    assert O.sample_codebook(h, m=3, span_fill=True).tolist() == [5 | 1 << 16, 7 | 2 << 16, 6 | 3 << 16,
                                                                   0 | 3 << 16]
    # codes beyond the span (1..4) stay without a code word; only symbol 0 when nothing else was seen
    assert O.sample_codebook(z, m=4, span_fill=True).tolist() == [0 | 1 << 16]


def test_average_per_block_is_the_same_code(O):
    rng = np.random.default_rng(3)
    h = np.zeros(1 << 10, np.uint64)
    idx = rng.integers(0, 1 << 10, 400)
    np.add.at(h, idx, rng.integers(1, 50, 400).astype(np.uint64))
    h[0] = 5  # present, so the forced count of symbol 0 does not apply
    base = O.sample_codebook(h, m=10)
    for s in (2, 7, 1000):
        assert np.array_equal(O.sample_codebook(h * np.uint64(s), m=10), base)


FORMS = {
    "lorenzo": dict(),
    "mlp": dict(stencil=7, h1=8, h2=8),
}


def _weights(O, x, eb, form):
    if form == "lorenzo":
        return None, 0
    best, W, s_in, _ = O.train(x, eb, k=7, h1=8, h2=8, seed=2, thr32=int(0.3 * 2 ** 32),
                               lrs=np.array([3e-2], np.float32), lams=np.array([0.0], np.float32))
    return W[0], s_in


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("shape,block", [((20, 27, 35), (8, 8, 8)), ((1, 45, 70), (1, 16, 32))])
def test_own_code_as_sample_code_gives_the_same_sections(O, form, shape, block):
    x = gen.signed_lognormal(shape, 3.0, 5, 2.0, 0.05)
    eb = 1e-3
    w, s_in = _weights(O, x, eb, form)
    kw = dict(block=block, weights=w, s_in=s_in, **FORMS[form])
    st, two = O.compress(x, eb, **kw)
    assert st == 0
    a = sections(two)
    st, one = O.compress(x, eb, codebook=a["cb"].copy(), **kw)
    assert st == 0
    b = sections(one)
    assert a["flags"] == 0 and b["flags"] == 1
    for key in ("n_used", "nblocks", "n_out", "swords", "w"):
        assert a[key] == b[key], key
    for key in ("cb", "bb", "bn", "st"):
        assert np.array_equal(a[key], b[key]), key
    assert a["ov"] == b["ov"]
    # the stream now precedes the balance values, each 16-byte aligned
    assert b["off_st"] < b["off_ov"] and b["off_st"] % 16 == 0 and b["off_ov"] % 16 == 0
    assert b["off_ov"] == (b["off_st"] + 4 * b["swords"] + 15) // 16 * 16
    assert b["total"] == len(one)
    st, y1 = O.decompress(two)
    st2, y2 = O.decompress(one)
    assert st == 0 and st2 == 0 and np.array_equal(y1.view(np.uint8), y2.view(np.uint8))


def test_dropped_symbol_becomes_balance_points(O):
    x = gen.signed_lognormal((24, 24, 40), 3.0, 8, 2.0, 0.05)
    eb = 1e-3
    st, two, d = O.compress(x, eb, dump=True)
    assert st == 0
    hist = d["hist"].copy()
    codes = d["codes"].reshape(-1, 512)
    # drop the third most frequent code (not 0)
    order = np.argsort(-hist.astype(np.int64), kind="stable")
    s = int([c for c in order if c != 0][2])
    h2 = hist.copy()
    h2[s] = 0
    cb = O.sample_codebook(h2, m=16)
    assert s not in (cb & 0xFFFF).tolist()
    st, one, d1 = O.compress(x, eb, codebook=cb, dump=True)
    assert st == 0
    c1 = d1["codes"].reshape(-1, 512)
    # exactly the points that had code s are now balance points; nothing else moved
    assert np.array_equal(c1 == 0, (codes == 0) | (codes == s))
    assert np.array_equal(c1[codes != s], codes[codes != s])
    a, b = sections(two), sections(one)
    assert b["n_out"] == a["n_out"] + int(hist[s])
    # each block's bits: the remaining codes under the list's lengths
    lens = np.zeros(1 << 16, np.int64)
    lens[cb & 0xFFFF] = cb >> 16
    want = np.array([lens[c1[i, 1:]].sum() for i in range(c1.shape[0])])
    assert np.array_equal(b["bb"] & 0x7FFFFFFF, want.astype(np.uint32))
    st, y = O.decompress(one)
    assert st == 0
    # the points with code s come back bit-exact (stored values); the rest as before
    st, y2 = O.decompress(two)
    xb = x.reshape(3, 8, 3, 8, 5, 8).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 512)
    yb = y.reshape(3, 8, 3, 8, 5, 8).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 512)
    y2b = y2.reshape(3, 8, 3, 8, 5, 8).transpose(0, 2, 4, 1, 3, 5).reshape(-1, 512)
    hit = codes == s
    assert hit.sum() == hist[s] > 0
    assert np.array_equal(yb[hit].view(np.uint32), xb[hit].view(np.uint32))
    assert np.array_equal(yb[~hit].view(np.uint32), y2b[~hit].view(np.uint32))


def test_sample_code_costs_the_simulated_size(O):
    # the sample code is the Huffman code of the validation histogram, so the validation
    # codes cost exactly the coded part of the simulated size (Section IV.C, pinned by hand)
    x = gen.positive_lognormal((24, 32, 32), 3.0, 4, 1.5)
    eb, thr = 1e-2, int(0.4 * 2 ** 32)
    _, (vin, vtg, vus) = O.gather_samples(x, eb, (8, 8, 8), 7, 3, thr)
    for m in (16, 6):
        h = O.val_hist(None, 7, 2, 0, 0, vin, vtg, vus, m=m)
        assert h[0] > 0 or m == 16
        cb = O.sample_codebook_for(x, eb, k=7, m=m, seed=3, thr32=thr)
        lens = np.zeros(1 << m, np.int64)
        lens[cb & 0xFFFF] = cb >> 16
        size = O.val_size(None, 7, 2, 0, 0, vin, vtg, vus, m=m, value_bits=32)
        if h[0] > 0:
            assert int((h.astype(np.int64) * lens).sum()) + 32 * int(h[0]) == size
        assert lens[0] > 0


@pytest.mark.parametrize("bad", ["dup", "decreasing", "kraft", "no_zero", "range", "single_long"])
def test_malformed_lists_are_refused(O, bad):
    x = gen.positive_lognormal((8, 8, 16), 3.0, 1, 1.0)
    st, two = O.compress(x, 1e-2)
    cb = sections(two)["cb"].copy()
    assert cb.size > 3
    if bad == "dup":
        cb[2] = (cb[2] & 0xFFFF0000) | (cb[1] & 0xFFFF)
    elif bad == "decreasing":
        cb = cb[::-1].copy()
    elif bad == "kraft":
        cb[-1] = (cb[-1] & 0xFFFF) | (1 << 16)
        cb = np.concatenate([cb[-1:], cb[:-1]])
    elif bad == "no_zero":
        cb = cb[(cb & 0xFFFF) != 0]
    elif bad == "range":
        cb[0] = (cb[0] & 0xFFFF0000) | 0xFFFF
        st, two = O.compress(x, 1e-2, m=8)
        cb8 = sections(two)["cb"].copy()
        cb8[0] = (cb8[0] & 0xFFFF0000) | 300
        assert O.compress(x, 1e-2, m=8, codebook=cb8)[0] == -1
        return
    elif bad == "single_long":
        cb = np.array([0 | 2 << 16], np.uint32)
    assert O.compress(x, 1e-2, codebook=cb)[0] == -1


def test_span_fill_leaves_only_codes_beyond_the_span(O):
    # with span fill, a point becomes a balance point only when its code lies outside the
    # sampled span (or outside the quantization range / bound check, as without a codebook)
    x = gen.positive_lognormal((32, 64, 64), 2.0, 0, 1.5)
    eb, thr = 1e-4, int(0.05 * 2 ** 32)
    _, (vin, vtg, vus) = O.gather_samples(x, eb, (8, 8, 8), 7, 0, thr)
    h = O.val_hist(None, 7, 2, 0, 0, vin, vtg, vus, m=16)
    nz = np.flatnonzero(h[1:]) + 1
    lo, hi = int(nz.min()), int(nz.max())
    cb = O.sample_codebook_for(x, eb, seed=0, thr32=thr, span_fill=True)
    syms = set((cb & 0xFFFF).tolist())
    assert syms == set(range(lo, hi + 1)) | {0}
    st, two, d2 = O.compress(x, eb, dump=True)
    st, one, d1 = O.compress(x, eb, codebook=cb, dump=True)
    c2, c1 = d2["codes"], d1["codes"]
    moved = (c1 == 0) & (c2 != 0)
    assert moved.any()
    assert np.all((c2[moved] < lo) | (c2[moved] > hi))
    assert np.array_equal(c1[~moved], c2[~moved])
    # and it codes far closer to the field's own code than the literal reading
    st, lit = O.compress(x, eb, codebook=O.sample_codebook_for(x, eb, seed=0, thr32=thr))
    assert len(one) < len(lit)
