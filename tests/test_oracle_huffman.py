"""Pins for Huffman code lengths, canonical codes and bit packing (steps a9-a12).

Optimality is checked against brute-force enumeration of length vectors and
against the textbook cost (sum of merged weights, computed with heapq); the
canonical construction against the worked example printed in RFC 1951
Section 3.2.2 (tests/golden/rfc1951_canonical.txt).
"""
import heapq
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def huffman_cost_heapq(freqs):
    """Textbook optimum: the sum of all merged node weights."""
    h = [f for f in freqs if f > 0]
    if len(h) <= 1:
        return sum(h)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a = heapq.heappop(h); b = heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def brute_force_cost(freqs, lmax):
    f = [x for x in freqs if x > 0]
    n = len(f)
    if n == 1:
        return f[0]
    best = None
    for lens in itertools.product(range(1, lmax + 1), repeat=n):
        if sum(2.0 ** -l for l in lens) <= 1.0 + 1e-12:
            c = sum(a * b for a, b in zip(f, lens))
            best = c if best is None else min(best, c)
    return best


def test_huffman_optimal_vs_enumeration(O):
    rng = np.random.default_rng(1)
    for n in range(1, 7):
        for _ in range(25):
            hist = np.zeros(16, np.uint64)
            syms = rng.choice(16, n, replace=False)
            hist[syms] = rng.integers(1, 40, n)
            lens = O.huffman_lengths(hist)
            cost = int((hist * lens).sum())
            assert cost == brute_force_cost(hist.tolist(), 6)
            assert cost == huffman_cost_heapq(hist.tolist()) or n == 1


def test_huffman_kraft_and_monotone(O):
    rng = np.random.default_rng(2)
    for _ in range(40):
        nsym = int(rng.integers(2, 3000))
        hist = np.zeros(65536, np.uint64)
        idx = rng.choice(65536, nsym, replace=False)
        hist[idx] = rng.geometric(0.01, nsym)
        lens = O.huffman_lengths(hist)
        used = hist > 0
        assert np.all((lens > 0) == used)
        kraft = sum(2.0 ** -int(l) for l in lens[used])
        assert abs(kraft - 1.0) < 1e-12
        assert int((hist * lens).sum()) == huffman_cost_heapq(hist.tolist())
        # more frequent symbols never get longer codes
        f = hist[used]; l = lens[used]
        order = np.argsort(f, kind="stable")
        assert np.all(np.diff(l[order].astype(int)) <= 0)


def test_huffman_length_limit(O):
    """Fibonacci weights force a deep tree; the T.81 Annex K.3 adjustment keeps
    the Kraft sum at one and every length within the limit."""
    fib = [1, 1]
    while len(fib) < 30:
        fib.append(fib[-1] + fib[-2])
    hist = np.zeros(64, np.uint64)
    hist[:30] = fib
    free = O.huffman_lengths(hist, lmax=64)
    assert free.max() == 29
    for lmax in (5, 8, 12, 24):
        lens = O.huffman_lengths(hist, lmax=lmax)
        used = hist > 0
        assert lens[used].max() <= lmax
        assert abs(sum(2.0 ** -int(l) for l in lens[used]) - 1.0) < 1e-12
        assert int((hist * lens).sum()) >= int((hist * free).sum())


def test_single_symbol(O):
    hist = np.zeros(8, np.uint64)
    hist[5] = 100
    lens = O.huffman_lengths(hist)
    assert lens[5] == 1 and lens.sum() == 1


def read_rfc_golden():
    rows = []
    with open(os.path.join(GOLDEN, "rfc1951_canonical.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                sym, ln, code = line.split()
                rows.append((sym, int(ln), code))
    return rows


def test_canonical_rfc1951_example(O):
    """The ordered construction with RFC 1951's order (length, then symbol)
    reproduces the RFC's worked example."""
    rows = read_rfc_golden()
    lens = np.array([r[1] for r in rows], np.uint8)
    codes = O.canonical_codes(lens)
    for (sym, ln, code), got in zip(rows, codes.tolist()):
        assert format(got, f"0{ln}b") == code, sym


def test_code_order_is_most_frequent_first(O):
    """The compressor's code order lists symbols by descending frequency
    (ties: larger symbol first), lengths never decrease along it, and the
    ordered construction then yields a prefix-free code."""
    rng = np.random.default_rng(4)
    hist = np.zeros(512, np.uint64)
    hist[rng.choice(512, 200, replace=False)] = rng.integers(1, 50, 200)
    lens, order = O.huffman_lengths(hist, with_order=True)
    f = hist[order].astype(np.int64)
    assert np.all((np.diff(f) < 0) | ((np.diff(f) == 0) & (np.diff(order.astype(np.int64)) < 0)))
    assert np.all(np.diff(lens[order].astype(int)) >= 0)
    codes = O.canonical_codes(lens, order)
    words = sorted(format(int(codes[s]), f"0{int(lens[s])}b") for s in order)
    for a, b in zip(words, words[1:]):
        assert not b.startswith(a)


def test_canonical_prefix_free(O):
    rng = np.random.default_rng(3)
    hist = np.zeros(4096, np.uint64)
    hist[rng.choice(4096, 900, replace=False)] = rng.integers(1, 10 ** 6, 900)
    lens = O.huffman_lengths(hist)
    codes = O.canonical_codes(lens)
    words = sorted(format(int(c), f"0{int(l)}b") for c, l in zip(codes, lens) if l)
    for a, b in zip(words, words[1:]):
        assert not b.startswith(a)
