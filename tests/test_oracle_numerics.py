"""Pins for the oracle's own log2/exp2, hash and checksum.

The log map (Eq. 6-8) and its inverse are evaluated by our own code: in
single precision by Tang's table-driven method (a 128-entry reciprocal table
and a short log2(1+r) series; a 32-entry table of 2^(j/32) and a short Taylor
series), in double precision by the atanh and Taylor series.  These tests
hold them to high-precision values from Python's decimal module and to exact
special cases.  The counter-based hash and the CRC are held to their published
definitions / library routines.
"""
import math
import zlib
from decimal import Decimal, getcontext

import numpy as np
import pytest

getcontext().prec = 60
LN2 = Decimal(2).ln()


def ulp32(v):
    return float(np.spacing(np.float32(abs(v)))) if v != 0 else 2.0 ** -149


def ulp64(v):
    return float(np.spacing(abs(float(v)))) if v != 0 else 2.0 ** -1074


def test_L32_powers_of_two_exact(O):
    for k in range(-126, 128):
        assert O.L32(2.0 ** k) == float(k)


def test_E32_integers_exact(O):
    for k in range(-149, 128):
        assert O.E32(float(k)) == 2.0 ** k


def test_L64_E64_exact_cases(O):
    for k in range(-1074, 1024, 7):
        assert O.L64(2.0 ** k) == float(k)
    for k in range(-1074, 1024, 5):
        assert O.E64(float(k)) == 2.0 ** k


def test_L32_accuracy(O):
    """Table-driven log2 (Tang's method): absolute error at most 2 ulp of the
    result plus 2^-24, i.e. relative accuracy except just below y = 1 where
    the result itself is tiny; the transform only needs absolute accuracy
    against the quantization step."""
    rng = np.random.default_rng(11)
    ys = np.concatenate([rng.uniform(0.5, 2.0, 4000), np.exp(rng.uniform(-87, 88, 4000)),
                         1.0 - rng.uniform(0, 1e-3, 500), 1.0 + rng.uniform(0, 1e-3, 500),
                         [np.float32(np.sqrt(2)), np.nextafter(np.float32(np.sqrt(2)), 0), 1.5, 0.75,
                          np.finfo(np.float32).tiny, np.finfo(np.float32).max]]).astype(np.float32)
    for y in ys.tolist():
        ex = Decimal(y).ln() / LN2
        L = O.L32(y)
        assert abs(Decimal(L) - ex) <= 2 * Decimal(ulp32(float(ex))) + Decimal(2) ** -24, (y, L, ex)


def test_E32_accuracy(O):
    rng = np.random.default_rng(12)
    ts = np.concatenate([rng.uniform(-126, 127, 4000), rng.uniform(-1, 1, 2000)]).astype(np.float32)
    for t in ts.tolist():
        ex = (Decimal(t) * LN2).exp()
        E = O.E32(t)
        assert abs(Decimal(E) - ex) <= 2 * Decimal(ulp32(float(ex))), (t, E, ex)


def test_L64_E64_accuracy(O):
    rng = np.random.default_rng(13)
    for y in np.exp(rng.uniform(-700, 700, 1500)).tolist() + [1.0 + 1e-15, 0.7071067811865476, 2.0 ** -1070]:
        ex = Decimal(y).ln() / LN2
        assert abs(Decimal(O.L64(y)) - ex) <= 8 * Decimal(ulp64(float(ex))), y
    for t in rng.uniform(-1000, 1000, 1500).tolist():
        ex = (Decimal(t) * LN2).exp()
        assert abs(Decimal(O.E64(t)) - ex) <= 8 * Decimal(ulp64(float(ex))), t


def test_L_E_roundtrip_monotone_region(O):
    # E(L(y)) returns y to within a few ulp: the pair inverts (Eq. 1-2 rely on it)
    rng = np.random.default_rng(14)
    for y in np.exp(rng.uniform(-80, 80, 2000)).astype(np.float32).tolist():
        r = O.E32(O.L32(y))
        assert abs(r - y) <= 256 * ulp32(y), (y, r)


def splitmix64_reference(seed):
    """SplitMix64 (Steele, Lea, Flood 2014): state += golden gamma, then mix."""
    M = (1 << 64) - 1
    state = seed & M
    while True:
        state = (state + 0x9E3779B97F4A7C15) & M
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        yield z ^ (z >> 31)


def test_mix64_is_splitmix64(O):
    for seed in (0, 1, 1234567, 2 ** 63 + 5):
        g = splitmix64_reference(seed)
        for i in range(20):
            assert O.mix64(seed, i) == next(g)


def test_crc32_matches_zlib(O):
    rng = np.random.default_rng(15)
    for n in (0, 1, 7, 252, 1000):
        b = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert O.crc32(b) == zlib.crc32(b)
