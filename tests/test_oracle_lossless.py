"""Pins for the lossless back-end stage (Section IV.A's fourth SZ stage): an
LZ77-style matcher over 16 KiB chunks of the bitstream bytes.

  - a 16-byte periodic string worked by hand: four literals, then one match of
    12 bytes at distance 4 (the copy overlaps its source), 8 token bytes;
  - a chunk whose tokens would not be shorter is stored as is;
  - decode(encode(x)) = x for periodic, random, mixed and multi-chunk inputs;
  - damaged sections (a distance beyond the output, a wrong size, a wrong
    raw length) are refused;
  - in a container the stage replaces exactly the stream section (flag 8,
    its length at byte 240), and the container decodes to the same field.
"""
import struct

import numpy as np
import pytest

from paper_2309_09778_gb300 import gen


def test_periodic_string_by_hand(O):
    sec = O.lz_encode(b"ABCD" * 4)
    # section header: 1 chunk of 16384 bytes, 16 raw bytes; table entry: 8 coded bytes
    assert struct.unpack_from("<IIQ", sec, 0) == (1, 16384, 16)
    assert struct.unpack_from("<I", sec, 16)[0] == 8
    assert sec[20:32] == bytes(12)  # table padded to 16 bytes
    # tokens: literal run of 4 (control 3), then match of 12 (control 128 + 8) at distance 4
    assert sec[32:] == bytes([3]) + b"ABCD" + bytes([136, 4, 0])
    st, raw = O.lz_decode(sec, 16)
    assert st == 0 and raw == b"ABCD" * 4


def test_incompressible_chunk_is_stored(O):
    rng = np.random.default_rng(0)
    data = rng.integers(0, 256, 1000, dtype=np.uint8).tobytes()
    sec = O.lz_encode(data)
    assert struct.unpack_from("<I", sec, 16)[0] == 1000 | 0x80000000
    assert sec[32:] == data


@pytest.mark.parametrize("kind", ["zeros", "random", "mixed", "long"])
def test_round_trip(O, kind):
    rng = np.random.default_rng(1)
    if kind == "zeros":
        data = bytes(40000)
    elif kind == "random":
        data = rng.integers(0, 256, 50004, dtype=np.uint8).tobytes()
    elif kind == "mixed":
        parts = [bytes(rng.integers(0, 4, 3000, dtype=np.uint8)), bytes(5000), b"xyz" * 2000,
                 rng.integers(0, 256, 7000, dtype=np.uint8).tobytes()]
        data = b"".join(parts * 3)
        data = data[: len(data) // 4 * 4]
    else:
        data = (b"0123456789abcdef" * 5000)[:65536 + 12]
    sec = O.lz_encode(data)
    nch = (len(data) + 16383) // 16384
    assert struct.unpack_from("<IIQ", sec, 0) == (nch, 16384, len(data))
    st, back = O.lz_decode(sec, len(data))
    assert st == 0 and back == data
    if kind in ("zeros", "long"):
        assert len(sec) < len(data) // 10


def test_damaged_sections_are_refused(O):
    sec = bytearray(O.lz_encode(b"ABCD" * 4))
    bad = bytearray(sec)
    bad[37] = 9                     # match distance 9 > the 4 bytes decoded so far
    assert O.lz_decode(bytes(bad), 16)[0] == -5
    bad = bytearray(sec)
    struct.pack_into("<I", bad, 16, 9)  # coded size past the section
    assert O.lz_decode(bytes(bad), 16)[0] == -5
    assert O.lz_decode(bytes(sec), 20)[0] == -5  # raw length differs from the header


def test_container_stage_replaces_the_stream(O):
    x = gen.signed_lognormal((40, 48, 64), 11 / 3, 0, 2.0, 0.6)  # 60% muted zeros: compressible runs
    st, plain = O.compress(x, 1e-2)
    st2, lz = O.compress(x, 1e-2, lossless=True)
    assert st == 0 and st2 == 0
    off_st = struct.unpack_from("<Q", plain, 208)[0]
    swords = struct.unpack_from("<Q", plain, 160)[0]
    stream = plain[off_st: off_st + 4 * swords]
    sec = O.lz_encode(stream)
    assert lz[:off_st][256:] == plain[:off_st][256:]           # every section before the stream
    assert struct.unpack_from("<I", lz, 228)[0] == 8
    assert struct.unpack_from("<Q", lz, 240)[0] == len(sec)
    assert lz[off_st: off_st + len(sec)] == sec
    assert len(lz) == (off_st + len(sec) + 15) // 16 * 16 and len(lz) < len(plain)
    st, y = O.decompress(lz)
    st2, y0 = O.decompress(plain)
    assert st == 0 and np.array_equal(y.view(np.uint32), y0.view(np.uint32))
