"""Pins for the training phase's selection by simulated compression and the
coverage rule for m (Section IV.C).

Hand-computed: the simulated size is the Huffman-coded size of the
predictor's validation codes under their own histogram plus the stored value
of every balance point; the coverage rule picks the m whose coverage is
closest to 50% (eb_rel < 1.5%) or 80% (otherwise), the larger m on a tie.
"""
import numpy as np

from paper_2309_09778_gb300 import gen


def test_simulated_size_by_hand(O):
    # Lorenzo on all-zero inputs predicts 0, so residual = target.
    tg = np.array([0, 0, 0, 0, 1, 1, -1, 100], np.int32)
    inp = np.zeros((tg.size, 7), np.int32)
    use = np.ones(tg.size, np.uint8)
    # m = 4 (R = 8): codes 8, 8, 8, 8, 9, 9, 7 and a balance point (|100| > 7).
    # Histogram {8: 4, 9: 2, 7: 1, 0: 1}; Huffman: merge the two 1s, then 9 (2) with
    # that node (2, leaf first), then 8 (4): lengths 8 -> 1, 9 -> 2, 7 -> 3, 0 -> 3.
    # Bits 4*1 + 2*2 + 1*3 + 1*3 = 14, plus one stored value of 32 (or 64) bits.
    assert O.val_size(None, 7, 2, 0, 0, inp, tg, use, m=4, value_bits=32) == 46
    assert O.val_size(None, 7, 2, 0, 0, inp, tg, use, m=4, value_bits=64) == 78
    # m = 16: no balance point, the same weight pattern: 14 bits
    assert O.val_size(None, 7, 2, 0, 0, inp, tg, use, m=16, value_bits=32) == 14
    # an unused sample does not count: drop the 100 -> {8: 4, 9: 2, 7: 1}: lengths 1, 2, 2 -> 4 + 4 + 2 = 10
    use[7] = 0
    assert O.val_size(None, 7, 2, 0, 0, inp, tg, use, m=4, value_bits=32) == 10


def test_coverage_rule_by_hand(O):
    # residual bit lengths 0, 1, 2, 2, 3, 4, 5, 6, 7, 10: coverage(m) = share with bitlen <= m - 1
    # m = 2: 0.2, 3: 0.4, 4: 0.5, 5: 0.6, 6: 0.7, 7: 0.8, 8..10: 0.9, 11..16: 1.0
    tg = np.array([0, 1, 2, 3, 5, 9, 17, 40, 100, 1000], np.int32)
    inp = np.zeros((tg.size, 7), np.int32)
    use = np.ones(tg.size, np.uint8)
    assert O.coverage_m(None, 7, 2, 0, 0, inp, tg, use, 1e-3) == 4     # closest to 50%
    assert O.coverage_m(None, 7, 2, 0, 0, inp, tg, use, 2e-2) == 7     # closest to 80%
    # a tie (50% at m = 2 and at m = 3) goes to the larger m
    tg2 = np.array([1, 1, 5, 5], np.int32)
    assert O.coverage_m(None, 7, 2, 0, 0, np.zeros((4, 7), np.int32), tg2, np.ones(4, np.uint8), 1e-3) == 3


def test_select_keeps_the_smallest_simulated_size(O):
    x = gen.positive_lognormal((32, 40, 40), 3.0, 1, 1.5)
    lrs = np.array([3e-2, 1e-1, 0.0], np.float32)
    lams = np.array([0.0, 1e-4, 0.0], np.float32)
    best, W, s_in, sizes, m = O.train_select(x, 1e-2, k=7, h1=8, h2=8, seed=1, thr32=int(0.5 * 2 ** 32),
                                             lrs=lrs, lams=lams)
    # the learning-rate-0 model is the Lorenzo-equal initialisation: it ties with Lorenzo
    assert sizes[2] == sizes[3]
    want = -1
    for h in range(3):
        if sizes[h] < (sizes[want] if want >= 0 else sizes[3]):
            want = h
    assert best == want and best >= 0
    assert 2 <= m <= 16
