"""CPU pins of the hub-net threshold rule as the GPU tests restate it
(tests/hubrule.py): the smallest size on the ladder 512 * 2^(k/2) whose nets
above it, at the first round's bitmap width, take at most half the L2 cache.
The expected values below are worked out by hand from that rule."""
import numpy as np

import hubrule


def test_first_round_words_by_hand():
    # largest net 600, C = 64, Q = 16: colors up to 599 + 1024, plus C + 2
    # spare colors: 1689 -> 53 words (ceil(1689 / 32)), + 3 rounded down to
    # a multiple of 4 -> 56
    assert hubrule.first_round_words(600, 64, 16) == 56
    # largest net 5000: 4999 + 1024 + 66 = 6089 -> 191 words -> 194 -> 192
    assert hubrule.first_round_words(5000, 64, 16) == 192
    # no net: 0 + 1024 + 66 = 1090 -> 35 words -> 38 -> 36
    assert hubrule.first_round_words(0, 64, 16) == 36


def test_ladder():
    assert hubrule.LADDER[:6] == [512, 724, 1024, 1448, 2048, 2896]
    assert len(hubrule.LADDER) == 24 and hubrule.LADDER[-1] == 724 << 11


def test_no_net_above_the_floor():
    sizes = np.full(1000, 512)  # "more than" the threshold: none qualifies
    assert hubrule.expected_threshold(sizes, 64, 16, 1 << 27) == 512


def test_bitmaps_fit():
    # 100 nets of 600 members: 100 * 56 words * 4 B = 22,400 B, far below half
    # of a 126 MiB L2
    sizes = np.r_[np.full(100, 600), np.full(5000, 10)]
    assert hubrule.expected_threshold(sizes, 64, 16, 126 << 20) == 512


def test_bitmaps_spill_raise_the_threshold():
    sizes = np.r_[np.full(100, 600), np.full(5000, 10)]
    # half the L2 just below 22,400 B: 512 fails, 724 leaves no hub at all
    assert hubrule.expected_threshold(sizes, 64, 16, 2 * 22400 - 8) == 724
    # exactly 22,400 B: 512 fits
    assert hubrule.expected_threshold(sizes, 64, 16, 2 * 22400) == 512


def test_mixed_sizes():
    # 10 nets of 5000 and 1000 of 600, words 192: at 512 the hubs take
    # 1010 * 768 B = 775,680 B, above 724 only the 10 large ones, 7,680 B
    sizes = np.r_[np.full(10, 5000), np.full(1000, 600)]
    assert hubrule.expected_threshold(sizes, 64, 16, 2 * 100_000) == 724
    assert hubrule.expected_threshold(sizes, 64, 16, 2 * 775_680) == 512
    # a budget below 7,680 B: no ladder size up to 5000 fits, the first one
    # above every net (5792) does, with no hub
    assert hubrule.expected_threshold(sizes, 64, 16, 2 * 7_000) == 5792


def test_empty():
    assert hubrule.expected_threshold(np.zeros(0, np.int64), 64, 16, 1 << 27) == hubrule.NONE
