"""Pins of the oracle's histogram-voting inlier preselection (Sec. II): a
common displacement, a hand-counted example, the range and bin-edge rules,
and the property it exists for -- with 85 % outliers the top-ranked matches
are inliers."""
import numpy as np

import oracle
import synth


def _uv(disp, base=(100.0, 50.0)):
    d = np.asarray(disp, np.float32)
    uv1 = np.tile(np.asarray(base, np.float32), (len(d), 1))
    return uv1, uv1 + d


def test_common_displacement():
    uv1, uv2 = _uv([(5.0, -2.0)] * 7)
    hist, score, order = oracle.vote_matches(uv1, uv2, 4.0, 32.0)
    assert hist.shape == (16, 16) and hist.sum() == 7
    assert np.all(score == 7) and np.array_equal(order, np.arange(7))


def test_hand_counted_example():
    # bin 4, range 16: bin x = floor((du + 16) / 4)
    disp = [(1.0, 1.0),      # bin (4, 4)
            (30.0, 0.0),     # bin (11, 4): far away
            (2.0, 3.0),      # bin (4, 4)
            (5.0, 1.0),      # bin (5, 4): next to (4, 4)
            (-1.0, 2.0),     # bin (3, 4)
            (3.5, 3.9)]      # bin (4, 4)
    uv1, uv2 = _uv(disp)
    hist, score, order = oracle.vote_matches(uv1, uv2, 4.0, 16.0)
    assert hist[4, 4] == 3 and hist[4, 5] == 1 and hist[4, 3] == 1 and hist.sum() == 5  # (30, 0) out of range
    # (4,4): 3 + 1 + 1 = 5; (5,4): 1 + 3 = 4; (3,4): 1 + 3 = 4; out of range: 0
    assert list(score) == [5, 0, 5, 4, 4, 5]
    assert list(order) == [0, 2, 5, 3, 4, 1]


def test_bin_edges_and_range():
    # du + range exactly on a bin edge goes to the upper bin; -range is in, +range is out
    uv1, uv2 = _uv([(-8.0, 0.0), (-16.0, 0.0), (16.0, 0.0), (0.0, 0.0)])
    hist, score, order = oracle.vote_matches(uv1, uv2, 4.0, 16.0)
    assert hist[4, 2] == 1 and hist[4, 0] == 1 and hist[4, 4] == 1 and hist.sum() == 3
    assert score[2] == 0 and order[-1] == 2


def test_inliers_rank_first_with_85_percent_outliers():
    uv1, uv2, inl = synth.feature_matches(12345, n=4000, inlier_frac=0.15)
    hist, score, order = oracle.vote_matches(uv1, uv2, 4.0, 128.0)
    top = order[: inl.sum() // 2]
    assert inl[top].mean() >= 0.95
    # scores are non-increasing along the order, ties by index
    s = score[order]
    assert np.all(np.diff(s) <= 0)
    same = np.diff(s) == 0
    assert np.all(np.diff(order)[same] > 0)
