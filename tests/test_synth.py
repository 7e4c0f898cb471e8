"""The seeded generators: determinism, shapes and ranges, and that the right
view really is the left view seen through the ground-truth field (the oracle's
winner-take-all recovers it on textured pixels)."""
import numpy as np

import oracle
import synth


def test_deterministic_and_ranges():
    a = synth.perlin_pair(synth.seed_for(0))
    b = synth.perlin_pair(synth.seed_for(0))
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    L, R, gt = a
    assert L.shape == R.shape == gt.shape == (240, 320)
    assert L.dtype == np.uint8 and L.min() >= 20 and L.max() <= 235
    assert abs(gt.min() - 2.0) < 1e-9 and abs(gt.max() - 28.0) < 1e-9
    Lc, Rc, gtc = synth.tissue_pair(synth.seed_for(1), 320, 180)
    assert Lc.shape == Rc.shape == (180, 320, 3) and Lc.dtype == np.uint8
    assert abs(gtc.min() - 10) < 1e-9 and abs(gtc.max() - 110) < 1e-9


def test_right_view_follows_ground_truth():
    L, R, gt = synth.perlin_pair(synth.seed_for(0))
    ys = slice(40, 56)
    m = oracle.match(L[ys.start - 5:ys.stop + 5], R[ys.start - 5:ys.stop + 5], 0, 32, 5)
    dl = m["dL"][5:-5, 40:300].astype(float)
    err = np.abs(dl - gt[ys, 40:300])
    assert np.median(err) < 0.6
