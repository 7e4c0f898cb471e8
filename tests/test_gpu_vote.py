"""Histogram-voting inlier preselection on the GPU (Sec. II) against the
oracle: histogram, scores and the ranking bit-exact (integer work; the bin
decision is taken in single precision on both sides), on the synthetic
85 %-outlier matches at several sizes (ragged, a power of two, the maximum),
the hand-counted example, and the size limit."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    st.lib()
    return torch.device("cuda:0")


def _run(dev, uv1, uv2, bin, rng):
    t1 = torch.from_numpy(np.ascontiguousarray(uv1)).to(dev)
    t2 = torch.from_numpy(np.ascontiguousarray(uv2)).to(dev)
    h, s, o = st.stereo_vote_matches(t1, t2, bin, rng)
    torch.cuda.synchronize()
    return h.cpu().numpy(), s.cpu().numpy(), o.cpu().numpy()


@pytest.mark.parametrize("n", [1, 777, 2048, 5000, 16384])
def test_synthetic_matches(dev, n):
    uv1, uv2, inl = synth.feature_matches(synth.seed_for(7, n % 97), n=n, inlier_frac=0.15)
    g = _run(dev, uv1, uv2, 4.0, 128.0)
    r = oracle.vote_matches(uv1, uv2, 4.0, 128.0)
    for a, b in zip(g, r):
        assert np.array_equal(a, b)


def test_hand_counted_example(dev):
    d = np.array([(1.0, 1.0), (30.0, 0.0), (2.0, 3.0), (5.0, 1.0), (-1.0, 2.0), (3.5, 3.9)], np.float32)
    uv1 = np.tile(np.array([100.0, 50.0], np.float32), (6, 1))
    h, s, o = _run(dev, uv1, uv1 + d, 4.0, 16.0)
    assert list(s) == [5, 0, 5, 4, 4, 5] and list(o) == [0, 2, 5, 3, 4, 1]


def test_size_limit(dev):
    t = torch.zeros((16385, 2), dtype=torch.float32, device=dev)
    with pytest.raises(st.StereoError):
        st.stereo_vote_matches(t, t, 4.0, 128.0)
