"""The batched form: many pairs of mixed sizes, disparity ranges and windows
in one persistent cost launch (graph-replayed), against the single-pair path
on each pair (identical arithmetic, so identical results), plus the
autotuner."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2007_12623_b300 as st  # noqa: E402

SHAPES = [(120, 200, 0, 64, 4), (90, 160, 0, 32, 5), (150, 260, 2, 96, 7), (70, 110, -3, 24, 3)]


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available()
    st.lib()
    return torch.device("cuda:0")


def _pairs(dev):
    out = []
    for i, (H, W, d_min, D, r) in enumerate(SHAPES):
        Lrgb, Rrgb, gt = synth.tissue_pair(synth.seed_for(3, i), W, H, max(2, d_min + 2), d_min + 0.8 * D)
        out.append(dict(left=torch.from_numpy(Lrgb).to(dev), right=torch.from_numpy(Rrgb).to(dev),
                        d_min=d_min, num_disp=D, win_radius=r))
    return out


def _outs(dev, H, W):
    return dict(disp_wta=torch.empty((H, W), dtype=torch.int16, device=dev),
                disp_sub=torch.empty((H, W), dtype=torch.float32, device=dev),
                disp_post=torch.empty((H, W), dtype=torch.int16, device=dev),
                disp_final=torch.empty((H, W), dtype=torch.float32, device=dev))


@pytest.mark.parametrize("cdt", [st.COST_F16, st.COST_F32])
def test_batched_equals_single_pair_path(dev, cdt):
    pairs = _pairs(dev)
    maxH = max(s[0] for s in SHAPES)
    maxW = max(s[1] for s in SHAPES)
    p = st.stereo_default_params(max_width=maxW, max_height=maxH, num_disp=96, cost_dtype=cdt,
                                 smooth_radius=15)
    hb = st.stereo_create(p, max_batch=len(pairs))
    hs = st.stereo_create(p)
    s = torch.cuda.Stream()
    for rows, K in ((0, 0), (8, 2), (24, 4)):
        st.stereo_set_batch_config(hb, rows, K)
        batch = []
        for d in pairs:
            H, W = d["left"].shape[:2]
            batch.append(dict(d, **_outs(dev, H, W)))
        for rep in range(2):                       # capture, then replay
            with torch.cuda.stream(s):
                st.stereo_match_batched(hb, batch, use_graph=True, stream=s)
            s.synchronize()
        for d in batch:
            H, W = d["left"].shape[:2]
            ref = _outs(dev, H, W)
            st.stereo_match(hs, d["left"], d["right"], d_min=d["d_min"], num_disp=d["num_disp"],
                            win_radius=d["win_radius"], **ref)
            torch.cuda.synchronize()
            for k in ref:
                assert torch.equal(d[k].nan_to_num(-7), ref[k].nan_to_num(-7)), (k, rows, K)
    hb.close()
    hs.close()


def test_batched_matches_oracle_wta(dev):
    """Each pair's winner-take-all map from the batched launch against the
    oracle (near-ties exempt)."""
    pairs = _pairs(dev)
    p = st.stereo_default_params(max_width=260, max_height=150, num_disp=96, cost_dtype=st.COST_F16)
    hb = st.stereo_create(p, max_batch=len(pairs))
    batch = []
    for d in pairs:
        H, W = d["left"].shape[:2]
        batch.append(dict(d, **_outs(dev, H, W)))
    st.stereo_match_batched(hb, batch, use_graph=False)
    torch.cuda.synchronize()
    for d in batch:
        Lg, Rg = oracle.gray(d["left"].cpu().numpy()), oracle.gray(d["right"].cpu().numpy())
        m = oracle.match(Lg, Rg, d["d_min"], d["num_disp"], d["win_radius"])
        g = d["disp_wta"].cpu().numpy()
        bad = (g != m["dL"]) & ~(m["gapL"] < 1e-5)
        assert not bad.any(), np.argwhere(bad)[:5]
    hb.close()


def test_autotuner_picks_a_configuration(dev):
    pairs = _pairs(dev)
    p = st.stereo_default_params(max_width=260, max_height=150, num_disp=96, cost_dtype=st.COST_F16)
    hb = st.stereo_create(p, max_batch=len(pairs))
    batch = []
    for d in pairs:
        H, W = d["left"].shape[:2]
        batch.append(dict(d, **_outs(dev, H, W)))
    s = torch.cuda.Stream()
    res = st.stereo_autotune_batched(hb, batch, stream=s)
    assert res["K"] in (2, 4) and res["rows"] in (8, 12, 16, 24, 32, 48) and res["ms"] > 0
    with torch.cuda.stream(s):
        st.stereo_match_batched(hb, batch, stream=s)
    s.synchronize()
    hb.close()
