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

# (H, W, d_min, D, r): D = 160 runs 128 disparities at K = 4 and 32 at K = 2
SHAPES = [(120, 200, 0, 64, 4), (90, 160, 0, 32, 5), (150, 260, 2, 96, 7), (70, 110, -3, 24, 3),
          (64, 300, 0, 160, 5)]


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


@pytest.mark.parametrize("cdt,stages,smooth", [(st.COST_F16, 0, 15), (st.COST_F32, 0, 15), (st.COST_F16, 1, 15),
                                                (st.COST_F32, 1, 15), (st.COST_F16, 1, 40)])
def test_batched_equals_single_pair_path(dev, cdt, stages, smooth):
    """Every output of every pair equals the single-pair path's, for the
    per-pair K split and both forced K, in both stage modes (one launch per
    stage over all pairs, or per-pair launches on parallel streams; a
    smoothing radius beyond the tile kernels' limit falls back to per-pair
    launches)."""
    pairs = _pairs(dev)
    maxH = max(s[0] for s in SHAPES)
    maxW = max(s[1] for s in SHAPES)
    p = st.stereo_default_params(max_width=maxW, max_height=maxH, num_disp=160, cost_dtype=cdt,
                                 smooth_radius=smooth)
    hb = st.stereo_create(p, max_batch=len(pairs))
    hs = st.stereo_create(p)
    st.stereo_set_batch_stages(hb, stages)
    s = torch.cuda.Stream()
    for rows, K in ((0, 0), (8, 2), (24, 4)):
        st.stereo_set_batch_config(hb, rows, K)
        assert st.stereo_get_batch_config(hb) == dict(rows=rows, K=K, stages=stages)
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
    p = st.stereo_default_params(max_width=300, max_height=150, num_disp=160, cost_dtype=st.COST_F16)
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
    p = st.stereo_default_params(max_width=300, max_height=150, num_disp=160, cost_dtype=st.COST_F16)
    hb = st.stereo_create(p, max_batch=len(pairs))
    batch = []
    for d in pairs:
        H, W = d["left"].shape[:2]
        batch.append(dict(d, **_outs(dev, H, W)))
    s = torch.cuda.Stream()
    res = st.stereo_autotune_batched(hb, batch, stream=s)
    assert res["K"] in (0, 2, 4) and res["rows"] in (8, 12, 16, 24, 32, 48) and res["ms"] > 0
    assert res["stages"] in (0, 1)
    with torch.cuda.stream(s):
        st.stereo_match_batched(hb, batch, stream=s)
    s.synchronize()
    hb.close()
