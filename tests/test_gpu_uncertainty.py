"""Tracking uncertainty on the GPU (Sec. 3.4 "Tracking": Eq. 6 residual R,
Eq. 15 sigma^2 = 2R, motion mask R > 1/4) against the FP64 oracle, both fed
the same seeded synthetic images and targets (a forward on the same cameras
only sets up the views).

Bar: R and sigma^2 within 1e-5 relative + 1e-6 absolute (FP32 sums of at most
3 + 9 + 3 N_l terms); the motion mask bit-exact except where the oracle's R
lies within 1e-5 of the 1/4 threshold (there the FP32 and FP64 decisions may
differ; the count is bounded)."""
import numpy as np
import pytest

import oracle
from gpu_cases import round_cams
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def synth(seed, cams, nf):
    """Per-view rendered-like images and targets, FP32-representable."""
    rng = np.random.default_rng(seed)
    out = []
    for c in cams:
        H, W = c.height, c.width
        f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
        img = dict(color=f32(rng.uniform(0, 1, (3, H, W))), depth=f32(rng.uniform(1, 3, (H, W))),
                   feat=f32(rng.normal(size=(nf, H, W))), T=f32(rng.uniform(0, 0.2, (H, W))))
        tgt = dict(color=f32(rng.uniform(0, 1, (3, H, W))), depth=f32(rng.uniform(1, 3, (H, W))),
                   feat=f32(rng.normal(size=(nf, H, W))))
        if nf:
            img["feat"][:, 0, :5] = 0.0   # zero rendered features: cos read as 0
            tgt["feat"][:, 1, :3] = 0.0
        out.append((img, tgt))
    return out


def to_device(views, nf):
    import torch
    cat = lambda k, src: torch.tensor(np.concatenate([v[src][k].reshape(-1) for v in views]),
                                      dtype=torch.float32, device="cuda")
    img = {k: cat(k, 0) for k in ("color", "depth", "T")}
    tgt = {k: cat(k, 1) for k in ("color", "depth")}
    if nf:
        img["feat"] = cat("feat", 0)
        tgt["feat"] = cat("feat", 1)
    return img, tgt


def run_case(cams, nf, seed, rcfg=oracle.ResidualCfg()):
    import torch
    cams = round_cams(cams)
    R = B.Renderer(n_feat=nf, k=1)
    g = scenes.plain_gaussians(seed, 200, nf)
    R.forward(B.to_set(g), cams)  # sets up the views of the ctx
    views = synth(seed + 1, cams, nf)
    img, tgt = to_device(views, nf)
    out = R.tracking_uncertainty(img, tgt, rcfg.lambda_color, rcfg.lambda_depth, rcfg.lambda_feat, rcfg.t_mask)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    off = 0
    n_amb = 0
    for c, (vi, vt) in zip(cams, views):
        P = c.width * c.height
        Ro, s2o, mo = oracle.tracking_uncertainty(vi, vt, rcfg, nf)
        Rg = got["R"][off:off + P].reshape(c.height, c.width).astype(np.float64)
        s2g = got["sigma2"][off:off + P].reshape(c.height, c.width).astype(np.float64)
        mg = got["motion"][off:off + P].reshape(c.height, c.width)
        assert np.allclose(Rg, Ro, rtol=1e-5, atol=1e-6), np.abs(Rg - Ro).max()
        assert np.allclose(s2g, s2o, rtol=1e-5, atol=2e-6)
        amb = np.abs(Ro - 0.25) <= 1e-5
        assert np.array_equal(mg[~amb], mo[~amb])
        assert np.all(Rg[vi["T"] >= rcfg.t_mask] == 0.0)
        n_amb += int(amb.sum())
        off += P
    return n_amb, got


def test_ragged_views_feat16():
    cams = scenes.cameras(3, 3, 64, 48, 80.0)
    cams[1] = cams[1].scaled(0.75)
    cams[2] = cams[2].scaled(0.5)
    n_amb, got = run_case(cams, 16, 5)
    assert n_amb <= 3
    m = got["motion"]
    assert 0 < m.sum() < m.size  # both classes occur


@pytest.mark.parametrize("nf", [0, 32])
def test_feature_widths(nf):
    cams = scenes.cameras(4, 2, 40, 30, 50.0)
    n_amb, _ = run_case(cams, nf, 7)
    assert n_amb <= 3


def test_other_weights_and_mask():
    cams = scenes.cameras(5, 1, 33, 17, 40.0)  # ragged: neither side a multiple of the block
    n_amb, _ = run_case(cams, 16, 9, oracle.ResidualCfg(1.0, 0.5, 2.0, 0.15))
    assert n_amb <= 3


def test_mapping_batch_full_size():
    """8 views of 640x480 (the bench batch): every pixel against the oracle."""
    cams = scenes.cameras(0, 8, 640, 480, 600.0)
    n_amb, got = run_case(cams, 16, 11)
    assert n_amb <= 50
    assert got["R"].shape[0] == 8 * 640 * 480
