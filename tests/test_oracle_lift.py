"""Pins of the feature-lifting oracle (Sec. 3.3, Eq. 11-12): bilinear DINO
upsampling (Sec. 3.2) against exact values, the 1x1-convolution MLP against a
per-pixel loop, L_d in closed form, and every gradient against central finite
differences of the loss; no GPU."""
import numpy as np
import pytest

import oracle


def test_upsampling_exact_at_patch_centres_and_linear_between():
    rng = np.random.default_rng(0)
    patch, hp, wp, nh = 3, 4, 5, 2
    grid = rng.normal(size=(hp, wp, nh))
    up = oracle.dino_upsample(grid, hp * patch, wp * patch, patch)
    # pixel (patch*j + 1, patch*i + 1) is the centre of patch (i, j) for patch = 3
    for i in range(hp):
        for j in range(wp):
            assert np.allclose(up[:, patch * i + 1, patch * j + 1], grid[i, j], atol=1e-14)
    # a grid linear in (i, j) gives values linear in the pixel position inside
    # the clamped region and constant outside it
    ii, jj = np.meshgrid(np.arange(hp), np.arange(wp), indexing="ij")
    lin = np.stack([2.0 * ii - 3.0 * jj + 1.0, 0.5 * jj], axis=-1)
    up = oracle.dino_upsample(lin, hp * patch, wp * patch, patch)
    y, x = 5, 7
    u, v = (x + 0.5) / patch - 0.5, (y + 0.5) / patch - 0.5
    assert up[0, y, x] == pytest.approx(2.0 * v - 3.0 * u + 1.0, abs=1e-12)
    assert np.allclose(up[:, 0, 0], lin[0, 0]) and np.allclose(up[:, -1, -1], lin[-1, -1])
    assert np.allclose(oracle.dino_upsample(np.full((2, 3, 4), 1.5), 9, 13, 5), 1.5)


def problem(seed, nf=3, H=5, W=4, nh=6, patch=2):
    rng = np.random.default_rng(seed)
    mlp = dict(w1=rng.normal(size=(128, nf)) * 0.5, b1=rng.normal(size=128) * 0.1,
               w2=rng.normal(size=(nh, 128)) * 0.2, b2=rng.normal(size=nh) * 0.1)
    feat = rng.normal(size=(nf, H, W))
    grid = rng.normal(size=((H + patch - 1) // patch, (W + patch - 1) // patch, nh))
    return mlp, feat, grid, oracle.LiftCfg(n_h=nh, patch=patch)


def test_mlp_is_the_same_per_pixel_map():
    mlp, feat, grid, cfg = problem(1)
    nf, H, W = feat.shape
    # with patch = 1 the target of pixel (x, y) is grid[y, x]; rebuild L_d with a plain loop
    grid1 = np.random.default_rng(2).normal(size=(H, W, cfg.n_h))
    cfg1 = oracle.LiftCfg(n_h=cfg.n_h, patch=1)
    loss, _ = oracle.feature_lift(feat, grid1, mlp, cfg1, n_pix=H * W, scale=0.7)
    ref = 0.0
    for y in range(H):
        for x in range(W):
            h = np.array([max(0.0, sum(mlp["w1"][k, c] * feat[c, y, x] for c in range(nf)) + mlp["b1"][k])
                          for k in range(128)])
            fh = np.array([sum(mlp["w2"][o, k] * h[k] for k in range(128)) + mlp["b2"][o] for o in range(cfg.n_h)])
            f = grid1[y, x]
            ref += 1.0 - f @ fh / (np.linalg.norm(f) * np.linalg.norm(fh))
    assert loss == pytest.approx(0.7 * ref / (H * W), rel=1e-12)


def test_distillation_loss_closed_forms():
    mlp, feat, _, cfg = problem(3)
    nf, H, W = feat.shape
    cfg1 = oracle.LiftCfg(n_h=cfg.n_h, patch=1)
    # the rendered high-dimensional features themselves (zero target -> read back F^ via its gradient-free path)
    X = feat.reshape(nf, -1).T
    Fh = np.maximum(X @ mlp["w1"].T + mlp["b1"], 0) @ mlp["w2"].T + mlp["b2"]
    Fh = Fh.T.reshape(cfg.n_h, H, W)
    same = np.moveaxis(2.5 * Fh, 0, -1)
    loss, gr = oracle.feature_lift(feat, same, mlp, cfg1, n_pix=H * W)
    assert abs(loss) < 1e-14 and max(np.abs(v).max() for v in gr.values()) < 1e-12
    loss, _ = oracle.feature_lift(feat, -same, mlp, cfg1, n_pix=H * W, scale=3.0)
    assert loss == pytest.approx(3.0 * 2.0, rel=1e-12)
    # a zero target vector: cos read as 0, no gradient
    loss, gr = oracle.feature_lift(feat, np.zeros_like(same), mlp, cfg1, n_pix=H * W)
    assert loss == pytest.approx(1.0) and max(np.abs(v).max() for v in gr.values()) == 0.0


@pytest.mark.parametrize("seed", [4, 5])
def test_gradients_against_central_differences(seed):
    mlp, feat, grid, cfg = problem(seed)
    nf, H, W = feat.shape
    n_pix = 2 * H * W  # the view is one of two
    X = feat.reshape(nf, -1).T
    Z = X @ mlp["w1"].T + mlp["b1"]
    assert np.abs(Z).min() > 1e-4  # no ReLU kink within the step
    loss, gr = oracle.feature_lift(feat, grid, mlp, cfg, n_pix, scale=0.9)
    rng = np.random.default_rng(seed + 10)
    h = 1e-6
    params = dict(mlp, feat=feat)
    for name, arr in params.items():
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + h
            lp, _ = oracle.feature_lift(params["feat"], grid, {k: params[k] for k in mlp}, cfg, n_pix, 0.9)
            arr[idx] = old - h
            lm, _ = oracle.feature_lift(params["feat"], grid, {k: params[k] for k in mlp}, cfg, n_pix, 0.9)
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            assert gr[name][idx] == pytest.approx(fd, rel=1e-5, abs=1e-10), (name, idx)


def test_weighted_loss_gradients_against_central_differences():
    mlp, feat, grid, cfg = problem(7)
    nf, H, W = feat.shape
    w = np.random.default_rng(8).uniform(0, 1, (H, W))
    w[1, :] = 0.0
    X = feat.reshape(nf, -1).T
    assert np.abs(X @ mlp["w1"].T + mlp["b1"]).min() > 1e-5
    l1, _ = oracle.feature_lift(feat, grid, mlp, cfg, H * W, 0.5)
    l2, _ = oracle.feature_lift(feat, grid, mlp, cfg, H * W, 0.5, weight=np.ones((H, W)))
    assert l1 == pytest.approx(l2, rel=1e-14)
    _, gr = oracle.feature_lift(feat, grid, mlp, cfg, H * W, 0.5, weight=w)
    h = 1e-6
    for name, arr in [("w2", mlp["w2"]), ("feat", feat)]:
        for idx in [(0, 0), (2, 3)] if name == "w2" else [(0, 2, 1), (1, 1, 2), (2, 4, 3)]:
            old = arr[idx]
            arr[idx] = old + h
            lp = oracle.feature_lift(feat, grid, mlp, cfg, H * W, 0.5, weight=w)[0]
            arr[idx] = old - h
            lm = oracle.feature_lift(feat, grid, mlp, cfg, H * W, 0.5, weight=w)[0]
            arr[idx] = old
            assert gr[name][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-11), (name, idx)
