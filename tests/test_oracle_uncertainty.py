"""Pins of the tracking-uncertainty oracle (Sec. 3.4 "Tracking": Eq. 6 residual,
Eq. 15 per-pixel minimiser) against closed forms, a generic numerical
minimiser and scipy's box filter; no GPU."""
import numpy as np
import pytest

import oracle

RC = oracle.ResidualCfg()


def views(H=6, W=7, nf=4, seed=0):
    rng = np.random.default_rng(seed)
    img = dict(color=rng.uniform(0, 1, (3, H, W)), depth=rng.uniform(1, 3, (H, W)),
               feat=rng.normal(size=(nf, H, W)), T=np.zeros((H, W)))
    tgt = dict(color=rng.uniform(0, 1, (3, H, W)), depth=rng.uniform(1, 3, (H, W)),
               feat=rng.normal(size=(nf, H, W)))
    return img, tgt


def test_paper_weights_are_the_defaults():
    # Sec. 4 "Implementation Details": residual weights (0.25, 0.7, 0.1); Eq. 6: T~ < 0.1
    assert (RC.lambda_color, RC.lambda_depth, RC.lambda_feat, RC.t_mask) == (0.25, 0.7, 0.1, 0.1)


def test_box_filter_border_and_interior():
    d = np.zeros((5, 6))
    d[0, 0] = 9.0   # corner: 4-pixel window
    d[0, 3] = 12.0  # edge: 6-pixel window
    d[3, 3] = 18.0  # interior: 9-pixel window
    b = oracle.box3(d)
    assert b[0, 0] == pytest.approx(9.0 / 4) and b[1, 1] == pytest.approx(9.0 / 9)
    assert b[0, 3] == pytest.approx(12.0 / 6) and b[1, 3] == pytest.approx(12.0 / 9)
    assert b[2, 3] == pytest.approx(18.0 / 9) and b[2, 4] == pytest.approx(18.0 / 9)
    assert b[4, 3] == pytest.approx(18.0 / 6) and b[2, 2] == pytest.approx(18.0 / 9)
    assert np.allclose(oracle.box3(np.full((4, 4), 2.5)), 2.5)
    # interior pixels against a library box filter
    ndi = pytest.importorskip("scipy.ndimage")
    r = np.random.default_rng(1).normal(size=(9, 11))
    assert np.allclose(oracle.box3(r)[1:-1, 1:-1], ndi.uniform_filter(r, 3)[1:-1, 1:-1], atol=1e-12)


@pytest.mark.parametrize("R", [1e-4, 0.03, 0.25, 0.7, 4.0])
def test_eq15_minimiser_is_two_r(R):
    """Minimise 1/2 (R / sigma^2 + log sigma) numerically (over log sigma) and
    compare with the closed form used by the oracle."""
    opt = pytest.importorskip("scipy.optimize")
    f = lambda ls: 0.5 * (R / np.exp(2 * ls) + ls)
    res = opt.minimize_scalar(f, bracket=(-10.0, 5.0), tol=1e-12)
    img, tgt = views(1, 1, 0)
    # a pixel whose residual is exactly R: colour only, lambda_color = 1
    img["color"][:] = 0.0
    tgt["color"][:] = 0.0
    tgt["color"][0] = R
    img["depth"][:] = tgt["depth"]
    cfg = oracle.ResidualCfg(lambda_color=1.0, lambda_depth=1.0, lambda_feat=1.0)
    Rg, s2, _ = oracle.tracking_uncertainty(img, tgt, cfg, 0)
    assert Rg[0, 0] == pytest.approx(R, rel=1e-12)
    assert s2[0, 0] == pytest.approx(np.exp(2 * res.x), rel=1e-6)


def test_residual_terms_closed_forms():
    H, W, nf = 3, 4, 3
    img, tgt = views(H, W, nf, seed=2)
    img["T"][:] = 0.0
    # colour: |delta|_1 over the channels
    img["color"] = tgt["color"] + np.array([0.1, -0.2, 0.3])[:, None, None]
    # depth: rendered depth = box-filtered target depth + 0.05
    tgt["depth"] = np.full((H, W), 2.0)
    img["depth"] = np.full((H, W), 2.05)
    # features: column 0 equal, column 1 orthogonal, column 2 opposite, column 3 zero
    base = np.array([1.0, 2.0, -1.0])
    orth = np.array([2.0, -1.0, 0.0])
    tgt["feat"] = np.broadcast_to(base[:, None, None], (nf, H, W)).copy()
    img["feat"][:, :, 0] = 3.0 * base[:, None]
    img["feat"][:, :, 1] = orth[:, None]
    img["feat"][:, :, 2] = -base[:, None]
    img["feat"][:, :, 3] = 0.0
    R, s2, m = oracle.tracking_uncertainty(img, tgt, RC, nf)
    rf = np.array([0.0, 1.0, 1.0, 1.0])  # 1 - cos: 0, 1, 2 capped at 1, zero vector -> cos 0
    want = 0.25 * 0.6 + 0.7 * 0.05 + 0.1 * rf[None, :]
    assert np.allclose(R, np.broadcast_to(want, (H, W)), rtol=1e-12, atol=1e-15)
    assert np.allclose(s2, 2 * R)
    assert np.array_equal(m, (R > 0.25).astype(np.uint8))


def test_visibility_mask_and_motion_threshold():
    img, tgt = views(2, 3, 0, seed=3)
    img["T"] = np.array([[0.0, 0.0999, 0.1], [0.5, 1.0, 0.05]])
    R, _, _ = oracle.tracking_uncertainty(img, tgt, RC, 0)
    assert np.all(R[img["T"] >= 0.1] == 0.0) and np.all(R[img["T"] < 0.1] > 0.0)
    # motion: 2 sigma^2 > 1 strictly, i.e. R > 1/4
    img, tgt = views(1, 2, 0, seed=4)
    img["color"][:] = 0.0
    tgt["color"][:] = 0.0
    img["depth"][:] = 2.0  # constant: the box filter leaves it unchanged
    tgt["depth"][:] = 2.0
    tgt["color"][0, 0, 0] = 0.25
    tgt["color"][0, 0, 1] = 0.25 + 1e-9
    cfg = oracle.ResidualCfg(lambda_color=1.0)
    R, s2, m = oracle.tracking_uncertainty(img, tgt, cfg, 0)
    assert list(m[0]) == [0, 1]
