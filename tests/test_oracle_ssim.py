"""Pins of the D-SSIM oracle (Eq. 4; SSIM of Wang et al.): the window, SSIM of
an image with itself, constant images in closed form, the SSIM map against a
per-pixel brute-force loop, and the gradient against central finite
differences; no GPU."""
import numpy as np
import pytest

import oracle

pytest.importorskip("scipy.ndimage")


def test_window():
    w = oracle.ssim_window()
    assert w.shape == (11, 11) and w.sum() == pytest.approx(1.0, abs=1e-15)
    assert w[5, 6] / w[5, 5] == pytest.approx(np.exp(-1.0 / 4.5), rel=1e-12)
    assert np.allclose(w, w.T) and np.allclose(w, w[::-1, ::-1])


def test_identical_images_give_zero_loss_and_gradient():
    x = np.random.default_rng(0).uniform(0, 1, (3, 14, 17))
    loss, g = oracle.ssim_loss(x, x.copy(), n_pix=14 * 17)
    assert abs(loss) < 1e-12 and np.abs(g).max() < 1e-12


def test_constant_images_closed_form_in_the_interior():
    a, b = 0.3, 0.7
    H, W = 14, 15
    x = np.full((H, W), a)
    y = np.full((H, W), b)
    # interior (window inside the image): mu = a, b and no variance, so
    # S = (2ab + C1) C2 / ((a^2 + b^2 + C1) C2)
    S = brute_ssim_map(x, y)
    closed = (2 * a * b + oracle.SSIM_C1) / (a * a + b * b + oracle.SSIM_C1)
    assert np.allclose(S[5:-5, 5:-5], closed, rtol=1e-9)
    loss, _ = oracle.ssim_loss(np.stack([x] * 3), np.stack([y] * 3), n_pix=H * W)
    assert loss == pytest.approx((1 - S).sum() / (H * W), rel=1e-10)


def brute_ssim_map(x, y):
    H, W = x.shape
    w = oracle.ssim_window()
    S = np.zeros((H, W))
    for p in range(H):
        for q in range(W):
            m = {k: 0.0 for k in ("x", "y", "xx", "yy", "xy")}
            for i in range(-5, 6):
                for j in range(-5, 6):
                    r, c = p + i, q + j
                    if 0 <= r < H and 0 <= c < W:
                        ww = w[i + 5, j + 5]
                        m["x"] += ww * x[r, c]; m["y"] += ww * y[r, c]
                        m["xx"] += ww * x[r, c] ** 2; m["yy"] += ww * y[r, c] ** 2; m["xy"] += ww * x[r, c] * y[r, c]
            A1 = 2 * m["x"] * m["y"] + oracle.SSIM_C1
            A2 = 2 * (m["xy"] - m["x"] * m["y"]) + oracle.SSIM_C2
            B1 = m["x"] ** 2 + m["y"] ** 2 + oracle.SSIM_C1
            B2 = m["xx"] - m["x"] ** 2 + m["yy"] - m["y"] ** 2 + oracle.SSIM_C2
            S[p, q] = A1 * A2 / (B1 * B2)
    return S


def test_loss_against_brute_force_loop():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (3, 9, 12))
    y = rng.uniform(0, 1, (3, 9, 12))
    loss, _ = oracle.ssim_loss(x, y, n_pix=2 * 9 * 12, scale=0.8)
    ref = sum((1 - brute_ssim_map(x[c], y[c])).sum() for c in range(3)) * 0.8 / (3 * 2 * 9 * 12)
    assert loss == pytest.approx(ref, rel=1e-12)


def test_gradient_against_central_differences():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 1, (3, 13, 12))
    y = rng.uniform(0, 1, (3, 13, 12))
    n_pix = 3 * 13 * 12
    _, g = oracle.ssim_loss(x, y, n_pix, scale=0.6)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 6, 5), (2, 12, 11), (0, 3, 10), (1, 0, 7), (2, 9, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle.ssim_loss(xp, y, n_pix, 0.6)[0] - oracle.ssim_loss(xm, y, n_pix, 0.6)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-12), idx


def test_weighted_ssim_matches_unit_weight_and_differences():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (3, 11, 12))
    y = rng.uniform(0, 1, (3, 11, 12))
    n_pix = 11 * 12
    l1, g1 = oracle.ssim_loss(x, y, n_pix, 0.5)
    l2, g2 = oracle.ssim_loss(x, y, n_pix, 0.5, weight=np.ones((11, 12)))
    assert l1 == pytest.approx(l2, rel=1e-14) and np.allclose(g1, g2, rtol=1e-14, atol=0)
    w = rng.uniform(0, 1, (11, 12))
    w[3:6, 2:9] = 0.0  # a masked block (Eq. 14's mask)
    _, g = oracle.ssim_loss(x, y, n_pix, 0.5, weight=w)
    h = 1e-6
    for idx in [(0, 4, 4), (1, 0, 0), (2, 10, 11), (0, 7, 3)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle.ssim_loss(xp, y, n_pix, 0.5, w)[0] - oracle.ssim_loss(xm, y, n_pix, 0.5, w)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-6, abs=1e-12), idx
