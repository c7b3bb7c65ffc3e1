"""Pins of the uncertainty-MLP oracle (Sec. 3.3, Eq. 5, Eq. 13): sigma in closed
form, Eq. 5's stationary point sigma^2 = R / lambda, the motion mask threshold,
and every gradient against central finite differences; no GPU."""
import numpy as np
import pytest

import oracle


def problem(seed, H=6, W=5, nh=8, patch=2):
    rng = np.random.default_rng(seed)
    mlp = dict(w1=rng.normal(size=(128, nh)) * 0.3, b1=rng.normal(size=128) * 0.1,
               w2=rng.normal(size=128) * 0.2, b2=np.array([0.3]))
    grid = rng.normal(size=((H + patch - 1) // patch, (W + patch - 1) // patch, nh))
    R = rng.uniform(0.0, 2.0, (H, W))
    return mlp, grid, R, oracle.LiftCfg(n_h=nh, patch=patch)


def test_sigma_closed_form_and_mask():
    mlp, grid, R, cfg = problem(0)
    mlp["w2"][:] = 0.0  # sigma = softplus(b2) everywhere
    for b2, want_mask in ((-1.0, 0), (1.2, 1)):  # 2 softplus(b2)^2 = 0.196 and 4.27
        mlp["b2"][0] = b2
        _, _, sigma, m = oracle.uncertainty_mlp(grid, R, mlp, cfg, n_pix=R.size)
        s = np.log1p(np.exp(b2))
        assert np.allclose(sigma, s, rtol=1e-14)
        assert np.all(m == (1 if 2 * s * s > 1 else 0)) and np.all(m == want_mask)


def test_eq5_stationary_point_in_b2():
    """With sigma = softplus(b2) and uniform R, dL/db2 vanishes exactly where
    sigma^2 = R / lambda (the minimiser of R / (2 sigma^2) + lambda log sigma)."""
    mlp, grid, R, cfg = problem(1)
    mlp["w2"][:] = 0.0
    R[:] = 0.8
    lam = 0.5
    s_star = np.sqrt(0.8 / lam)
    b_star = np.log(np.expm1(s_star))
    for b2, sign in ((b_star, 0), (b_star - 0.3, -1), (b_star + 0.3, 1)):
        mlp["b2"][0] = b2
        _, gr, _, _ = oracle.uncertainty_mlp(grid, R, mlp, cfg, n_pix=R.size, lam=lam)
        if sign == 0:
            assert abs(gr["b2"][0]) < 1e-12
        else:
            assert np.sign(gr["b2"][0]) == sign


@pytest.mark.parametrize("seed", [2, 3])
def test_gradients_against_central_differences(seed):
    mlp, grid, R, cfg = problem(seed)
    F = oracle.dino_upsample(grid, *R.shape, cfg.patch).reshape(cfg.n_h, -1).T
    Z = F @ mlp["w1"].T + mlp["b1"]
    assert np.abs(Z).min() > 1e-5  # no ReLU kink within the step (a 1e-6 step moves Z by < 4e-6)
    n_pix, lam, scale = 3 * R.size, 0.7, 1.3
    _, gr, _, _ = oracle.uncertainty_mlp(grid, R, mlp, cfg, n_pix, lam, scale)
    rng = np.random.default_rng(seed + 5)
    h = 1e-6
    for name, arr in mlp.items():
        for _ in range(5):
            idx = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[idx]
            arr[idx] = old + h
            lp = oracle.uncertainty_mlp(grid, R, mlp, cfg, n_pix, lam, scale)[0]
            arr[idx] = old - h
            lm = oracle.uncertainty_mlp(grid, R, mlp, cfg, n_pix, lam, scale)[0]
            arr[idx] = old
            assert gr[name][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-11), (name, idx)
