"""An independent formulation of feature lifting and L_d (Sec. 3.3, Eq. 11-12)
that never forms the n_h-wide F^_p, checked against oracle.feature_lift.

With F_p = sum_k w_k g_{c_k} (bilinear from the four patch vectors around p)
and F^_p = W2 H_p + b2:
  F^_p . F_p = H_p . e_p + sum_k w_k (b2 . g_{c_k}),  e_p = sum_k w_k W2^T g_{c_k}
  |F^_p|^2   = H_p^T (W2^T W2) H_p + 2 (W2^T b2) . H_p + |b2|^2
  |F_p|^2    = w^T Gram(g_{c_0..3}) w
and with dL/dF^_p = a_p F_p + b_p F^_p (a_p = -g/(|F||F^|), b_p = g cos/|F^|^2):
  dL/dH_p = a_p e_p + b_p (W2^T W2 H_p + W2^T b2)
  dW2 = sum_c g_c D_c^T + W2 (sum_p b_p H_p H_p^T) + b2 (sum_p b_p H_p)^T,
        D_c = sum over (p, k) with c_k = c of a_p w_k H_p
  db2 = sum_c g_c alpha_c + W2 sum_p b_p H_p + b2 sum_p b_p,  alpha_c = sum a_p w_k.
Agreement to rounding pins the oracle's loss and every gradient by a second
derivation; no GPU."""
import numpy as np
import pytest

import oracle


def corners(H, W, hp, wp, patch):
    u = np.clip((np.arange(W) + 0.5) / patch - 0.5, 0.0, wp - 1)
    v = np.clip((np.arange(H) + 0.5) / patch - 0.5, 0.0, hp - 1)
    x0, y0 = np.floor(u).astype(int), np.floor(v).astype(int)
    x1, y1 = np.minimum(x0 + 1, wp - 1), np.minimum(y0 + 1, hp - 1)
    ax, ay = u - x0, v - y0
    Y0, X0 = np.meshgrid(y0, x0, indexing="ij")
    Y1, X1 = np.meshgrid(y1, x1, indexing="ij")
    AY, AX = np.meshgrid(ay, ax, indexing="ij")
    c = np.stack([Y0 * wp + X0, Y0 * wp + X1, Y1 * wp + X0, Y1 * wp + X1], -1).reshape(-1, 4)
    w = np.stack([(1 - AX) * (1 - AY), AX * (1 - AY), (1 - AX) * AY, AX * AY], -1).reshape(-1, 4)
    return c, w


def lift_reduced(feat, grid, mlp, patch, n_pix, scale, weight):
    nf, H, W = feat.shape
    hp, wp, nh = grid.shape
    G = grid.reshape(-1, nh)
    W1, b1, W2, b2 = mlp["w1"], mlp["b1"], mlp["w2"], mlp["b2"]
    E, s = G @ W2, G @ b2
    M, u, beta = W2.T @ W2, W2.T @ b2, b2 @ b2
    c, w = corners(H, W, hp, wp, patch)
    X = feat.reshape(nf, -1).T
    Z = X @ W1.T + b1
    Hh = np.maximum(Z, 0.0)
    e = (w[:, :, None] * E[c]).sum(1)
    dot = (Hh * e).sum(1) + (w * s[c]).sum(1)
    nF2 = np.einsum("pk,pkl,pl->p", w, np.einsum("pkn,pln->pkl", G[c], G[c]), w)
    MH = Hh @ M
    nFh2 = (Hh * MH).sum(1) + 2.0 * Hh @ u + beta
    ok = (nF2 > 0) & (nFh2 > 0)
    nF, nFh = np.sqrt(np.where(ok, nF2, 1.0)), np.sqrt(np.where(ok, nFh2, 1.0))
    cos = np.where(ok, dot / (nF * nFh), 0.0)
    g = scale / n_pix * weight.reshape(-1)
    loss = (g * (1.0 - cos)).sum()
    a = np.where(ok, -g / (nF * nFh), 0.0)
    b = np.where(ok, g * cos / nFh ** 2, 0.0)
    dZ = (a[:, None] * e + b[:, None] * (MH + u)) * (Z > 0)
    D, alpha = np.zeros((G.shape[0], 128)), np.zeros(G.shape[0])
    for k in range(4):
        np.add.at(D, c[:, k], (a * w[:, k])[:, None] * Hh)
        np.add.at(alpha, c[:, k], a * w[:, k])
    Gb, hb = (b[:, None] * Hh).T @ Hh, b @ Hh
    return loss, dict(w1=dZ.T @ X, b1=dZ.sum(0), w2=G.T @ D + W2 @ Gb + np.outer(b2, hb),
                      b2=G.T @ alpha + W2 @ hb + b2 * b.sum(), feat=(dZ @ W1).T.reshape(nf, H, W))


@pytest.mark.parametrize("H,W,patch,nf,nh", [(37, 53, 14, 16, 64), (29, 30, 7, 32, 384), (14, 14, 14, 16, 32)])
def test_reduced_form_equals_oracle(H, W, patch, nf, nh):
    rng = np.random.default_rng(H * W + nh)
    hp, wp = -(-H // patch), -(-W // patch)
    mlp = dict(w1=rng.normal(size=(128, nf)) * 0.3, b1=rng.normal(size=128) * 0.1,
               w2=rng.normal(size=(nh, 128)) * 0.1, b2=rng.normal(size=nh) * 0.1)
    feat, grid = rng.normal(size=(nf, H, W)), rng.normal(size=(hp, wp, nh))
    wt = rng.uniform(0, 1, (H, W))
    wt[3, :] = 0.0
    l0, g0 = oracle.feature_lift(feat, grid, mlp, oracle.LiftCfg(n_h=nh, patch=patch), 2 * H * W, 0.7, weight=wt)
    l1, g1 = lift_reduced(feat, grid, mlp, patch, 2 * H * W, 0.7, wt)
    assert l1 == pytest.approx(l0, rel=1e-13)
    for k in g0:
        assert np.abs(g1[k] - g0[k]).max() <= 1e-12 * np.abs(g0[k]).max(), k
