"""Uncertainty MLP F_u and L_u on the GPU (Sec. 3.3, Eq. 5, Eq. 13) against the
FP64 oracle, both fed the same seeded DINO patch grids, residual maps and
weights (a forward on the same cameras only sets up the views).  The GPU
evaluates the first layer once per patch and interpolates it (exact by
linearity); the oracle upsamples the features per pixel.

FP32 arithmetic throughout (the library's own FP32 GEMM on the patches).
sigma: the first layer sums n_h products and the second 128 in FP32 (the GPU
interpolates W1 g per patch, the oracle interpolates F first: the same sum in
another order), n u ~ 384 x 6e-8 ~ 2.3e-5 relative on the pre-activations at
worst: bar 5e-5 relative + 1e-6; the loss within 1e-5 relative and the
gradients within 1e-4 relative L2 (means over all pixels); the motion mask
bit-exact outside a 1e-4 band around 2 sigma^2 = 1."""
import numpy as np
import pytest

import oracle
from gpu_cases import rel_l2, round_cams
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def run_case(cams, nh, patch, seed, lam=1.0, scale=0.3):
    import torch
    cams = round_cams(cams)
    rng = np.random.default_rng(seed)
    R = B.Renderer(n_feat=0, k=1)
    R.forward(B.to_set(scenes.plain_gaussians(seed, 50, 0)), cams)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    mlp = dict(w1=f32(rng.normal(size=(128, nh)) * 0.2), b1=f32(rng.normal(size=128) * 0.1),
               w2=f32(rng.normal(size=128) * 0.2), b2=f32(np.array([0.2])))
    grids = [f32(rng.normal(size=(-(-c.height // patch), -(-c.width // patch), nh))) for c in cams]
    res = [f32(rng.uniform(0, 1.5, (c.height, c.width))) for c in cams]
    dev = lambda arrs: torch.tensor(np.concatenate([a.reshape(-1) for a in arrs]), dtype=torch.float32,
                                    device="cuda")
    dm = {k: torch.zeros(v.shape, dtype=torch.float32, device="cuda") for k, v in mlp.items()}
    loss, out = R.uncertainty_mlp(dev(grids), dev(res), {k: dev([v]) for k, v in mlp.items()}, n_h=nh,
                                  patch=patch, lam=lam, scale=scale, d_mlp=dm)
    torch.cuda.synchronize()
    n_pix = sum(c.width * c.height for c in cams)
    ref_loss, ref = 0.0, {k: np.zeros_like(v) for k, v in mlp.items()}
    sig, mot = [], []
    for gr, r in zip(grids, res):
        l, g, s, m = oracle.uncertainty_mlp(gr, r, mlp, oracle.LiftCfg(n_h=nh, patch=patch), n_pix, lam, scale)
        ref_loss += l
        for k in ref:
            ref[k] += g[k]
        sig.append(s.reshape(-1))
        mot.append(m.reshape(-1))
    sig, mot = np.concatenate(sig), np.concatenate(mot)
    gs = out["sigma"].cpu().numpy().astype(np.float64)
    gm = out["motion"].cpu().numpy()
    print(f"unc mlp nh={nh} sigma max rel {np.max(np.abs(gs - sig) / sig):.2e}")
    assert np.allclose(gs, sig, rtol=5e-5, atol=1e-6), np.abs(gs - sig).max()
    amb = np.abs(2 * sig * sig - 1) <= 1e-4
    assert np.array_equal(gm[~amb], mot[~amb]) and amb.sum() <= max(3, 1e-4 * amb.size)
    le = abs(float(loss.item()) - ref_loss) / abs(ref_loss)
    errs = {k: rel_l2(dm[k].cpu().numpy().astype(np.float64), ref[k]) for k in ref}
    print(f"unc mlp nh={nh} loss rel {le:.2e}", {k: f"{v:.2e}" for k, v in errs.items()})
    assert le < 1e-5, (float(loss.item()), ref_loss)
    assert all(v < 1e-4 for v in errs.values()), errs


def test_ragged_views():
    cams = scenes.cameras(3, 2, 45, 31, 50.0)
    cams[1] = cams[1].scaled(0.6)
    run_case(cams, 64, 14, 5)


def test_odd_patch_and_lambda():
    run_case(scenes.cameras(4, 1, 33, 20, 40.0), 32, 5, 6, lam=0.4)


def test_full_view_640x480():
    run_case(scenes.cameras(0, 1, 640, 480, 600.0, identity=True), 384, 14, 7)
