"""Parity at full benchmark sizes, on outputs the oracle can compute: one view of
the batched launch (views are independent in the forward and in the blending
backward), plus invariants that hold at any size.

* mapping batch: 100k anchors x K=10 (1M Gaussians), 8 keyframes 640x480, 16
  feature channels, weighted L1, FP32 decode — the launch the benchmark times;
* large scene: 300k anchors x K=10 (3M Gaussians), 32 feature channels, 16 views
  at 1280x720 in one launch, BF16 tensor-core decode: the render of the decoded
  set is compared with the oracle rendering the SAME decoded Gaussians (so the
  FP32 render bar applies), the decode itself against the stated BF16 errors.
"""
import numpy as np
import pytest

import oracle
from gpu_cases import (CFG, MARGIN, PIX_ATOL, PIX_RTOL, assert_pixels, feat_magnitude, last_blended_ids, rel_l2, tie_explained,
                       round_cams, round_dict, split_images)
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _run(A, K, nf, V, W, H, fx, bf16, seed=0):
    import torch
    anc = round_dict(scenes.anchors(seed, A, K))
    mlp = round_dict(scenes.mlp_weights(seed + 1000, K, nf))
    cams = round_cams(scenes.cameras(seed, V, W, H, fx))
    tg = [round_dict(t) for t in scenes.targets(seed + 1, cams, nf, weighted=True)]
    R = B.Renderer(n_feat=nf, k=K, decode_bf16=int(bf16))
    ad, md = B.anchors_to_device(anc, mlp)
    g = R.decode(ad, md, cams)
    img = R.forward(g, cams)
    loss, dimg = R.loss(img, B.targets_to_device(tg))
    grad, d_pose = R.backward(dimg, B.GRAD_POSE | B.GRAD_GAUSS)
    torch.cuda.synchronize()
    return dict(R=R, anc=anc, mlp=mlp, cams=cams, tg=tg, g=g, img=img, loss=loss.item(),
                dimg=dimg, stats=R.stats())


def _view_set(g, v, nf):
    """Decoded Gaussians of view v as float64 numpy (the oracle's input)."""
    mo = g.mean_opacity[v].cpu().numpy().astype(np.float64)
    return dict(mean=mo[:, :3], opacity=mo[:, 3], scale=g.scale[v].cpu().numpy().astype(np.float64)[:, :3],
                quat=g.quat[v].cpu().numpy().astype(np.float64), color=g.color[v].cpu().numpy().astype(np.float64)[:, :3],
                feat=g.feat[v].cpu().numpy().astype(np.float64) if nf else np.zeros((mo.shape[0], 0)))


def _invariants(views):
    for v in views:
        assert np.all(v["T"] >= 0) and np.all(v["T"] <= 1)
        s = v["color"].max(axis=0)
        assert np.all(v["color"] >= 0) and np.all(v["color"] <= 1 - v["T"] + 1e-5)
        assert np.all(v["depth"] >= 0)
        assert np.all(np.isfinite(v["feat"]))


def _check_view0(res, nf, grads):
    cam = res["cams"][0]
    gview = _view_set(res["g"], 0, nf)
    pr = oracle.project(gview, cam, CFG)
    ref = oracle.render(pr, gview, cam, CFG, nf)
    gpu_views = split_images(res["img"], res["cams"], nf)
    _invariants(gpu_views)
    mag = [feat_magnitude(pr, gview, cam, nf)]
    glist = res["R"].copy_buffer(0)
    grng = res["R"].copy_buffer(2).reshape(-1, 2)
    lst, rng = oracle.tile_lists(pr, cam, CFG)
    ids = [(last_blended_ids(gpu_views[0]["n_contrib"], glist, grng, 0, 0),
            last_blended_ids(ref["n_contrib"], lst, rng))]
    tie = [tie_explained(gpu_views[0]["n_contrib"], ref["n_contrib"], lst, rng, pr["pcam"][:, 2])]
    assert_pixels(gpu_views[:1], [ref], nf, feat_mag=mag, last_ids=ids, tie_ok=tie)
    if not grads:
        return
    # 2D gradient records of view 0 against the oracle blending backward fed
    # with the same image gradients (normalised by all views' pixels)
    P = cam.width * cam.height
    d = {k: res["dimg"][k].cpu().numpy().astype(np.float64) for k in ("color", "depth", "feat")}
    gi = dict(color=d["color"][:3 * P].reshape(3, cam.height, cam.width),
              depth=d["depth"][:P].reshape(cam.height, cam.width),
              feat=d["feat"][:nf * P].reshape(nf, cam.height, cam.width))
    g2 = oracle.render_bwd(pr, gview, cam, CFG, nf, gi)
    N = gview["mean"].shape[0]
    rec = res["R"].copy_buffer(6).reshape(-1, 12 + nf)[:N].astype(np.float64)
    for name, a, r in (("uv", rec[:, 0:2], g2["uv"]), ("z", rec[:, 2], g2["z"]), ("opacity", rec[:, 3], g2["opacity"]),
                       ("conic", rec[:, 4:7], g2["conic"]), ("color", rec[:, 8:11], g2["color"]),
                       ("feat", rec[:, 12:], g2["feat"])):
        e = rel_l2(a, r)
        assert e < 2e-3, (name, e)


def test_mapping_batch_full_size_view0():
    res = _run(100_000, 10, 16, 8, 640, 480, 600.0, bf16=False)
    st = res["stats"]
    assert st["n_gaussian_views"] == 8_000_000 and st["n_tiles"] == 8 * 1200
    assert st["n_instances"] > 1e7
    # decode of view 0 against the oracle (FP32 bar)
    ref = oracle.decode(res["anc"], res["mlp"], res["cams"][0], 10, 16)
    gview = _view_set(res["g"], 0, 16)
    for k, tol in (("mean", 1e-6), ("opacity", 1e-5), ("color", 1e-5)):
        np.testing.assert_allclose(gview[k], ref[k], atol=tol, rtol=1e-5)
    np.testing.assert_allclose(gview["feat"], ref["feat"], atol=1e-5, rtol=1e-5)
    _check_view0(res, 16, grads=True)


def test_large_scene_bf16_16_views_1280x720_view0():
    res = _run(300_000, 10, 32, 16, 1280, 720, 1200.0, bf16=True)
    st = res["stats"]
    assert st["n_gaussian_views"] == 16 * 3_000_000 and st["n_tiles"] == 16 * 3600
    assert st["key_bits"] == 16
    # BF16 decode of view 0 within the stated per-output errors
    ref = oracle.decode(res["anc"], res["mlp"], res["cams"][0], 10, 32)
    gview = _view_set(res["g"], 0, 32)
    assert np.abs(gview["opacity"] - ref["opacity"]).max() < 1e-2
    assert np.abs(gview["color"] - ref["color"]).max() < 1e-2
    assert np.sqrt(np.mean((gview["feat"] - ref["feat"]) ** 2)) < 1e-2
    _check_view0(res, 32, grads=False)
