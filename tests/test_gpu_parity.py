"""CUDA path vs the FP64 oracle, element by element, on seeded inputs.

Bars: tile lists and sort order bit-exact; forward pixels within 1e-5 absolute
+ 1e-4 relative (pixels with a visited pair within 1e-4 relative of the
alpha_min / alpha_max / t_min thresholds are counted, not compared); gradients
within 2e-3 relative L2 (atomic accumulation order is not deterministic).
"""
import numpy as np
import pytest

import oracle
from gpu_cases import (CFG, assert_grad, assert_pixels, blend_ids, check_plain, feat_magnitude, gauss_grads,
                       plain_case,
                       r32, rel_l2, round_cams, round_dict, split_images)
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()


# ---------------------------------------------------------------------------
# plain 3DGS (2,000 Gaussians, 160x120, identity pose, RGB + depth, L1)
# ---------------------------------------------------------------------------

def test_plain_2k_forward_backward():
    g, cams = scenes.workload_plain_2k(0)
    res = plain_case(0, 2000, cams, 0, weighted=False, g=g)
    check_plain(res, 0)


def _box_min_q(conic, du0, du1, dv0, dv1):
    """Minimum of a dx^2 + 2 b dx dy + c dy^2 over the boxes [du0, du1] x [dv0, dv1]
    (arrays), by dense evaluation on a 1/16-pixel grid plus the vertex rule on each
    edge; used only to decide which decisions are too close to call."""
    a, b, c = conic
    best = np.where((du0 <= 0) & (du1 >= 0) & (dv0 <= 0) & (dv1 >= 0), 0.0, np.inf)
    for dx_fixed in (du0, du1):
        dy = np.clip(-b * dx_fixed / c, dv0, dv1)
        best = np.minimum(best, a * dx_fixed ** 2 + 2 * b * dx_fixed * dy + c * dy ** 2)
    for dy_fixed in (dv0, dv1):
        dx = np.clip(-b * dy_fixed / a, du0, du1)
        best = np.minimum(best, a * dx ** 2 + 2 * b * dx * dy_fixed + c * dy_fixed ** 2)
    return best


def _ambiguous(proj, cam, eps=1e-3, rel=1e-3):
    """Gaussians whose tile membership is decided within eps px of a tile/image
    edge (the rect), or whose ellipse passes within `rel` (relative, in q) of a
    rect tile's box of pixel centres (the FP32 path tests with a small margin)."""
    ext = proj["extent"]
    amb = np.zeros(len(ext), bool)
    for lo, hi, lim in ((ext[:, 0], ext[:, 2], cam.width - 1), (ext[:, 1], ext[:, 3], cam.height - 1)):
        for e in (lo, hi):
            m = np.abs(e - np.round(e / 16) * 16) < eps
            m |= np.abs(e) < eps
            m |= np.abs(e - lim) < eps
            amb |= m
    for g in np.nonzero(proj["valid"] == 1)[0]:
        x0, y0, x1, y1 = proj["rect"][g]
        if x0 > x1 or y0 > y1:
            continue
        k2 = 2 * np.log(proj["opacity"][g] * 255)
        tx, ty = np.meshgrid(np.arange(x0, x1 + 1), np.arange(y0, y1 + 1))
        bx0, by0 = 16.0 * tx, 16.0 * ty
        bx1 = np.minimum(bx0 + 15, cam.width - 1)
        by1 = np.minimum(by0 + 15, cam.height - 1)
        u, v = proj["uv"][g]
        q_in = _box_min_q(proj["conic"][g], bx0 - u, bx1 - u, by0 - v, by1 - v)
        q_out = _box_min_q(proj["conic"][g], bx0 - u - 0.01, bx1 - u + 0.01, by0 - v - 0.01, by1 - v + 0.01)
        if np.any((q_in > k2 * (1 - rel)) & (q_out <= k2 * (1 + rel))):
            amb[g] = True
    return amb & (proj["valid"] == 1)


def test_plain_2k_tile_lists_and_sort_bit_exact():
    g, cams = scenes.workload_plain_2k(0)
    res = plain_case(0, 2000, cams, 0, weighted=False, g=g, list_cap=-1)  # whole lists
    R, cam = res["R"], res["cams"][0]
    gv = R.copy_buffer(0)
    keys = R.copy_buffer(1)
    ranges = R.copy_buffer(2).reshape(-1, 2)
    xyzo = R.copy_buffer(3).reshape(-1, 4)
    rect = R.copy_buffer(5).reshape(-1, 2)
    # (i) the sort stage: the GPU's instances are in (tile, float32 z, id) order,
    # each (tile, Gaussian) at most once, and the ranges delimit the tiles
    z = np.float32(xyzo[gv, 2]).view(np.uint32)
    order = np.lexsort((gv, z, keys))
    assert np.array_equal(order, np.arange(len(gv)))
    pair = keys.astype(np.int64) * (1 << 32) + gv
    assert len(np.unique(pair)) == len(pair)
    counts = np.bincount(keys, minlength=len(ranges))
    assert np.array_equal(ranges[:, 1] - ranges[:, 0], counts)
    nz = counts > 0
    assert np.array_equal(ranges[nz, 0], np.concatenate([[0], np.cumsum(counts)[:-1]])[nz])
    # every instance lies in its Gaussian's rect
    x0, y0 = rect[gv, 0] & 0xffff, rect[gv, 0] >> 16
    x1, y1 = rect[gv, 1] & 0xffff, rect[gv, 1] >> 16
    tiles_x = (cam.width + 15) // 16
    assert np.all((keys % tiles_x >= x0) & (keys % tiles_x <= x1) & (keys // tiles_x >= y0) & (keys // tiles_x <= y1))
    # (ii) tile lists against the oracle's own projection and stable sort
    pr = res["views"][0]["proj"]
    lst, orng = oracle.tile_lists(pr, cam, CFG)
    amb = _ambiguous(pr, cam)
    n_diff = 0
    for t in range(len(ranges)):
        a = gv[ranges[t, 0]:ranges[t, 1]]
        b = lst[orng[t, 0]:orng[t, 1]]
        a = a[~amb[a]]
        b = b[~amb[b]]
        if not np.array_equal(a, b):
            n_diff += 1
    assert n_diff == 0
    assert amb.sum() <= 20  # 1% of the scene


def test_multiview_ragged_feat16_weighted_l2():
    """Three views of different (ragged) sizes, 16 feature channels, uncertainty weights."""
    base = scenes.cameras(7, 3, 100, 70, 90.0)
    cams = [base[0], base[1].scaled(0.5), scenes.Camera(40.0, 40.0, 16.5, 8.5, 33, 17, base[2].T_cw)]
    res = plain_case(11, 3000, cams, 16, weighted=True, l2=True, lambda_scale=0.01)
    check_plain(res, 16)


def test_feat32_large_footprints():
    cams = scenes.cameras(3, 2, 96, 64, 60.0)
    g = scenes.plain_gaussians(5, 800, 32, scale_lo=0.02, scale_hi=0.15)
    res = plain_case(5, 800, cams, 32, weighted=True, g=g)
    check_plain(res, 32)


def test_empty_and_offscreen_scene():
    cams = scenes.cameras(0, 1, 48, 40, 50.0, identity=True)
    g = scenes.plain_gaussians(1, 50, 16)
    g["mean"][:, 2] = -1.0  # behind the camera: everything culled
    res = plain_case(1, 50, cams, 16, weighted=False, g=g)
    v = split_images(res["img"], res["cams"], 16)[0]
    assert np.all(v["color"] == 0) and np.all(v["T"] == 1) and np.all(v["n_contrib"] == 0)
    gg = gauss_grads(res["grad"], 16, 1)
    assert all(np.all(gg[k] == 0) for k in ("mean", "scale", "quat", "opacity", "color"))
    assert np.all(res["d_pose"] == 0)
    assert res["R"].stats()["n_instances"] == 0


def test_single_gaussian_peak_alpha():
    cams = scenes.cameras(0, 1, 64, 48, 100.0, identity=True)
    g = dict(mean=np.array([[0.0, 0.0, 2.0]]), scale=np.full((1, 3), 0.05),
             quat=np.array([[1.0, 0, 0, 0]]), opacity=np.array([0.8]),
             color=np.array([[1.0, 0.5, 0.25]]), feat=np.zeros((1, 16)))
    res = plain_case(2, 1, cams, 16, weighted=False, g=g)
    v = split_images(res["img"], res["cams"], 16)[0]
    assert abs(v["color"][0, 24, 32] - 0.8) < 1e-6
    assert abs(v["T"][24, 32] - 0.2) < 1e-6
    check_plain(res, 16)


# ---------------------------------------------------------------------------
# anchor decode + render (Eq. 8-9), FP32 decode
# ---------------------------------------------------------------------------

def anchor_case(seed, A, K, nf, cams, weighted=True, lambda_scale=0.01, mask=B.GRAD_ALL, opacity_tanh=False,
                bias_sigma=0.05, bf16=False):
    import torch
    anc = round_dict(scenes.anchors(seed, A, K))
    mlp = round_dict(scenes.mlp_weights(seed + 1, K, nf, bias_sigma=bias_sigma))
    cams = round_cams(cams)
    tg = [round_dict(t) for t in scenes.targets(seed + 2, cams, nf, weighted=weighted)]
    R = B.Renderer(n_feat=nf, k=K, opacity_tanh=int(opacity_tanh), decode_bf16=int(bf16))
    ad, md = B.anchors_to_device(anc, mlp)
    g = R.decode(ad, md, cams)
    img = R.forward(g, cams)
    loss, dimg = R.loss(img, B.targets_to_device(tg), lambda_scale=lambda_scale, g=g)
    V, N = len(cams), A * K
    grad, d_pose = R.backward(dimg, B.GRAD_ALL, scale_grad=lambda_scale / (3.0 * V * N))
    d_mlp = {k: torch.zeros_like(v) for k, v in md.items()}
    d_anc = {k: torch.zeros_like(v) for k, v in ad.items()}
    R.decode_backward(ad, md, cams, grad, mask, d_mlp, d_anc, d_pose)
    torch.cuda.synchronize()
    lc = oracle.LossCfg(lambda_scale=lambda_scale)
    L, ref, views, per_view = oracle.backward_anchor(anc, mlp, cams, tg, CFG, lc, K, nf, opacity_tanh=opacity_tanh)
    return dict(R=R, anc=anc, mlp=mlp, cams=cams, g=g, img=img, loss=float(loss.item()), L=L,
                ref=ref, views=views, per_view=per_view, grad=grad,
                d_pose=d_pose.cpu().numpy().astype(np.float64),
                d_mlp={k: v.cpu().numpy().astype(np.float64) for k, v in d_mlp.items()},
                d_anc={k: v.cpu().numpy().astype(np.float64) for k, v in d_anc.items()})


def check_anchor(res, nf):
    V = len(res["cams"])
    # decode outputs per view
    mo = res["g"].mean_opacity.cpu().numpy().astype(np.float64)
    sc = res["g"].scale.cpu().numpy().astype(np.float64)
    qt = res["g"].quat.cpu().numpy().astype(np.float64)
    co = res["g"].color.cpu().numpy().astype(np.float64)
    fe = res["g"].feat.cpu().numpy().astype(np.float64)
    for v in range(V):
        rg = res["views"][v]["g"]
        np.testing.assert_allclose(mo[v, :, :3], rg["mean"], atol=1e-6, rtol=1e-6)
        np.testing.assert_allclose(mo[v, :, 3], rg["opacity"], atol=2e-6, rtol=1e-5)
        np.testing.assert_allclose(sc[v, :, :3], rg["scale"], atol=1e-7, rtol=1e-5)
        np.testing.assert_allclose(qt[v], rg["quat"], atol=1e-5, rtol=1e-5)
        np.testing.assert_allclose(co[v, :, :3], rg["color"], atol=2e-6, rtol=1e-5)
        if nf:
            np.testing.assert_allclose(fe[v], rg["feat"], atol=1e-5, rtol=1e-5)
    gpu_views = split_images(res["img"], res["cams"], nf)
    mag = [feat_magnitude(v["proj"], v["g"], c, nf) for v, c in zip(res["views"], res["cams"])]
    assert_pixels(gpu_views, [v["img"] for v in res["views"]], nf, feat_mag=mag,
                  last_ids=blend_ids(res, gpu_views))
    assert abs(res["loss"] - res["L"]) <= 1e-5 + 1e-4 * abs(res["L"]), (res["loss"], res["L"])
    # per-view decoded-Gaussian gradients
    gg = gauss_grads(res["grad"], nf, V)
    for k in ("mean", "scale", "quat", "opacity", "color") + (("feat",) if nf else ()):
        ref = np.stack([pv["g3d"][k] for pv in res["per_view"]])
        assert_grad(k, gg[k], ref)
    for k in ("w1", "b1", "w2", "b2"):
        assert_grad(k, res["d_mlp"][k], res["ref"][k])
    for k in ("pos", "feat", "offsets", "scaling"):
        assert_grad("anchor_" + k, res["d_anc"][k], res["ref"][k])
    assert_grad("pose", res["d_pose"], res["ref"]["pose"])


def test_anchor_decode_render_small():
    cams = scenes.cameras(21, 2, 160, 120, 150.0)
    res = anchor_case(21, 600, 10, 16, cams)
    check_anchor(res, 16)


def test_anchor_decode_render_tanh_opacity():
    """The tanh opacity decode: Gaussians with o <= 0 (about half here) are culled
    by the projection on both sides; images, loss and every gradient as above."""
    cams = scenes.cameras(23, 2, 160, 120, 150.0)
    res = anchor_case(23, 600, 10, 16, cams, opacity_tanh=True, bias_sigma=0.5)
    o = res["g"].mean_opacity.cpu().numpy()[..., 3]
    assert (o <= 0).mean() > 0.2 and (o > 0.1).mean() > 0.1
    check_anchor(res, 16)


def test_anchor_decode_10k_anchors_640x480():
    """10k anchors x K=10 (100k Gaussians), 16-ch features, 640x480, full backward."""
    cams = scenes.cameras(0, 1, 640, 480, 600.0)
    res = anchor_case(0, 10000, 10, 16, cams)
    check_anchor(res, 16)


def test_anchor_decode_10k_anchors_640x480_bf16():
    """The same decode + render case with the BF16 tensor-core decode (FP32
    accumulation; projection, blending and every gradient FP32): pixels against
    the oracle's render of the GPU-decoded Gaussians (FP32 bar), and the loss and
    every gradient group against the FP64 oracle run from the seeded inputs within
    the stated BF16 bound (5e-2 relative L2; 1e-2 relative for the loss)."""
    cams = scenes.cameras(0, 1, 640, 480, 600.0)
    res = anchor_case(0, 10000, 10, 16, cams, bf16=True)
    nf = 16
    cam = res["cams"][0]
    mo = res["g"].mean_opacity[0].cpu().numpy().astype(np.float64)
    gview = dict(mean=mo[:, :3], opacity=mo[:, 3],
                 scale=res["g"].scale[0].cpu().numpy().astype(np.float64)[:, :3],
                 quat=res["g"].quat[0].cpu().numpy().astype(np.float64),
                 color=res["g"].color[0].cpu().numpy().astype(np.float64)[:, :3],
                 feat=res["g"].feat[0].cpu().numpy().astype(np.float64))
    pr = oracle.project(gview, cam, CFG)
    ref_img = oracle.render(pr, gview, cam, CFG, nf)
    gpu_views = split_images(res["img"], res["cams"], nf)
    lst, rng = oracle.tile_lists(pr, cam, CFG)
    from gpu_cases import last_blended_ids, tie_explained_groups, tie_groups, z_error_bound
    glist = res["R"].copy_buffer(0)
    grng = res["R"].copy_buffer(2).reshape(-1, 2)
    ids = [(last_blended_ids(gpu_views[0]["n_contrib"], glist, grng, 0, 0),
            last_blended_ids(ref_img["n_contrib"], lst, rng))]
    # the last blended Gaussian may differ only behind a depth-tie group (FP32 depth bound)
    grp = tie_groups(lst, rng, pr["pcam"][:, 2], z_error_bound(gview["mean"], cam.T_cw))
    tie = [tie_explained_groups(gpu_views[0]["n_contrib"], ref_img["n_contrib"], lst, rng, grp)]
    assert_pixels(gpu_views, [ref_img], nf, feat_mag=[feat_magnitude(pr, gview, cam, nf)], last_ids=ids,
                  tie_ok=tie)
    assert abs(res["loss"] - res["L"]) <= 1e-2 * abs(res["L"]), (res["loss"], res["L"])
    errs = {}
    gg = gauss_grads(res["grad"], nf, 1)
    for k in ("mean", "scale", "quat", "opacity", "color", "feat"):
        ref = np.stack([pv["g3d"][k] for pv in res["per_view"]])
        errs["g3d_" + k] = rel_l2(gg[k], ref)
    for k in ("w1", "b1", "w2", "b2"):
        errs["mlp_" + k] = rel_l2(res["d_mlp"][k], res["ref"][k])
    for k in ("pos", "feat", "offsets", "scaling"):
        errs["anchor_" + k] = rel_l2(res["d_anc"][k], res["ref"][k])
    errs["pose"] = rel_l2(res["d_pose"], res["ref"]["pose"])
    print("bf16 decode, 10k anchors x 10, 640x480: gradient rel L2 vs FP64 oracle", errs)
    assert all(e < 5e-2 for e in errs.values()), errs


# ---------------------------------------------------------------------------
# BF16 tensor-core decode: error against the FP64 oracle, stated per output
# ---------------------------------------------------------------------------

# max over all outputs, and rms; the quaternion direction is ill-conditioned
# where the raw decoded quaternion is short, hence its larger maximum
BF16_BOUNDS = dict(opacity=(1e-2, 2e-3), scale_rel=(4e-2, 6e-3), quat_dir=(0.3, 1e-2),
                   color=(1e-2, 2e-3), feat=(5e-2, 1e-2))


def test_bf16_decode_error_per_output():
    import json
    import os
    K, nf = 10, 16
    anc = round_dict(scenes.anchors(5, 10000, K))
    mlp = round_dict(scenes.mlp_weights(6, K, nf, bias_sigma=0.05))
    cams = round_cams(scenes.cameras(5, 2, 640, 480, 600.0))
    R = B.Renderer(n_feat=nf, k=K, decode_bf16=1)
    ad, md = B.anchors_to_device(anc, mlp)
    g = R.decode(ad, md, cams)
    mo = g.mean_opacity.cpu().numpy().astype(np.float64)
    sc = g.scale.cpu().numpy().astype(np.float64)
    qt = g.quat.cpu().numpy().astype(np.float64)
    co = g.color.cpu().numpy().astype(np.float64)
    fe = g.feat.cpu().numpy().astype(np.float64)
    stats = {}
    for v, c in enumerate(cams):
        ref = oracle.decode(anc, mlp, c, K, nf)
        qa = qt[v] / np.linalg.norm(qt[v], axis=1, keepdims=True)
        qr = ref["quat"] / np.linalg.norm(ref["quat"], axis=1, keepdims=True)
        qdir = np.minimum(np.linalg.norm(qa - qr, axis=1), np.linalg.norm(qa + qr, axis=1))
        errs = dict(opacity=np.abs(mo[v, :, 3] - ref["opacity"]),
                    scale_rel=np.abs(sc[v, :, :3] - ref["scale"]) / ref["scale"],
                    quat_dir=qdir, color=np.abs(co[v, :, :3] - ref["color"]),
                    feat=np.abs(fe[v] - ref["feat"]))
        np.testing.assert_allclose(mo[v, :, :3], ref["mean"], rtol=1e-6, atol=1e-6)
        for k, e in errs.items():
            st = stats.setdefault(k, dict(max=0.0, rms2=0.0, n=0))
            st["max"] = max(st["max"], float(e.max()))
            st["rms2"] += float((e ** 2).sum())
            st["n"] += e.size
    report = {k: dict(max=v["max"], rms=(v["rms2"] / v["n"]) ** 0.5) for k, v in stats.items()}
    out_dir = os.environ.get("UPS_REPORT_DIR")  # optional folder for the measured errors
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, "bf16_decode_error.json"), "w") as f:
            json.dump(report, f, indent=1)
    print("bf16 decode error vs FP64 oracle:", json.dumps(report))
    for k, (bmax, brms) in BF16_BOUNDS.items():
        assert report[k]["max"] < bmax and report[k]["rms"] < brms, (k, report[k])
