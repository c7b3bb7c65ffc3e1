"""Shared helpers of the GPU parity tests: run one seeded case through the CUDA
library (via the C ABI binding) and through the FP64 oracle on the same
float32-rounded inputs, and compare."""
import numpy as np

import oracle
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

CFG = oracle.RenderCfg()
PIX_ATOL, PIX_RTOL = 1e-5, 1e-4      # forward pixels
GRAD_RTOL = 2e-3                     # relative L2 of gradients
MARGIN = 1e-4                        # pixels this close to a threshold are compared separately


def r32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def round_dict(d):
    return {k: r32(v) for k, v in d.items()}


def round_cams(cams):
    for c in cams:
        c.T_cw = r32(c.T_cw)
        c.t_norm = float(np.float32(c.t_norm))
    return cams


def split_images(img, cams, nf):
    """Flat library images -> per-view dicts of numpy arrays."""
    out = []
    P = 0
    col = img["color"].cpu().numpy().astype(np.float64)
    dep = img["depth"].cpu().numpy().astype(np.float64)
    fea = img["feat"].cpu().numpy().astype(np.float64) if nf else None
    T = img["T"].cpu().numpy().astype(np.float64)
    nc = img["n_contrib"].cpu().numpy()
    for c in cams:
        h, w = c.height, c.width
        hw = h * w
        out.append(dict(color=col[3 * P:3 * P + 3 * hw].reshape(3, h, w),
                        depth=dep[P:P + hw].reshape(h, w),
                        feat=(fea[nf * P:nf * P + nf * hw].reshape(nf, h, w) if nf else np.zeros((0, h, w))),
                        T=T[P:P + hw].reshape(h, w), n_contrib=nc[P:P + hw].reshape(h, w)))
        P += hw
    return out


def feat_magnitude(proj, g, cam, nf):
    """sum_i w_i |f_i| per pixel and channel: the scale of the blended terms of
    Eq. 10.  Feature channels are signed, so the blended sum can cancel to far
    below its terms; the relative part of the pixel bar is taken against this
    magnitude (for non-negative channels it equals the pixel value itself)."""
    if not nf:
        return None
    ga = dict(g)
    ga["feat"] = np.abs(g["feat"])
    return oracle.render(proj, ga, cam, CFG, nf)["feat"]


def last_blended_ids(nc, lst, rng, tile_base=0, id_base=0):
    """Id of the last blended Gaussian of every pixel (-1 if none), from n_contrib
    and the tile lists.  List positions can shift between two correct renders
    when a tile list holds an extra Gaussian that blends nothing (a rect edge or
    depth tie decided differently), so pixels are compared by this id."""
    H, W = nc.shape
    tx = (W + 15) // 16
    t = (np.arange(H)[:, None] // 16) * tx + (np.arange(W)[None, :] // 16) + tile_base
    pos = rng[t, 0].astype(np.int64) + nc.astype(np.int64) - 1
    pos = np.clip(pos, 0, max(len(lst) - 1, 0))
    ids = lst[pos].astype(np.int64) - id_base if len(lst) else np.zeros_like(pos)
    return np.where(nc > 0, ids, -1)


def blend_ids(res, gpu_views):
    """Per view, (GPU, oracle) id of every pixel's last blended Gaussian: the
    GPU's tile lists may hold an extra Gaussian whose ellipse passes within the
    FP32 margin of a tile without blending there, which shifts n_contrib but not
    the blended Gaussians."""
    R, cams = res["R"], res["cams"]
    glist = R.copy_buffer(0)
    grng = R.copy_buffer(2).reshape(-1, 2)
    N = res["views"][0]["proj"]["valid"].shape[0]
    out, tile_base = [], 0
    for v, (cam, vw) in enumerate(zip(cams, res["views"])):
        lst, rng = oracle.tile_lists(vw["proj"], cam, CFG)
        out.append((last_blended_ids(gpu_views[v]["n_contrib"], glist, grng, tile_base, v * N),
                    last_blended_ids(vw["img"]["n_contrib"], lst, rng)))
        tile_base += ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    return out


def depth_tie(za, zb, ulps=4):
    """True where two depths are within `ulps` float32 ulps (order may flip)."""
    za = np.asarray(za, np.float32)
    zb = np.asarray(zb, np.float32)
    return np.abs(za.view(np.int32).astype(np.int64) - zb.view(np.int32).astype(np.int64)) <= ulps


def tie_explained(nc_gpu, nc_ref, lst, rng, z):
    """Pixels whose tile list (oracle order) has two consecutive Gaussians with
    float32 depths within 4 ulps before the end of the pixel's blended prefix:
    there the two renders may order the pair differently, which can move the
    last blended Gaussian (including through the termination rule)."""
    H, W = nc_ref.shape
    tx = (W + 15) // 16
    nt = rng.shape[0]
    zl = np.asarray(z, np.float32)[lst] if len(lst) else np.zeros(0, np.float32)
    first = np.full(nt, np.iinfo(np.int64).max, np.int64)
    if len(lst) > 1:
        same_tile = np.zeros(len(lst) - 1, bool)
        tile_of = np.repeat(np.arange(nt), rng[:, 1] - rng[:, 0])
        same_tile = tile_of[1:] == tile_of[:-1]
        tie = depth_tie(zl[1:], zl[:-1]) & same_tile
        idx = np.nonzero(tie)[0]
        pos_in_tile = idx - rng[tile_of[idx], 0]
        np.minimum.at(first, tile_of[idx], pos_in_tile)
    t = (np.arange(H)[:, None] // 16) * tx + (np.arange(W)[None, :] // 16)
    end = np.maximum(nc_gpu, nc_ref).astype(np.int64)
    return first[t] <= end


def assert_pixels(gpu_views, ref_views, nf, max_flag_frac=0.01, feat_mag=None, last_ids=None,
                  tie_ok=None):
    flagged = 0
    total = 0
    for vi, (gv, rv) in enumerate(zip(gpu_views, ref_views)):
        ok = rv["margin"] > MARGIN
        flagged += int((~ok).sum())
        total += ok.size
        for k in ("color", "depth", "T") + (("feat",) if nf else ()):
            a, r = gv[k], rv[k]
            diff = np.abs(a - r)
            scale = np.abs(r)
            if k == "feat" and feat_mag is not None:
                scale = np.maximum(scale, feat_mag[vi])
            tol = PIX_ATOL + PIX_RTOL * scale
            bad = (diff > tol) & np.broadcast_to(ok, diff.shape)
            assert not bad.any(), (k, int(bad.sum()), float(diff[bad].max()))
        if last_ids is None:
            assert np.array_equal(gv["n_contrib"][ok], rv["n_contrib"][ok])
        else:
            a, b = last_ids[vi]
            bad = ok & (a != b)
            if bad.any() and tie_ok is not None:
                # allowed only where a float32 depth near-tie precedes the end
                # of the blended prefix; counted and bounded
                assert tie_ok[vi][bad].all(), int((~tie_ok[vi][bad]).sum())
                assert bad.sum() <= 1e-4 * bad.size + 10, int(bad.sum())
            else:
                assert not bad.any(), int(bad.sum())
    assert flagged <= max_flag_frac * total, (flagged, total)
    return flagged


def rel_l2(a, r):
    a = np.asarray(a, np.float64).reshape(-1)
    r = np.asarray(r, np.float64).reshape(-1)
    return float(np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30))


def assert_grad(name, a, r, tol=GRAD_RTOL):
    e = rel_l2(a, r)
    assert e < tol, (name, e)
    return e


def gauss_grads(grad, nf, sets):
    mo = grad.mean_opacity.cpu().numpy().astype(np.float64)
    sc = grad.scale.cpu().numpy().astype(np.float64)
    qt = grad.quat.cpu().numpy().astype(np.float64)
    co = grad.color.cpu().numpy().astype(np.float64)
    fe = grad.feat.cpu().numpy().astype(np.float64)
    return dict(mean=mo[..., :3], opacity=mo[..., 3], scale=sc[..., :3], quat=qt,
                color=co[..., :3], feat=fe)


def plain_case(seed, n, cams, nf, weighted, l2=False, lambda_scale=0.0, g=None, list_cap=0):
    """Plain Gaussians shared by all views: GPU forward+loss+backward vs oracle
    (list_cap: 0 the library default, < 0 whole tile lists)."""
    if g is None:
        g = scenes.plain_gaussians(seed, n, nf)
    g = round_dict(g)
    cams = round_cams(cams)
    tg = [round_dict(t) for t in scenes.targets(seed + 1, cams, nf, weighted=weighted)]
    lc = oracle.LossCfg(lambda_scale=lambda_scale, l2=l2)
    R = B.Renderer(n_feat=nf, k=1, list_cap=list_cap)
    gs = B.to_set(g)
    img = R.forward(gs, cams)
    loss, dimg = R.loss(img, B.targets_to_device(tg), lambda_scale=lambda_scale, l2=l2, g=gs)
    sg = lambda_scale / (3.0 * n) if lambda_scale else 0.0
    grad, d_pose = R.backward(dimg, B.GRAD_POSE | B.GRAD_GAUSS, scale_grad=sg)
    L, ref, views, per_view = oracle.backward_plain(g, cams, tg, CFG, lc, nf)
    return dict(R=R, g=g, gs=gs, cams=cams, tg=tg, img=img, loss=float(loss.item()),
                grad=grad, d_pose=d_pose.cpu().numpy().astype(np.float64), L=L, ref=ref,
                views=views, per_view=per_view)


def check_plain(res, nf, grads=True):
    gpu_views = split_images(res["img"], res["cams"], nf)
    mag = [feat_magnitude(v["proj"], res["g"], c, nf) for v, c in zip(res["views"], res["cams"])]
    assert_pixels(gpu_views, [v["img"] for v in res["views"]], nf, feat_mag=mag,
                  last_ids=blend_ids(res, gpu_views))
    assert abs(res["loss"] - res["L"]) <= 1e-5 + 1e-4 * abs(res["L"]), (res["loss"], res["L"])
    if not grads:
        return
    gg = gauss_grads(res["grad"], nf, 1)
    for k in ("mean", "scale", "quat", "opacity", "color") + (("feat",) if nf else ()):
        assert_grad(k, gg[k][0], res["ref"][k])
    assert_grad("pose", res["d_pose"], res["ref"]["pose"])
