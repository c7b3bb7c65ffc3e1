"""Shared helpers of the GPU parity tests: run one seeded case through the CUDA
library (via the C ABI binding) and through the FP64 oracle on the same
float32-rounded inputs, and compare."""
import json
import os

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


# ---------------------------------------------------------------------------
# full-size tile lists: depth ties from the FP32 error bound, the margin band
# ---------------------------------------------------------------------------

U32 = 2.0 ** -24          # unit roundoff of float32, round to nearest
MARGIN_Q = 1e-4           # the kernel's relative margin on the alpha_min ellipse
MARGIN_PX = 1e-3          # the kernel's margin on every tile box and the rect, in pixels


def z_error_bound(mean, T_cw):
    """A-priori bound of the rounding error of the kernel's camera depth.

    The kernel evaluates z = fma(r20, x, fma(r21, y, fma(r22, z, t2))) on the
    same float32 inputs as the oracle (mean and pose rounded to float32 on both
    sides): three FMAs, each rounding once, so
    |z32 - z| <= u (|s1| + |s2| + |s3|), s1 = r22 z + t2, s2 = r21 y + s1,
    s3 = r20 x + s2, u = 2^-24 (first order; the 1e-6 factor covers the rest)."""
    m = np.asarray(mean, np.float64)
    R = np.asarray(T_cw, np.float64)
    s1 = R[2, 2] * m[:, 2] + R[2, 3]
    s2 = R[2, 1] * m[:, 1] + s1
    s3 = R[2, 0] * m[:, 0] + s2
    return U32 * (np.abs(s1) + np.abs(s2) + np.abs(s3)) * (1.0 + 1e-6)


def tie_groups(lst, rng, z64, ebound):
    """Group id of every entry of the oracle's tile lists (oracle order):
    consecutive entries of a tile whose FP64 depths are closer than the sum of
    their FP32 error bounds plus one float32 ulp (the oracle's own key is
    float32(z), ids break its ties) may be ordered either way by the GPU, and
    share a group.  Groups are numbered increasingly along the lists."""
    if len(lst) == 0:
        return np.zeros(0, np.int64)
    zl = np.asarray(z64, np.float64)[lst]
    el = np.asarray(ebound, np.float64)[lst]
    nt = rng.shape[0]
    tile_of = np.repeat(np.arange(nt), rng[:, 1] - rng[:, 0])
    win = el[1:] + el[:-1] + np.spacing(np.abs(zl[1:]).astype(np.float32)).astype(np.float64)
    tied = (np.abs(zl[1:] - zl[:-1]) <= win) & (tile_of[1:] == tile_of[:-1])
    return np.cumsum(np.concatenate([[True], ~tied])) - 1


def compare_tile_lists(glist, grng, lst, rng, grp, cap):
    """Per tile, the GPU's list (local Gaussian ids) against the oracle's.

    Expected: every oracle entry is in the GPU list (up to the cut of a capped
    list), the GPU list may hold extra entries (checked separately against the
    margin band), no entry twice, and the GPU order equals the oracle order up
    to reordering inside a tie group; a capped GPU list holds exactly the first
    entries of the oracle list, up to which members of the tie group at the cut
    it kept.  Returns counts and the (tile, id) pairs of extras and missing."""
    out = dict(tiles=0, cut=0, dup=0, order=0, prefix=0, extra=[], missing=[], compared=0)
    nt = rng.shape[0]
    for t in range(nt):
        a = glist[grng[t, 0]:grng[t, 1]].astype(np.int64)
        b = lst[rng[t, 0]:rng[t, 1]].astype(np.int64)
        gb = grp[rng[t, 0]:rng[t, 1]]
        out["tiles"] += 1
        if len(np.unique(a)) != len(a):
            out["dup"] += 1
        if len(b):
            srt = np.argsort(b, kind="stable")
            idx = np.searchsorted(b, a, sorter=srt)
            idx = np.minimum(idx, len(b) - 1)
            found = b[srt[idx]] == a
            pos = srt[idx[found]]
        else:
            found = np.zeros(len(a), bool)
            pos = np.zeros(0, np.int64)
        for g in a[~found]:
            out["extra"].append((t, int(g)))
        ga = gb[pos]
        if len(ga) > 1 and np.any(np.diff(ga) < 0):
            out["order"] += 1
        k = len(pos)
        out["compared"] += k
        cut = cap > 0 and len(a) >= cap
        if cut:
            out["cut"] += 1
            if not np.array_equal(ga, gb[:k]):
                out["prefix"] += 1
                miss = np.setdiff1d(b[:k], a)
                for g in miss:
                    out["missing"].append((t, int(g)))
        else:
            inb = np.zeros(len(b), bool)
            inb[pos] = True
            for g in b[~inb]:
                out["missing"].append((t, int(g)))
    return out


def box_min_q(conic, du0, du1, dv0, dv1):
    """Minimum of q = a dx^2 + 2 b dx dy + c dy^2 over the boxes
    [du0, du1] x [dv0, dv1] (arrays; conic rows (a, b, c)): 0 when the box holds
    the centre, else the least of the edge minima (q is convex, so on an edge
    its minimum is at the clamped stationary point)."""
    a, b, c = conic[:, 0], conic[:, 1], conic[:, 2]
    best = np.where((du0 <= 0) & (du1 >= 0) & (dv0 <= 0) & (dv1 >= 0), 0.0, np.inf)
    for dx in (du0, du1):
        dy = np.clip(-b * dx / c, dv0, dv1)
        best = np.minimum(best, a * dx ** 2 + 2 * b * dx * dy + c * dy ** 2)
    for dy in (dv0, dv1):
        dx = np.clip(-b * dy / a, du0, du1)
        best = np.minimum(best, a * dx ** 2 + 2 * b * dx * dy + c * dy ** 2)
    return best


def tile_q_ratio(proj, cam, pairs, grow=0.0, alpha_min=1.0 / 255):
    """For (tile, id) pairs: min over the tile's box of pixel centres (grown by
    `grow` px on each side) of the Gaussian's quadratic form, over the
    alpha_min threshold k2 = 2 ln(o / alpha_min) (FP64, oracle projection);
    <= 1 where the exact alpha_min ellipse meets the box.  Also returns the
    condition number of the 2D covariance of each pair's Gaussian."""
    if not pairs:
        return np.zeros(0), np.zeros(0)
    pr = np.asarray(pairs, np.int64)
    t, g = pr[:, 0], pr[:, 1]
    tx_n = (cam.width + 15) // 16
    tx, ty = t % tx_n, t // tx_n
    x0 = 16.0 * tx - grow
    x1 = np.minimum(16.0 * tx + 15, cam.width - 1) + grow
    y0 = 16.0 * ty - grow
    y1 = np.minimum(16.0 * ty + 15, cam.height - 1) + grow
    u, v = proj["uv"][g, 0], proj["uv"][g, 1]
    cn = proj["conic"][g]
    q = box_min_q(cn, x0 - u, x1 - u, y0 - v, y1 - v)
    k2 = 2.0 * np.log(proj["opacity"][g] / alpha_min)
    tr = cn[:, 0] + cn[:, 2]
    det = cn[:, 0] * cn[:, 2] - cn[:, 1] ** 2
    disc = np.sqrt(np.maximum(tr ** 2 / 4 - det, 0))
    kappa = (tr / 2 + disc) / np.maximum(tr / 2 - disc, 1e-300)
    return q / k2, kappa


def tie_explained_groups(nc_gpu, nc_ref, lst, rng, grp):
    """Pixels whose tile list (oracle order) holds a depth-tie group of two or
    more entries (tie_groups) starting before the end of the pixel's blended
    prefix: there the two renders may order the group's members differently,
    which can move the last blended Gaussian."""
    H, W = nc_ref.shape
    tx = (W + 15) // 16
    nt = rng.shape[0]
    first = np.full(nt, np.iinfo(np.int64).max, np.int64)
    if len(lst) > 1:
        tile_of = np.repeat(np.arange(nt), rng[:, 1] - rng[:, 0])
        idx = np.nonzero((grp[1:] == grp[:-1]) & (tile_of[1:] == tile_of[:-1]))[0]
        np.minimum.at(first, tile_of[idx], idx - rng[tile_of[idx], 0])
    t = (np.arange(H)[:, None] // 16) * tx + (np.arange(W)[None, :] // 16)
    end = np.maximum(nc_gpu, nc_ref).astype(np.int64)
    return first[t] < end


def report(name, data):
    """Print a measured-error report; also write it as JSON into the folder
    named by UPS_REPORT_DIR when that is set."""
    print(name, json.dumps(data))
    out_dir = os.environ.get("UPS_REPORT_DIR")
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, name + ".json"), "w") as f:
            json.dump(data, f, indent=1)
