"""FP64 CPU oracle of the anchor-decoded Gaussian render path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it.

The arithmetic lives in ``ups_oracle.c`` (plain C, double precision, one view
per call); this module marshals numpy arrays through ctypes and composes the
per-view steps into the full loss and its gradients:

  decode (Eq. 8-9) -> project (Eq. 1-2) -> blend (Eq. 3, Eq. 10)
  -> weighted loss (Eq. 4 / Eq. 14) -> analytic backward of each step;
  and, in numpy, the tracking uncertainty (Eq. 6 residual, Eq. 15 minimiser),
  the feature lifting with its distillation loss (Eq. 11-12), the uncertainty
  MLP with L_u (Eq. 5, Eq. 13), the D-SSIM term of Eq. 4 and the probabilistic
  anchor update with pruning and insertion (Eq. 7).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ups_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libups_oracle.so")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:2] + ["-fopenmp"] + base[2:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_tile_lists.restype = C.c_long
        _lib.orc_loss_view.restype = C.c_double
        _lib.orc_num_threads.restype = C.c_int
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


class _Cam(C.Structure):
    _fields_ = [("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("width", C.c_int), ("height", C.c_int),
                ("Tcw", C.c_double * 16)]


class _Cfg(C.Structure):
    _fields_ = [("alpha_min", C.c_double), ("alpha_max", C.c_double),
                ("t_min", C.c_double), ("dilation", C.c_double),
                ("near_z", C.c_double), ("guard", C.c_double),
                ("tile", C.c_int), ("brute", C.c_int)]


@dataclass
class RenderCfg:
    """Thresholds of the blending (readings of what Eq. 3 leaves open)."""
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    dilation: float = 0.3
    near_z: float = 0.2
    guard: float = 1.3
    tile: int = 16
    brute: bool = False

    def c(self):
        return _Cfg(self.alpha_min, self.alpha_max, self.t_min, self.dilation,
                    self.near_z, self.guard, self.tile, int(self.brute))


@dataclass
class LossCfg:
    """Image-loss weights (Eq. 4 / Eq. 14 with the per-pixel weight map)."""
    lambda_color: float = 1.0
    lambda_depth: float = 1.0
    lambda_feat: float = 1.0
    lambda_scale: float = 0.0
    l2: bool = False


def _cam(cam):
    T = np.ascontiguousarray(np.asarray(cam.T_cw, dtype=np.float64).reshape(16))
    return _Cam(float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
                int(cam.width), int(cam.height), (C.c_double * 16)(*T))


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _zeros(*shape):
    a = np.zeros(shape, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


# ----------------------------------------------------------------------------
# per-view steps
# ----------------------------------------------------------------------------

def decode(anc, mlp, cam, k, n_feat, opacity_tanh=False):
    """Eq. 8-9 for one view: returns mean, opacity, scale, quat, color, feat
    (opacity sigmoid, or tanh with opacity_tanh: the Scaffold-GS decode)."""
    A, F = anc["feat"].shape
    H = mlp["w2"].shape[1]
    keep = []
    args = []
    for name in ("pos", "feat", "offsets", "scaling"):
        a, p = _d(anc[name]); keep.append(a); args.append(p)
    for name in ("w1", "b1", "w2", "b2"):
        a, p = _d(mlp[name]); keep.append(a); args.append(p)
    N = A * k
    mean, pm = _zeros(N, 3)
    op, po = _zeros(N)
    sc, ps = _zeros(N, 3)
    qt, pq = _zeros(N, 4)
    co, pc = _zeros(N, 3)
    fe, pf = _zeros(N, n_feat)
    c = _cam(cam)
    lib().orc_decode_view(A, k, F, H, n_feat, int(bool(opacity_tanh)), *args, C.byref(c), C.c_double(cam.t_norm),
                          pm, po, ps, pq, pc, pf)
    return dict(mean=mean, opacity=op, scale=sc, quat=qt, color=co, feat=fe)


def project(g, cam, cfg: RenderCfg):
    """Eq. 1-2 for one view."""
    N = g["mean"].shape[0]
    keep = []
    args = []
    for name in ("mean", "opacity", "scale", "quat"):
        a, p = _d(g[name]); keep.append(a); args.append(p)
    valid = np.zeros(N, np.int32)
    rect = np.zeros((N, 4), np.int32)
    pcam, pp = _zeros(N, 3)
    uv, pu = _zeros(N, 2)
    cov, pcv = _zeros(N, 3)
    conic, pcn = _zeros(N, 3)
    ext, pe = _zeros(N, 4)
    c = _cam(cam)
    cf = cfg.c()
    lib().orc_project_view(N, *args, C.byref(c), C.byref(cf), valid.ctypes.data_as(_ip),
                           pp, pu, pcv, pcn, rect.ctypes.data_as(_ip), pe)
    return dict(valid=valid, pcam=pcam, uv=uv, cov2d=cov, conic=conic, rect=rect,
                extent=ext, opacity=np.ascontiguousarray(g["opacity"], dtype=np.float64))


def tile_lists(proj, cam, cfg: RenderCfg):
    """Per-tile Gaussian lists in ascending (float32(z), id) and their ranges: a
    tile of a Gaussian's rect lists it when the alpha >= alpha_min ellipse meets
    the tile's box of pixel centres."""
    N = proj["valid"].shape[0]
    tx = (cam.width + cfg.tile - 1) // cfg.tile
    ty = (cam.height + cfg.tile - 1) // cfg.tile
    va, pv = _i(proj["valid"])
    pc, ppc = _d(proj["pcam"])
    rc, prc = _i(proj["rect"])
    uv, puv = _d(proj["uv"])
    cn, pcn = _d(proj["conic"])
    op, pop = _d(proj["opacity"])
    args = (N, pv, ppc, prc, puv, pcn, pop, C.c_double(cfg.alpha_min), cam.width, cam.height, cfg.tile)
    total = lib().orc_tile_lists(*args, None, None)
    lst = np.zeros(max(total, 1), np.int32)
    rng = np.zeros((tx * ty, 2), np.int32)
    lib().orc_tile_lists(*args, lst.ctypes.data_as(_ip), rng.ctypes.data_as(_ip))
    return lst[:total], rng


def render(proj, g, cam, cfg: RenderCfg, n_feat):
    """Eq. 3 / Eq. 10 for one view: colour, depth, feature, T_final, n_contrib."""
    N = proj["valid"].shape[0]
    H, W = cam.height, cam.width
    keep = []
    va, pv = _i(proj["valid"]); keep.append(va)
    rc, prc = _i(proj["rect"]); keep.append(rc)
    ptr = {}
    for name, src in (("pcam", proj), ("uv", proj), ("conic", proj),
                      ("opacity", g), ("color", g)):
        a, p = _d(src[name]); keep.append(a); ptr[name] = p
    fe, pf = _d(g["feat"] if n_feat else np.zeros((N, 0)))
    col, pcol = _zeros(3, H, W)
    dep, pdep = _zeros(H, W)
    fo, pfo = _zeros(n_feat, H, W)
    T, pT = _zeros(H, W)
    nc = np.zeros((H, W), np.int32)
    mg, pmg = _zeros(H, W)
    c = _cam(cam)
    cf = cfg.c()
    lib().orc_render_view(N, n_feat, pv, ptr["pcam"], ptr["uv"], ptr["conic"],
                          ptr["opacity"], ptr["color"], pf, prc, C.byref(c), C.byref(cf),
                          pcol, pdep, pfo, pT, nc.ctypes.data_as(_ip), pmg)
    return dict(color=col, depth=dep, feat=fo, T=T, n_contrib=nc, margin=mg)


def loss_view(img, tgt, lcfg: LossCfg, n_feat, norm):
    """Weighted image loss of one view and its image gradients."""
    H, W = img["depth"].shape
    keep = []
    ptr = []
    for a in (img["color"], img["depth"], img["feat"] if n_feat else np.zeros(1),
              tgt["color"], tgt["depth"], tgt["feat"] if n_feat else np.zeros(1),
              tgt["weight"]):
        arr, p = _d(a); keep.append(arr); ptr.append(p)
    gc, pgc = _zeros(3, H, W)
    gd, pgd = _zeros(H, W)
    gf, pgf = _zeros(n_feat, H, W)
    L = lib().orc_loss_view(W, H, n_feat, *ptr, C.c_double(lcfg.lambda_color),
                            C.c_double(lcfg.lambda_depth), C.c_double(lcfg.lambda_feat),
                            int(lcfg.l2), C.c_double(norm), pgc, pgd,
                            pgf if n_feat else None)
    return L, dict(color=gc, depth=gd, feat=gf)


@dataclass
class ResidualCfg:
    """Residual weights and visibility threshold of the tracking uncertainty
    (Eq. 6; the values of Sec. 4 "Implementation Details")."""
    lambda_color: float = 0.25
    lambda_depth: float = 0.7
    lambda_feat: float = 0.1
    t_mask: float = 0.1


def box3(d):
    """B (Eq. 6): 3x3 box filter, the mean over the window's pixels inside the
    image (reading: the window is cut at the border, not padded)."""
    H, W = d.shape
    s = np.zeros((H, W))
    n = np.zeros((H, W))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            ys = slice(max(0, -dy), H - max(0, dy))   # pixels whose neighbour (y+dy, x+dx) is inside
            xs = slice(max(0, -dx), W - max(0, dx))
            yn = slice(max(0, dy), H - max(0, -dy))   # those neighbours
            xn = slice(max(0, dx), W - max(0, -dx))
            s[ys, xs] += d[yn, xn]
            n[ys, xs] += 1.0
    return s / n


def tracking_uncertainty(img, tgt, rcfg: ResidualCfg, n_feat):
    """Training-free uncertainty of one view (Sec. 3.4 "Tracking").

    Eq. 6:  R = (T < t_mask) (l1 |C~ - C|_1 + l2 |D~ - B(D)| + l3 ceil1(1 - cos(F, F~)))
    with T the final transmittance (Eq. 3's T~ read as transmittance: the mask
    keeps covered pixels), |.|_1 the sum over the colour channels, ceil1 the cap
    at 1, and cos = 0 when either feature vector is zero.
    Eq. 15 minimises 1/2 (R / sigma^2 + log sigma) pixel by pixel; setting the
    derivative 1/2 (-2R / sigma^3 + 1 / sigma) to zero gives sigma^2 = 2R (R = 0:
    the limit 0), and the motion mask 2 sigma^2 > 1 (Sec. 3.3) is R > 1/4.
    Returns R, sigma2 and the motion mask (uint8) as [H, W] arrays."""
    rc = np.abs(img["color"] - tgt["color"]).sum(axis=0)
    rd = np.abs(img["depth"] - box3(tgt["depth"]))
    if n_feat:
        f, fh = tgt["feat"], img["feat"]
        dot = (f * fh).sum(axis=0)
        na = np.sqrt((f * f).sum(axis=0))
        nb = np.sqrt((fh * fh).sum(axis=0))
        ok = (na > 0) & (nb > 0)
        cos = np.where(ok, dot / np.where(ok, na * nb, 1.0), 0.0)
        rf = np.minimum(1.0, 1.0 - cos)
    else:
        rf = np.zeros_like(rd)
    R = np.where(img["T"] < rcfg.t_mask,
                 rcfg.lambda_color * rc + rcfg.lambda_depth * rd + rcfg.lambda_feat * rf, 0.0)
    sigma2 = 2.0 * R
    motion = (2.0 * sigma2 > 1.0).astype(np.uint8)
    return R, sigma2, motion


@dataclass
class LiftCfg:
    """DINO feature width and patch size of the feature lifting (Eq. 11-12)."""
    n_h: int = 384
    patch: int = 14


def dino_upsample(grid, H, W, patch):
    """Sec. 3.2: DINO features are per image patch and bilinearly upsampled to
    the image.  grid [hp][wp][n_h]; pixel (x, y) samples it at
    ((x + 0.5) / patch - 0.5, (y + 0.5) / patch - 0.5), clamped to the grid.
    Returns [n_h][H][W]."""
    hp, wp, _ = grid.shape
    u = np.clip((np.arange(W) + 0.5) / patch - 0.5, 0.0, wp - 1)
    v = np.clip((np.arange(H) + 0.5) / patch - 0.5, 0.0, hp - 1)
    x0 = np.floor(u).astype(int); y0 = np.floor(v).astype(int)
    x1 = np.minimum(x0 + 1, wp - 1); y1 = np.minimum(y0 + 1, hp - 1)
    ax = (u - x0)[None, :, None]; ay = (v - y0)[:, None, None]
    top = (1 - ax) * grid[y0][:, x0] + ax * grid[y0][:, x1]
    bot = (1 - ax) * grid[y1][:, x0] + ax * grid[y1][:, x1]
    return np.moveaxis((1 - ay) * top + ay * bot, 2, 0)


def feature_lift(feat, grid, mlp, lcfg: LiftCfg, n_pix, scale=1.0, weight=None):
    """Feature lifting and distillation of one view (Sec. 3.3, Eq. 11-12; App.
    "MLP Implementation Details": F_m = conv -> ReLU -> conv, hidden 128, read as
    1x1 convolutions, i.e. the same MLP at every pixel).

    F^_p = W2 relu(W1 F~_p + b1) + b2;  loss = scale / n_pix * sum_p (1 - cos(F_p, F^_p))
    (n_pix: pixels of all views; cos = 0, and no gradient, where a vector is 0),
    with F the upsampled DINO feature.  Returns the loss contribution and
    scale * d(loss)/d(w1, b1, w2, b2, feat)."""
    nf, H, W = feat.shape
    X = feat.reshape(nf, H * W).T                       # [P][nf]
    Z = X @ mlp["w1"].T + mlp["b1"]                     # [P][128]
    Hh = np.maximum(Z, 0.0)
    Fh = Hh @ mlp["w2"].T + mlp["b2"]                   # [P][n_h]
    T = dino_upsample(grid, H, W, lcfg.patch).reshape(lcfg.n_h, H * W).T
    na = np.sqrt((T * T).sum(1)); nb = np.sqrt((Fh * Fh).sum(1))
    ok = (na > 0) & (nb > 0)
    den = np.where(ok, na * nb, 1.0)
    cos = np.where(ok, (T * Fh).sum(1) / den, 0.0)
    wp = np.ones(H * W) if weight is None else weight.reshape(-1)   # per-pixel weight (Eq. 14's mask)
    g = scale / n_pix * wp
    loss = (g * (1.0 - cos)).sum()
    # d(1 - cos)/dF^ = cos F^ / |F^|^2 - F / (|F| |F^|)
    nb2 = np.where(ok, nb * nb, 1.0)
    dFh = np.where(ok[:, None], g[:, None] * (cos[:, None] * Fh / nb2[:, None] - T / den[:, None]), 0.0)
    dW2 = dFh.T @ Hh
    db2 = dFh.sum(0)
    dZ = (dFh @ mlp["w2"]) * (Z > 0)
    dW1 = dZ.T @ X
    db1 = dZ.sum(0)
    dX = dZ @ mlp["w1"]
    return loss, dict(w1=dW1, b1=db1, w2=dW2, b2=db2, feat=dX.T.reshape(nf, H, W))


def uncertainty_mlp(grid, R, mlp, lcfg: LiftCfg, n_pix, lam=1.0, scale=1.0):
    """Uncertainty MLP and its loss for one view (Sec. 3.3 "Uncertainty
    Prediction for Mapping", Eq. 5, Eq. 13; App.): F_u = conv -> ReLU -> conv ->
    SoftPlus (1x1, hidden 128, one output) on the upsampled DINO feature F_p:
        sigma_p = softplus(w2 . relu(W1 F_p + b1) + b2)
        loss = scale / n_pix sum_p [R_p / (2 sigma_p^2) + lam log sigma_p]   (Eq. 5)
    The gradient goes to F_u's parameters only.  Returns the loss contribution,
    scale * d(loss)/d(w1, b1, w2, b2), sigma [H][W] and the mask 2 sigma^2 > 1."""
    H, W = R.shape
    F = dino_upsample(grid, H, W, lcfg.patch).reshape(lcfg.n_h, H * W).T   # [P][n_h]
    Z = F @ mlp["w1"].T + mlp["b1"]
    Hh = np.maximum(Z, 0.0)
    z2 = Hh @ mlp["w2"] + mlp["b2"][0]
    s = np.where(z2 > 20, z2, np.log1p(np.exp(np.minimum(z2, 20))))          # softplus
    r = R.reshape(-1)
    g = scale / n_pix
    loss = g * (r / (2 * s * s) + lam * np.log(s)).sum()
    dz2 = g * (-r / s ** 3 + lam / s) / (1 + np.exp(-z2))                    # d/ds times softplus' = sigmoid
    dZ = dz2[:, None] * mlp["w2"][None, :] * (Z > 0)
    grads = dict(w1=dZ.T @ F, b1=dZ.sum(0), w2=Hh.T @ dz2, b2=np.array([dz2.sum()]))
    sigma = s.reshape(H, W)
    return loss, grads, sigma, (2 * sigma * sigma > 1).astype(np.uint8)


SSIM_C1, SSIM_C2 = 0.01 ** 2, 0.03 ** 2


def ssim_window(radius=5, sigma=1.5):
    """11 x 11 Gaussian window of SSIM (Wang et al.), sigma 1.5, summing to 1."""
    k = np.arange(-radius, radius + 1, dtype=float)
    w = np.exp(-k * k / (2.0 * sigma * sigma))
    w /= w.sum()
    return np.outer(w, w)


def ssim_loss(color, t_color, n_pix, scale=1.0, weight=None):
    """The D-SSIM term of Eq. 4 for one view: scale / (3 n_pix) sum over the three
    channels and the pixels of (1 - S), S the SSIM map of Wang et al. (the
    paper's citation): window moments mu, E[x^2], E[xy] with the Gaussian window
    and zero padding, C1 = 0.01^2, C2 = 0.03^2.  n_pix: pixels of all views.
    Returns the loss contribution and scale * d/d(color) ([3][H][W]).

    Gradient: S = A1 A2 / (B1 B2) with A1 = 2 mu_x mu_y + C1, A2 = 2 (E[xy] -
    mu_x mu_y) + C2, B1 = mu_x^2 + mu_y^2 + C1, B2 = E[x^2] - mu_x^2 + E[y^2] -
    mu_y^2 + C2; a pixel q enters the moments of p with weight w(q - p), so
    dS_p/dx_q = w(q - p) (dS/dmu_x + 2 x_q dS/dE[x^2] + y_q dS/dE[xy])(p)."""
    from scipy.ndimage import correlate
    W2 = ssim_window()
    conv = lambda a: correlate(a, W2, mode="constant", cval=0.0)             # sum_k w(k) a(p + k)
    back = lambda a: correlate(a, W2[::-1, ::-1], mode="constant", cval=0.0)  # sum_p w(q - p) a(p)
    g = scale / (3.0 * n_pix)
    loss = 0.0
    grad = np.zeros_like(color, dtype=float)
    for c in range(3):
        x, y = color[c], t_color[c]
        mx, my = conv(x), conv(y)
        exx, eyy, exy = conv(x * x), conv(y * y), conv(x * y)
        A1 = 2 * mx * my + SSIM_C1
        A2 = 2 * (exy - mx * my) + SSIM_C2
        B1 = mx * mx + my * my + SSIM_C1
        B2 = (exx - mx * mx) + (eyy - my * my) + SSIM_C2
        S = A1 * A2 / (B1 * B2)
        wp = 1.0 if weight is None else weight                              # per-pixel weight (Eq. 14's mask)
        loss += g * (wp * (1.0 - S)).sum()
        d_mu = wp * S * (2 * my / A1 - 2 * my / A2 - 2 * mx / B1 + 2 * mx / B2)  # w dS/dmu_x (E fixed)
        d_xx = wp * (-S / B2)                                                    # w dS/dE[x^2]
        d_xy = wp * (2 * S / A2)                                                 # w dS/dE[xy]
        grad[c] = -g * (back(d_mu) + 2 * x * back(d_xx) + y * back(d_xy))
    return loss, grad


def render_bwd(proj, g, cam, cfg: RenderCfg, n_feat, grads_img):
    """Backward of Eq. 3 / Eq. 10: per-Gaussian 2D gradients of one view."""
    N = proj["valid"].shape[0]
    keep = []
    va, pv = _i(proj["valid"]); keep.append(va)
    rc, prc = _i(proj["rect"]); keep.append(rc)
    ptr = {}
    for name, src in (("pcam", proj), ("uv", proj), ("conic", proj),
                      ("opacity", g), ("color", g)):
        a, p = _d(src[name]); keep.append(a); ptr[name] = p
    fe, pf = _d(g["feat"] if n_feat else np.zeros((N, 0)))
    gi = []
    for name in ("color", "depth", "feat", "T"):
        v = grads_img.get(name)
        if v is None or (name == "feat" and not n_feat):
            gi.append(None)
        else:
            a, p = _d(v); keep.append(a); gi.append(p)
    g_uv, p1 = _zeros(N, 2)
    g_cn, p2 = _zeros(N, 3)
    g_op, p3 = _zeros(N)
    g_co, p4 = _zeros(N, 3)
    g_z, p5 = _zeros(N)
    g_fe, p6 = _zeros(N, max(n_feat, 0))
    c = _cam(cam)
    cf = cfg.c()
    lib().orc_render_bwd_view(N, n_feat, pv, ptr["pcam"], ptr["uv"], ptr["conic"],
                              ptr["opacity"], ptr["color"], pf, prc, C.byref(c), C.byref(cf),
                              *gi, p1, p2, p3, p4, p5, p6)
    return dict(uv=g_uv, conic=g_cn, opacity=g_op, color=g_co, z=g_z, feat=g_fe)


def project_bwd(g, proj, cam, cfg: RenderCfg, g2d, scale_reg=0.0):
    """Backward of Eq. 1-2: gradients of mean, scale, quaternion and pose."""
    N = g["mean"].shape[0]
    keep = []
    args = []
    for name in ("mean", "scale", "quat"):
        a, p = _d(g[name]); keep.append(a); args.append(p)
    va, pv = _i(proj["valid"]); keep.append(va)
    gp = []
    for name in ("uv", "conic", "z"):
        a, p = _d(g2d[name]); keep.append(a); gp.append(p)
    gm, p1 = _zeros(N, 3)
    gs, p2 = _zeros(N, 3)
    gq, p3 = _zeros(N, 4)
    pose, p4 = _zeros(6)
    c = _cam(cam)
    cf = cfg.c()
    lib().orc_project_bwd_view(N, *args, pv, C.byref(c), C.byref(cf), *gp,
                               C.c_double(scale_reg), p1, p2, p3, p4)
    return dict(mean=gm, scale=gs, quat=gq, pose=pose)


def decode_bwd(anc, mlp, cam, k, n_feat, g3d, acc, opacity_tanh=False):
    """Backward of Eq. 8-9 for one view; accumulates into `acc`, returns pose[6]."""
    A, F = anc["feat"].shape
    H = mlp["w2"].shape[1]
    keep = []
    args = []
    for name in ("pos", "feat", "offsets", "scaling"):
        a, p = _d(anc[name]); keep.append(a); args.append(p)
    for name in ("w1", "b1", "w2", "b2"):
        a, p = _d(mlp[name]); keep.append(a); args.append(p)
    gin = []
    for name in ("mean", "opacity", "scale", "quat", "color", "feat"):
        a, p = _d(g3d[name]); keep.append(a); gin.append(p)
    outs = []
    for name in ("w1", "b1", "w2", "b2", "pos", "feat", "offsets", "scaling"):
        arr = acc[name]
        assert arr.dtype == np.float64 and arr.flags.c_contiguous
        outs.append(arr.ctypes.data_as(_dp))
    pose, pp = _zeros(6)
    c = _cam(cam)
    lib().orc_decode_bwd_view(A, k, F, H, n_feat, int(bool(opacity_tanh)), *args, C.byref(c),
                              C.c_double(cam.t_norm),
                              *gin, *outs, pp)
    return pose


# ----------------------------------------------------------------------------
# composed loss and gradients
# ----------------------------------------------------------------------------

def _norm(cams):
    return float(sum(c.width * c.height for c in cams))


def _scale_count(n_views_data, n):
    return 3.0 * n_views_data * n


def forward_plain(g, cams, tgts, cfg: RenderCfg, lcfg: LossCfg, n_feat, keep=False):
    """Loss of Gaussians given directly (shared by all views)."""
    norm = _norm(cams)
    L = 0.0
    views = []
    for cam, tgt in zip(cams, tgts):
        pr = project(g, cam, cfg)
        img = render(pr, g, cam, cfg, n_feat)
        Lv, gimg = loss_view(img, tgt, lcfg, n_feat, norm)
        L += Lv
        views.append(dict(proj=pr, img=img, gimg=gimg))
    if lcfg.lambda_scale:
        L += lcfg.lambda_scale * float(np.mean(g["scale"]))
    return (L, views) if keep else L


def backward_plain(g, cams, tgts, cfg: RenderCfg, lcfg: LossCfg, n_feat):
    """Loss and analytic gradients for shared Gaussians + per-view pose."""
    L, views = forward_plain(g, cams, tgts, cfg, lcfg, n_feat, keep=True)
    N = g["mean"].shape[0]
    out = dict(mean=np.zeros((N, 3)), scale=np.zeros((N, 3)), quat=np.zeros((N, 4)),
               opacity=np.zeros(N), color=np.zeros((N, 3)), feat=np.zeros((N, n_feat)),
               pose=np.zeros((len(cams), 6)))
    reg = lcfg.lambda_scale / _scale_count(1, N) if lcfg.lambda_scale else 0.0
    per_view = []
    for v, (cam, vw) in enumerate(zip(cams, views)):
        g2 = render_bwd(vw["proj"], g, cam, cfg, n_feat, vw["gimg"])
        g3 = project_bwd(g, vw["proj"], cam, cfg, g2, reg if v == 0 else 0.0)
        for k in ("mean", "scale", "quat"):
            out[k] += g3[k]
        out["opacity"] += g2["opacity"]
        out["color"] += g2["color"]
        out["feat"] += g2["feat"]
        out["pose"][v] = g3["pose"]
        per_view.append(dict(g2d=g2, g3d=g3))
    return L, out, views, per_view


def forward_anchor(anc, mlp, cams, tgts, cfg: RenderCfg, lcfg: LossCfg, k, n_feat,
                   keep=False, opacity_tanh=False):
    """Loss of anchor-decoded Gaussians (decode per view, then render)."""
    norm = _norm(cams)
    L = 0.0
    views = []
    ssum = 0.0
    for cam, tgt in zip(cams, tgts):
        g = decode(anc, mlp, cam, k, n_feat, opacity_tanh)
        pr = project(g, cam, cfg)
        img = render(pr, g, cam, cfg, n_feat)
        Lv, gimg = loss_view(img, tgt, lcfg, n_feat, norm)
        L += Lv
        ssum += float(np.sum(g["scale"]))
        views.append(dict(g=g, proj=pr, img=img, gimg=gimg))
    if lcfg.lambda_scale:
        N = anc["pos"].shape[0] * k
        L += lcfg.lambda_scale * ssum / _scale_count(len(cams), N)
    return (L, views) if keep else L


def backward_anchor(anc, mlp, cams, tgts, cfg: RenderCfg, lcfg: LossCfg, k, n_feat, opacity_tanh=False):
    """Loss and analytic gradients of MLP weights, anchors and per-view pose."""
    L, views = forward_anchor(anc, mlp, cams, tgts, cfg, lcfg, k, n_feat, keep=True, opacity_tanh=opacity_tanh)
    A = anc["pos"].shape[0]
    N = A * k
    acc = dict(w1=np.zeros_like(mlp["w1"]), b1=np.zeros_like(mlp["b1"]),
               w2=np.zeros_like(mlp["w2"]), b2=np.zeros_like(mlp["b2"]),
               pos=np.zeros_like(anc["pos"]), feat=np.zeros_like(anc["feat"]),
               offsets=np.zeros_like(anc["offsets"]), scaling=np.zeros_like(anc["scaling"]))
    acc = {kk: np.ascontiguousarray(v, dtype=np.float64) for kk, v in acc.items()}
    pose = np.zeros((len(cams), 6))
    reg = lcfg.lambda_scale / _scale_count(len(cams), N) if lcfg.lambda_scale else 0.0
    per_view = []
    for v, (cam, vw) in enumerate(zip(cams, views)):
        g = vw["g"]
        g2 = render_bwd(vw["proj"], g, cam, cfg, n_feat, vw["gimg"])
        g3 = project_bwd(g, vw["proj"], cam, cfg, g2, reg)
        g3d = dict(mean=g3["mean"], opacity=g2["opacity"], scale=g3["scale"],
                   quat=g3["quat"], color=g2["color"], feat=g2["feat"])
        pd = decode_bwd(anc, mlp, cam, k, n_feat, g3d, acc, opacity_tanh)
        pose[v] = g3["pose"] + pd
        per_view.append(dict(g2d=g2, g3d=g3d, pose_project=g3["pose"], pose_decode=pd))
    acc["pose"] = pose
    return L, acc, views, per_view


# ----------------------------------------------------------------------------
# probabilistic anchors (Sec. 3.3 "Adaptively Structured Gaussian", Eq. 7)
# ----------------------------------------------------------------------------

def logodds(p):
    """L(p) = log(p / (1 - p)), the log-odds of a probability."""
    return math.log(p / (1.0 - p))


def anchor_posterior(p_obs, p_prev, p_prior):
    """Eq. 7, in FP64, with the reading of its garbled last factor as
    P(n) / (1 - P(n)) (the Bayes update of OctoMap, which the paper cites):
      P(n|z_1:t) = [1 + (1 - P(n|z_t)) / P(n|z_t)
                          * (1 - P(n|z_1:t-1)) / P(n|z_1:t-1) * P(n) / (1 - P(n))]^-1."""
    return 1.0 / (1.0 + (1.0 - p_obs) / p_obs * (1.0 - p_prev) / p_prev * p_prior / (1.0 - p_prior))


@dataclass
class AnchorCfg:
    """Eq. 7 in log-odds form, L(n|z_1:t) = L(n|z_1:t-1) + L(n|z_t) - L(n),
    and the readings of its observation model (the paper states neither the
    inverse sensor model nor the thresholds; the probabilities are OctoMap's
    defaults).  Values are log-odds (FP32 on both implementations)."""
    l_prior: float = 0.0                     # L(P(n)), P(n) = 0.5
    l_hit: float = math.log(0.7 / 0.3)       # L(P(n|z_t)) of a static surface observation
    l_miss: float = math.log(0.4 / 0.6)      # ... of free space or a dynamic surface
    l_min: float = math.log(0.12 / 0.88)     # clamping of the posterior
    l_max: float = math.log(0.97 / 0.03)
    l_prune: float = 0.0                     # delete anchors whose posterior is below P = 0.5
    voxel: float = 0.05                      # anchor voxel edge (m)
    margin: float = 0.05                     # half-width of the surface band along the ray (m)
    near_z: float = 0.2                      # depths at or below this are not observations


VOXEL_RANGE = 1 << 20   # voxel indices in [-2^20, 2^20) on every axis


def _cam32(cam):
    T = np.asarray(cam.T_cw, dtype=np.float64).reshape(4, 4).astype(np.float32)
    f = np.float32
    return T[:3, :3], T[:3, 3], f(cam.fx), f(cam.fy), f(cam.cx), f(cam.cy)


def anchor_observe(pos, cam, depth, motion, acfg: AnchorCfg):
    """The observation z_t of each anchor in one keyframe (reading of the paper's
    occupancy observation; decisions in FP32, one rounding per operation in the
    order written): the anchor centre x goes to the camera, X = R x + t summed
    left to right, and to pixel (floor(fx X/Z + cx + 1/2), floor(fy Y/Z + cy + 1/2))
    (pixel (i, j) sits at image coordinate (i, j)).  With D the keyframe depth there:
      Z <= near_z, outside the image, or D <= near_z   -> no observation (0)
      Z <  D - margin  (the ray passed through x)      -> miss (2)
      Z <= D + margin  (x on the observed surface)     -> hit (1), or miss (2)
                                                          when the pixel is dynamic
      Z >  D + margin  (x hidden behind the surface)   -> no observation (0).
    Returns int8 [n]."""
    R, t, fx, fy, cx, cy = _cam32(cam)
    f = np.float32
    P = np.asarray(pos, np.float32).reshape(-1, 3)
    H, W = depth.shape
    Xc = [((R[r, 0] * P[:, 0] + R[r, 1] * P[:, 1]) + R[r, 2] * P[:, 2]) + t[r] for r in range(3)]
    Z = Xc[2]
    obs = np.zeros(P.shape[0], np.int8)
    front = Z > f(acfg.near_z)
    with np.errstate(all="ignore"):
        u = fx * (Xc[0] / Z) + cx
        v = fy * (Xc[1] / Z) + cy
        iu = np.floor(u + f(0.5))
        iv = np.floor(v + f(0.5))
    inside = front & (iu >= 0) & (iu < W) & (iv >= 0) & (iv < H)
    idx = np.nonzero(inside)[0]
    jj, ii = iv[idx].astype(np.int64), iu[idx].astype(np.int64)
    D = np.asarray(depth, np.float32)[jj, ii]
    dyn = (np.asarray(motion)[jj, ii] != 0) if motion is not None else np.zeros(len(idx), bool)
    z = Z[idx]
    valid = D > f(acfg.near_z)
    lo = D - f(acfg.margin)
    hi = D + f(acfg.margin)
    free = valid & (z < lo)
    surf = valid & (z >= lo) & (z <= hi)
    o = np.zeros(len(idx), np.int8)
    o[surf & ~dyn] = 1
    o[free | (surf & dyn)] = 2
    obs[idx] = o
    return obs


def _voxel(x, voxel):
    """floor(x / voxel) per axis in FP32 and whether every index is in range."""
    q = np.floor(np.asarray(x, np.float32) / np.float32(voxel))
    ok = np.all((q >= -VOXEL_RANGE) & (q < VOXEL_RANGE), axis=-1)
    return q, ok


def anchor_update(anc, logodds_in, cam, depth, motion, acfg: AnchorCfg, capacity):
    """One keyframe of the probabilistic anchor map (Sec. 3.3, Eq. 7; the
    probabilistic octree of Sec. 1 read as a voxel grid of edge `voxel` holding
    the anchors, whose probabilities decide deletion and whose empty voxels
    decide allocation):
      1. update: each observed anchor's log-odds l <- clamp(l + (L(z_t) - L(n)),
         l_min, l_max) (Eq. 7; unobserved anchors keep theirs);
      2. prune: anchors whose posterior log-odds is below l_prune are deleted,
         the rest keep their order;
      3. insert: every static pixel (motion 0) with a valid depth D > near_z is
         back-projected, x = R^T ((i - cx) / fx D - t_x, (j - cy) / fy D - t_y,
         D - t_z), to its voxel floor(x / voxel); each voxel that holds no kept
         anchor gets a new anchor at its centre, in the raster order of the first
         pixel that reached it, up to `capacity` anchors in total.  A new anchor
         starts from the prior with this one hit (l = clamp(L(n) + (L_hit - L(n)))),
         zero feature and offsets, and scaling = voxel (readings).
    FP32 throughout, one rounding per operation in the order written.
    anc: dict pos [n,3], feat [n,F], offsets [n,K,3], scaling [n,3]; depth [H,W];
    motion [H,W] uint8 or None (all static).  Returns a dict with the output
    arrays (pos, feat, offsets, scaling, logodds), src ([m] int: source row, or
    -1 - p for an anchor inserted from pixel p), n_kept, n_inserted, n_dropped
    (new voxels beyond capacity), n_hit, n_miss."""
    f = np.float32
    pos = np.asarray(anc["pos"], np.float32).reshape(-1, 3)
    n = pos.shape[0]
    l = np.asarray(logodds_in, np.float32).reshape(n).copy()
    obs = anchor_observe(pos, cam, depth, motion, acfg)
    dh = f(acfg.l_hit) - f(acfg.l_prior)
    dm = f(acfg.l_miss) - f(acfg.l_prior)
    lo, hi = f(acfg.l_min), f(acfg.l_max)
    upd = np.where(obs == 1, l + dh, l + dm)
    l = np.where(obs != 0, np.minimum(np.maximum(upd, lo), hi), l)
    keep = np.nonzero(l >= f(acfg.l_prune))[0]
    # insertion candidates
    R, t, fx, fy, cx, cy = _cam32(cam)
    H, W = depth.shape
    D = np.asarray(depth, np.float32)
    cand = D > f(acfg.near_z)
    if motion is not None:
        cand &= np.asarray(motion) == 0
    jj, ii = np.nonzero(cand)            # raster order
    d = D[jj, ii]
    Xc = [((ii.astype(np.float32) - cx) / fx) * d, ((jj.astype(np.float32) - cy) / fy) * d, d]
    dd = [Xc[r] - t[r] for r in range(3)]
    Xw = np.stack([(R[0, a] * dd[0] + R[1, a] * dd[1]) + R[2, a] * dd[2] for a in range(3)], axis=-1)
    q, ok = _voxel(Xw, acfg.voxel)
    pix = (jj * W + ii)[ok]
    q = q[ok].astype(np.int64)
    qa, oka = _voxel(pos[keep], acfg.voxel)
    held = set(map(tuple, qa[oka].astype(np.int64)))
    new_q, new_p = [], []
    if len(q):
        uq, first = np.unique(q, axis=0, return_index=True)
        order = np.argsort(first, kind="stable")
        for r in order:
            key = tuple(uq[r])
            if key not in held:
                new_q.append(uq[r])
                new_p.append(int(pix[first[r]]))
    n_kept = len(keep)
    n_ins = max(0, min(len(new_q), capacity - n_kept))
    nq = np.array(new_q[:n_ins], np.float32).reshape(-1, 3)
    F = np.asarray(anc["feat"]).shape[-1]
    K = np.asarray(anc["offsets"]).shape[-2]
    l_new = np.minimum(np.maximum(f(acfg.l_prior) + dh, lo), hi)
    vox = f(acfg.voxel)
    out = dict(
        pos=np.concatenate([pos[keep], (nq + f(0.5)) * vox]),
        feat=np.concatenate([np.asarray(anc["feat"], np.float32).reshape(n, F)[keep], np.zeros((n_ins, F), np.float32)]),
        offsets=np.concatenate([np.asarray(anc["offsets"], np.float32).reshape(n, K, 3)[keep],
                                np.zeros((n_ins, K, 3), np.float32)]),
        scaling=np.concatenate([np.asarray(anc["scaling"], np.float32).reshape(n, 3)[keep],
                                np.full((n_ins, 3), vox, np.float32)]),
        logodds=np.concatenate([l[keep], np.full(n_ins, l_new, np.float32)]),
        src=np.concatenate([keep.astype(np.int64), -1 - np.array(new_p[:n_ins], np.int64)]),
        n_kept=n_kept, n_inserted=n_ins, n_dropped=len(new_q) - n_ins,
        n_hit=int((obs == 1).sum()), n_miss=int((obs == 2).sum()))
    return out
