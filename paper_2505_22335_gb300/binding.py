"""Thin ctypes binding of the C ABI in include/ups.h.

Argument marshalling only: torch supplies device memory and the current CUDA
stream; every step of the render path runs in the CUDA library.  There is no
fallback: if libups.so has not been built (``build.build()``) or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_f, _i, _p, _ll = C.c_float, C.c_int, C.c_void_p, C.c_longlong

UPS_OK, UPS_PENDING = 0, 1
STATUS = {0: "OK", 1: "PENDING", 2: "ERR_ARG", 3: "ERR_OOM", 4: "ERR_CUDA", 5: "ERR_TIMEOUT",
          6: "ERR_CANCELLED", 7: "ERR_NONFINITE", 8: "ERR_CAPACITY", 9: "ERR_STATE"}
GRAD_POSE, GRAD_GAUSS, GRAD_MLP, GRAD_ANCHOR, GRAD_ALL = 1, 2, 4, 8, 15
MAX_VIEWS = 64


class Config(C.Structure):
    _fields_ = [("alpha_min", _f), ("alpha_max", _f), ("t_min", _f), ("dilation", _f),
                ("near_z", _f), ("guard", _f), ("n_feat", _i), ("k", _i), ("feat_dim", _i),
                ("hidden", _i), ("decode_bf16", _i), ("check_finite", _i), ("list_cap", _i),
                ("opacity_tanh", _i), ("decode_bwd_bf16", _i)]


class Camera(C.Structure):
    _fields_ = [("fx", _f), ("fy", _f), ("cx", _f), ("cy", _f), ("width", _i), ("height", _i),
                ("T_cw", _f * 16), ("t_norm", _f)]


class Gaussians(C.Structure):
    _fields_ = [("n", _i), ("per_view", _i), ("mean_opacity", _p), ("scale", _p), ("quat", _p),
                ("color", _p), ("feat", _p)]


class Images(C.Structure):
    _fields_ = [("color", _p), ("depth", _p), ("feat", _p), ("T", _p), ("n_contrib", _p)]


class ImageGrads(C.Structure):
    _fields_ = [("color", _p), ("depth", _p), ("feat", _p), ("T", _p)]


class Targets(C.Structure):
    _fields_ = [("color", _p), ("depth", _p), ("feat", _p), ("weight", _p)]


class ResidualCfg(C.Structure):
    _fields_ = [("lambda_color", _f), ("lambda_depth", _f), ("lambda_feat", _f), ("t_mask", _f)]


class LiftCfg(C.Structure):
    _fields_ = [("n_h", _i), ("patch", _i)]


class LiftMLP(C.Structure):
    _fields_ = [("w1", _p), ("b1", _p), ("w2", _p), ("b2", _p)]


class LossCfg(C.Structure):
    _fields_ = [("lambda_color", _f), ("lambda_depth", _f), ("lambda_feat", _f),
                ("lambda_scale", _f), ("l2", _i)]


class AnchorCfg(C.Structure):
    _fields_ = [("l_prior", _f), ("l_hit", _f), ("l_miss", _f), ("l_min", _f), ("l_max", _f), ("l_prune", _f),
                ("voxel", _f), ("margin", _f), ("near_z", _f)]


class AnchorResult(C.Structure):
    _fields_ = [("n_kept", _i), ("n_inserted", _i), ("n_dropped", _i), ("n_hit", _i), ("n_miss", _i)]


class Anchors(C.Structure):
    _fields_ = [("n", _i), ("pos", _p), ("feat", _p), ("offsets", _p), ("scaling", _p)]


class MLP(C.Structure):
    _fields_ = [("w1", _p), ("b1", _p), ("w2", _p), ("b2", _p)]


class Request(C.Structure):
    _fields_ = [("kind", _i), ("n_views", _i), ("levels", _i), ("cams", C.POINTER(Camera)),
                ("targets", Targets), ("loss", _p), ("d_pose", _p), ("d_mlp", MLP),
                ("d_anchors", Anchors)]


class ServerConfig(C.Structure):
    _fields_ = [("slots", _i), ("max_batch_views", _i), ("batching", _i),
                ("memory_budget_gb", C.c_double), ("loss", LossCfg)]


class Result(C.Structure):
    _fields_ = [("status", _i), ("submit_ms", C.c_double), ("start_ms", C.c_double),
                ("end_ms", C.c_double), ("batch_id", _i), ("batch_requests", _i),
                ("batch_views", _i)]


class Stats(C.Structure):
    _fields_ = [("n_views", _i), ("n_gaussian_views", _ll), ("n_visible", _ll),
                ("n_instances", _ll), ("n_tiles", _ll), ("n_pixels", _ll), ("key_bits", _i),
                ("n_listed", _ll), ("list_refills", _i)]


# every entry point of include/ups.h (checked by the CPU test suite)
EXPORTS = ["ups_config_default", "ups_version", "ups_create", "ups_destroy", "ups_last_error",
           "ups_decode_anchors", "ups_render_forward", "ups_loss_weighted", "ups_tracking_uncertainty",
           "ups_feature_lift", "ups_ssim_loss", "ups_uncertainty_mlp", "ups_anchor_cfg_default",
           "ups_anchor_update",
           "ups_render_backward", "ups_decode_backward", "ups_get_stats", "ups_copy_buffer",
           "ups_profile_enable", "ups_profile_read", "ups_render_forward_static",
           "ups_server_create", "ups_server_destroy", "ups_submit", "ups_poll", "ups_cancel",
           "ups_server_wait_idle", "ups_server_set_scene", "ups_server_last_error"]

_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load():
    """Load libups.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(path)
    L.ups_version.restype = C.c_char_p
    L.ups_last_error.restype = C.c_char_p
    L.ups_last_error.argtypes = [_p]
    L.ups_config_default.argtypes = [C.POINTER(Config)]
    L.ups_create.argtypes = [C.POINTER(Config), _i, C.POINTER(_p)]
    L.ups_destroy.argtypes = [_p]
    L.ups_decode_anchors.argtypes = [_p, C.POINTER(Anchors), C.POINTER(MLP), C.POINTER(Camera), _i,
                                     C.POINTER(Gaussians), _p]
    L.ups_render_forward.argtypes = [_p, C.POINTER(Gaussians), C.POINTER(Camera), _i,
                                     C.POINTER(Images), _p]
    L.ups_loss_weighted.argtypes = [_p, C.POINTER(Images), C.POINTER(Targets), C.POINTER(LossCfg),
                                    C.POINTER(Gaussians), _p, C.POINTER(Images), _p]
    L.ups_tracking_uncertainty.argtypes = [_p, C.POINTER(Images), C.POINTER(Targets), C.POINTER(ResidualCfg),
                                           _p, _p, _p, _p]
    L.ups_ssim_loss.argtypes = [_p, _p, _p, _p, _f, _p, _p, _p]
    L.ups_uncertainty_mlp.argtypes = [_p, C.POINTER(LiftCfg), _p, _p, C.POINTER(LiftMLP), _f, _f, _p,
                                      C.POINTER(LiftMLP), _p, _p, _p]
    L.ups_feature_lift.argtypes = [_p, C.POINTER(LiftCfg), _p, _p, C.POINTER(LiftMLP), _p, _f, _p,
                                   C.POINTER(LiftMLP), _p, _p]
    L.ups_anchor_cfg_default.argtypes = [C.POINTER(AnchorCfg)]
    L.ups_anchor_update.argtypes = [_p, C.POINTER(AnchorCfg), C.POINTER(Camera), _p, _p, C.POINTER(Anchors), _p,
                                    C.POINTER(Anchors), _p, _i, _p, C.POINTER(AnchorResult), _p]
    L.ups_render_backward.argtypes = [_p, C.POINTER(ImageGrads), C.c_uint, _f,
                                      C.POINTER(Gaussians), _p, _p]
    L.ups_decode_backward.argtypes = [_p, C.POINTER(Anchors), C.POINTER(MLP), C.POINTER(Camera), _i,
                                      C.POINTER(Gaussians), C.c_uint, C.POINTER(MLP),
                                      C.POINTER(Anchors), _p, _p]
    L.ups_get_stats.argtypes = [_p, C.POINTER(Stats)]
    L.ups_copy_buffer.argtypes = [_p, _i, _p, C.c_size_t, C.POINTER(C.c_size_t)]
    L.ups_profile_enable.argtypes = [_p, _i]
    L.ups_profile_read.argtypes = [_p, C.c_char_p, C.c_size_t, C.POINTER(_ll)]
    L.ups_render_forward_static.argtypes = [C.POINTER(Config), C.POINTER(Gaussians), C.POINTER(Camera),
                                            _i, C.POINTER(Images), _p]
    L.ups_server_create.argtypes = [C.POINTER(Config), C.POINTER(ServerConfig), _i, C.POINTER(Anchors),
                                    C.POINTER(MLP), C.POINTER(_p)]
    L.ups_server_destroy.argtypes = [_p]
    L.ups_submit.argtypes = [_p, C.POINTER(Request), C.POINTER(C.c_uint64)]
    L.ups_poll.argtypes = [_p, C.c_uint64, C.POINTER(Result)]
    L.ups_cancel.argtypes = [_p, C.c_uint64]
    L.ups_server_wait_idle.argtypes = [_p, C.c_double]
    L.ups_server_set_scene.argtypes = [_p, C.POINTER(Anchors), C.POINTER(MLP), C.c_double]
    L.ups_server_last_error.argtypes = [_p]
    L.ups_server_last_error.restype = C.c_char_p
    _lib = L
    return L


class UpsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_cameras(cams):
    """scenes.Camera list -> ctypes array of ups_camera."""
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        T = np.asarray(c.T_cw, dtype=np.float64).reshape(16)
        arr[i] = Camera(float(c.fx), float(c.fy), float(c.cx), float(c.cy), int(c.width),
                        int(c.height), (_f * 16)(*[float(x) for x in T]), float(c.t_norm))
    return arr


@dataclass
class GaussianSet:
    """Device tensors of a Gaussian set in the library layout ([sets, n, 4] float4 records)."""
    mean_opacity: "object"
    scale: "object"
    quat: "object"
    color: "object"
    feat: "object"
    per_view: bool

    @property
    def n(self):
        return int(self.mean_opacity.shape[1])

    def c(self):
        return Gaussians(self.n, int(self.per_view), _ptr(self.mean_opacity), _ptr(self.scale),
                         _ptr(self.quat), _ptr(self.color),
                         _ptr(self.feat) if self.feat is not None and self.feat.numel() else None)

    @staticmethod
    def empty(sets, n, n_feat, per_view, device="cuda"):
        import torch
        z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=device)
        return GaussianSet(z(sets, n, 4), z(sets, n, 4), z(sets, n, 4), z(sets, n, 4),
                           z(sets, n, max(n_feat, 0)), per_view)


class Renderer:
    """One library context (scratch memory + the saved forward state)."""

    def __init__(self, n_feat=16, k=10, device=0, **overrides):
        L = load()
        cfg = Config()
        L.ups_config_default(C.byref(cfg))
        cfg.n_feat = n_feat
        cfg.k = k
        for key, val in overrides.items():
            setattr(cfg, key, val)
        self.cfg = cfg
        h = _p()
        st = L.ups_create(C.byref(cfg), device, C.byref(h))
        if st != UPS_OK:
            raise UpsError(st, L.ups_last_error(None).decode())
        self._h = h
        self._L = L
        self.n_feat = n_feat
        self.k = k
        self._keep = []
        self.cams = None

    def close(self):
        if getattr(self, "_h", None):
            self._L.ups_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != UPS_OK:
            raise UpsError(st, self._L.ups_last_error(self._h).decode())

    # ---------------------------------------------------------------- decode
    def decode(self, anchors, mlp, cams, out: GaussianSet | None = None, stream=None):
        """anchors: dict pos [A,3], feat [A,32], offsets [A,K,3], scaling [A,3]; mlp: w1 b1 w2 b2."""
        A = int(anchors["pos"].shape[0])
        V = len(cams)
        if out is None:
            out = GaussianSet.empty(V, A * self.k, self.n_feat, True, anchors["pos"].device)
        ca = Anchors(A, _ptr(anchors["pos"]), _ptr(anchors["feat"]), _ptr(anchors["offsets"]),
                     _ptr(anchors["scaling"]))
        cm = MLP(_ptr(mlp["w1"]), _ptr(mlp["b1"]), _ptr(mlp["w2"]), _ptr(mlp["b2"]))
        cc = make_cameras(cams)
        og = out.c()
        self._check(self._L.ups_decode_anchors(self._h, C.byref(ca), C.byref(cm), cc, V,
                                               C.byref(og), _stream(stream)))
        return out

    def decode_backward(self, anchors, mlp, cams, dG: GaussianSet, mask=GRAD_ALL, d_mlp=None,
                        d_anchors=None, d_pose=None, stream=None):
        A = int(anchors["pos"].shape[0])
        ca = Anchors(A, _ptr(anchors["pos"]), _ptr(anchors["feat"]), _ptr(anchors["offsets"]),
                     _ptr(anchors["scaling"]))
        cm = MLP(_ptr(mlp["w1"]), _ptr(mlp["b1"]), _ptr(mlp["w2"]), _ptr(mlp["b2"]))
        dm = MLP(*[_ptr(d_mlp[k]) for k in ("w1", "b1", "w2", "b2")]) if d_mlp else MLP()
        da = (Anchors(A, *[_ptr(d_anchors[k]) for k in ("pos", "feat", "offsets", "scaling")])
              if d_anchors else Anchors())
        cc = make_cameras(cams)
        dg = dG.c()
        self._check(self._L.ups_decode_backward(self._h, C.byref(ca), C.byref(cm), cc, len(cams),
                                                C.byref(dg), mask, C.byref(dm), C.byref(da),
                                                _ptr(d_pose), _stream(stream)))

    # --------------------------------------------------------------- forward
    def alloc_images(self, cams, device="cuda"):
        import torch
        P = sum(c.width * c.height for c in cams)
        z = lambda n: torch.zeros(n, dtype=torch.float32, device=device)
        return dict(color=z(3 * P), depth=z(P), feat=z(max(self.n_feat, 0) * P), T=z(P),
                    n_contrib=torch.zeros(P, dtype=torch.int32, device=device))

    def forward(self, g: GaussianSet, cams, out=None, stream=None):
        out = out if out is not None else self.alloc_images(cams, g.mean_opacity.device)
        ci = Images(_ptr(out["color"]), _ptr(out["depth"]),
                    _ptr(out["feat"]) if self.n_feat else None, _ptr(out["T"]),
                    _ptr(out["n_contrib"]))
        cg = g.c()
        cc = make_cameras(cams)
        self._check(self._L.ups_render_forward(self._h, C.byref(cg), cc, len(cams), C.byref(ci),
                                               _stream(stream)))
        self._keep = [g, out]
        self.cams = cams
        return out

    def loss(self, img, tgt, lambda_color=1.0, lambda_depth=1.0, lambda_feat=1.0,
             lambda_scale=0.0, l2=False, g: GaussianSet | None = None, loss_out=None,
             grad_out=None, stream=None):
        import torch
        dev = img["color"].device
        loss_out = loss_out if loss_out is not None else torch.zeros(1, dtype=torch.float32, device=dev)
        if grad_out is None:
            grad_out = dict(color=torch.empty_like(img["color"]), depth=torch.empty_like(img["depth"]),
                            feat=torch.empty_like(img["feat"]))
        ci = Images(_ptr(img["color"]), _ptr(img["depth"]), _ptr(img["feat"]) if self.n_feat else None,
                    None, None)
        ct = Targets(_ptr(tgt["color"]), _ptr(tgt["depth"]),
                     _ptr(tgt["feat"]) if self.n_feat else None, _ptr(tgt.get("weight")))
        cl = LossCfg(lambda_color, lambda_depth, lambda_feat, lambda_scale, int(l2))
        cd = Images(_ptr(grad_out["color"]), _ptr(grad_out["depth"]),
                    _ptr(grad_out["feat"]) if self.n_feat else None, None, None)
        cg = g.c() if g is not None else None
        self._check(self._L.ups_loss_weighted(self._h, C.byref(ci), C.byref(ct), C.byref(cl),
                                              C.byref(cg) if cg is not None else None,
                                              _ptr(loss_out), C.byref(cd), _stream(stream)))
        return loss_out, grad_out

    def tracking_uncertainty(self, img, tgt, lambda_color=0.25, lambda_depth=0.7, lambda_feat=0.1, t_mask=0.1,
                             out=None, stream=None):
        """Eq. 6 residual R, Eq. 15 sigma^2 = 2R and the motion mask R > 1/4 of the
        last forward's images (dict with color, depth, feat, T) against tgt."""
        import torch
        dev = img["depth"].device
        if out is None:
            out = dict(R=torch.empty_like(img["depth"]), sigma2=torch.empty_like(img["depth"]),
                       motion=torch.empty(img["depth"].shape, dtype=torch.uint8, device=dev))
        ci = Images(_ptr(img["color"]), _ptr(img["depth"]), _ptr(img["feat"]) if self.n_feat else None,
                    _ptr(img["T"]), None)
        ct = Targets(_ptr(tgt["color"]), _ptr(tgt["depth"]), _ptr(tgt["feat"]) if self.n_feat else None, None)
        rc = ResidualCfg(lambda_color, lambda_depth, lambda_feat, t_mask)
        self._check(self._L.ups_tracking_uncertainty(self._h, C.byref(ci), C.byref(ct), C.byref(rc),
                                                     _ptr(out.get("R")), _ptr(out.get("sigma2")),
                                                     _ptr(out.get("motion")), _stream(stream)))
        return out

    def uncertainty_mlp(self, dino, R, mlp, n_h=384, patch=14, lam=1.0, scale=1.0, d_mlp=None, out=None,
                        loss_out=None, stream=None):
        """Eq. 5 / Eq. 13: sigma = F_u(F) per pixel, scale * L_u and (if d_mlp) its
        gradient into F_u; returns (loss, dict(sigma, motion))."""
        import torch
        dev = R.device
        loss_out = loss_out if loss_out is not None else torch.zeros(1, dtype=torch.float32, device=dev)
        if out is None:
            out = dict(sigma=torch.empty_like(R), motion=torch.empty(R.shape, dtype=torch.uint8, device=dev))
        cm = LiftMLP(*(_ptr(mlp[k]) for k in ("w1", "b1", "w2", "b2")))
        dm = LiftMLP(*(_ptr(d_mlp.get(k)) for k in ("w1", "b1", "w2", "b2"))) if d_mlp is not None else None
        self._check(self._L.ups_uncertainty_mlp(self._h, C.byref(LiftCfg(n_h, patch)), _ptr(dino), _ptr(R),
                                                C.byref(cm), float(lam), float(scale), _ptr(loss_out),
                                                C.byref(dm) if dm is not None else None, _ptr(out.get("sigma")),
                                                _ptr(out.get("motion")), _stream(stream)))
        return loss_out, out

    def ssim_loss(self, color, t_color, scale=1.0, d_color=None, weight=None, loss_out=None, stream=None):
        """Eq. 4's D-SSIM term scale * (1 - SSIM) of the last forward's views (each
        pixel weighted by `weight` when given); scale * d/dC~ is added to d_color."""
        import torch
        loss_out = loss_out if loss_out is not None else torch.zeros(1, dtype=torch.float32, device=color.device)
        self._check(self._L.ups_ssim_loss(self._h, _ptr(color), _ptr(t_color), _ptr(weight), float(scale),
                                          _ptr(loss_out), _ptr(d_color), _stream(stream)))
        return loss_out

    def feature_lift(self, feat, dino, mlp, n_h=384, patch=14, scale=1.0, d_mlp=None, d_feat=None, weight=None,
                     loss_out=None, stream=None):
        """Eq. 11-12: scale * L_d of the rendered feature map `feat` (image layout)
        against the per-view DINO patch grids `dino` (concatenated [hp][wp][n_h]);
        mlp / d_mlp: dicts w1, b1, w2, b2 (d_mlp and d_feat are accumulated)."""
        import torch
        loss_out = loss_out if loss_out is not None else torch.zeros(1, dtype=torch.float32, device=feat.device)
        cm = LiftMLP(*(_ptr(mlp[k]) for k in ("w1", "b1", "w2", "b2")))
        dm = LiftMLP(*(_ptr(d_mlp.get(k)) for k in ("w1", "b1", "w2", "b2"))) if d_mlp is not None else None
        self._check(self._L.ups_feature_lift(self._h, C.byref(LiftCfg(n_h, patch)), _ptr(feat), _ptr(dino),
                                             C.byref(cm), _ptr(weight), float(scale), _ptr(loss_out),
                                             C.byref(dm) if dm is not None else None, _ptr(d_feat),
                                             _stream(stream)))
        return loss_out

    def anchor_update(self, anchors, logodds, cam, depth, motion=None, capacity=None, stream=None, **cfg):
        """Eq. 7 on one keyframe: update, prune and insert anchors (dicts of device
        tensors pos [n,3], feat [n,F], offsets [n,K,3], scaling [n,3]; logodds [n]).
        cfg overrides fields of ups_anchor_cfg.  Returns (anchors, logodds, src_index,
        counts) with the outputs cut to the new anchor count."""
        import torch
        n = int(anchors["pos"].shape[0])
        cap = n if capacity is None else int(capacity)
        dev = anchors["pos"].device
        F = int(anchors["feat"].shape[1])
        K = int(anchors["offsets"].shape[1])
        if F != self.cfg.feat_dim or K != self.k:
            raise ValueError(f"anchors have feat width {F} and k {K}; the context has {self.cfg.feat_dim} and {self.k}")
        z = lambda *sh: torch.empty(*sh, dtype=torch.float32, device=dev)
        out = dict(pos=z(cap, 3), feat=z(cap, F), offsets=z(cap, K, 3), scaling=z(cap, 3))
        lout = z(cap)
        src = torch.empty(cap, dtype=torch.int32, device=dev)
        ac = AnchorCfg()
        self._L.ups_anchor_cfg_default(C.byref(ac))
        for key, val in cfg.items():
            setattr(ac, key, float(val))
        ca = Anchors(n, *(_ptr(anchors[k]) for k in ("pos", "feat", "offsets", "scaling")))
        co = Anchors(cap, *(_ptr(out[k]) for k in ("pos", "feat", "offsets", "scaling")))
        res = AnchorResult()
        self._check(self._L.ups_anchor_update(self._h, C.byref(ac), make_cameras([cam]), _ptr(depth), _ptr(motion),
                                              C.byref(ca), _ptr(logodds), C.byref(co), _ptr(lout), cap, _ptr(src),
                                              C.byref(res), _stream(stream)))
        m = co.n
        return ({k: v[:m] for k, v in out.items()}, lout[:m], src[:m],
                {k: getattr(res, k) for k, _ in AnchorResult._fields_})

    # -------------------------------------------------------------- backward
    def backward(self, dL, mask=GRAD_POSE | GRAD_GAUSS, scale_grad=0.0, grad: GaussianSet | None = None,
                 d_pose=None, stream=None):
        import torch
        g = self._keep[0]
        dev = g.mean_opacity.device
        V = len(self.cams)
        if (mask & GRAD_GAUSS) and grad is None:
            sets = V if g.per_view else 1
            grad = GaussianSet.empty(sets, g.n, self.n_feat, g.per_view, dev)
        if (mask & GRAD_POSE) and d_pose is None:
            d_pose = torch.zeros(V, 6, dtype=torch.float32, device=dev)
        cd = ImageGrads(_ptr(dL.get("color")), _ptr(dL.get("depth")),
                        _ptr(dL.get("feat")) if self.n_feat else None, _ptr(dL.get("T")))
        cg = grad.c() if grad is not None else None
        self._check(self._L.ups_render_backward(self._h, C.byref(cd), mask, float(scale_grad),
                                                C.byref(cg) if cg is not None else None,
                                                _ptr(d_pose), _stream(stream)))
        return grad, d_pose

    # ------------------------------------------------------------ inspection
    def stats(self):
        s = Stats()
        self._check(self._L.ups_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def profile(self, on=True):
        self._check(self._L.ups_profile_enable(self._h, int(on)))

    def profile_read(self):
        """-> ({stage: (total_ms, calls)}, kernel launches since the last read)."""
        import json
        buf = C.create_string_buffer(8192)
        n = _ll(0)
        self._check(self._L.ups_profile_read(self._h, buf, len(buf), C.byref(n)))
        return {k: tuple(v) for k, v in json.loads(buf.value.decode()).items()}, int(n.value)

    def copy_buffer(self, which):
        size = C.c_size_t(0)
        self._check(self._L.ups_copy_buffer(self._h, which, None, 0, C.byref(size)))
        dtype = {0: np.uint32, 1: np.uint32, 2: np.uint32, 3: np.float32, 4: np.float32,
                 5: np.uint32, 6: np.float32}[which]
        arr = np.zeros(size.value // 4, dtype=dtype)
        if size.value:
            self._check(self._L.ups_copy_buffer(self._h, which, arr.ctypes.data_as(_p), size.value,
                                                None))
        return arr


def render_forward_static(g: GaussianSet, cams, out, n_feat, stream=None, **overrides):
    """Allocation-free forward (no context): scratch lives in a static device
    array of the library; `out` must be preallocated (see Renderer.alloc_images)."""
    L = load()
    cfg = Config()
    L.ups_config_default(C.byref(cfg))
    cfg.n_feat = n_feat
    for key, val in overrides.items():
        setattr(cfg, key, val)
    ci = Images(_ptr(out["color"]), _ptr(out["depth"]), _ptr(out["feat"]) if n_feat else None,
                _ptr(out["T"]), _ptr(out["n_contrib"]))
    cg = g.c()
    cc = make_cameras(cams)
    st = L.ups_render_forward_static(C.byref(cfg), C.byref(cg), cc, len(cams), C.byref(ci),
                                     _stream(stream))
    if st != UPS_OK:
        raise UpsError(st, L.ups_last_error(None).decode())
    return out


TRACK, MAP = 0, 1


class Server:
    """Request queue with continuous batching over a resident anchor scene."""

    def __init__(self, anchors, mlp, n_feat=16, k=10, slots=2, max_batch_views=16, batching=True,
                 memory_budget_gb=64.0, device=0, loss=None, **overrides):
        L = load()
        cfg = Config()
        L.ups_config_default(C.byref(cfg))
        cfg.n_feat = n_feat
        cfg.k = k
        for key, val in overrides.items():
            setattr(cfg, key, val)
        lc = loss or {}
        sc = ServerConfig(slots, max_batch_views, int(batching), memory_budget_gb,
                          LossCfg(lc.get("lambda_color", 1.0), lc.get("lambda_depth", 1.0),
                                  lc.get("lambda_feat", 1.0), 0.0, int(lc.get("l2", False))))
        self._keep = (anchors, mlp)
        A = int(anchors["pos"].shape[0])
        ca = Anchors(A, _ptr(anchors["pos"]), _ptr(anchors["feat"]), _ptr(anchors["offsets"]),
                     _ptr(anchors["scaling"]))
        cm = MLP(_ptr(mlp["w1"]), _ptr(mlp["b1"]), _ptr(mlp["w2"]), _ptr(mlp["b2"]))
        h = _p()
        st = L.ups_server_create(C.byref(cfg), C.byref(sc), device, C.byref(ca), C.byref(cm), C.byref(h))
        if st != UPS_OK:
            raise UpsError(st, "ups_server_create failed: " + L.ups_last_error(None).decode())
        self._h, self._L = h, L
        self.n_feat, self.k, self.A = n_feat, k, A
        self._live = {}

    def submit(self, kind, cams, targets, loss, d_pose, d_mlp=None, d_anchors=None, levels=3):
        """targets: dict of device tensors (colour, depth, feature, weight) of the request's views."""
        cc = make_cameras(cams)
        req = Request(kind, len(cams), levels, cc,
                      Targets(_ptr(targets["color"]), _ptr(targets["depth"]),
                              _ptr(targets.get("feat")) if self.n_feat else None,
                              _ptr(targets.get("weight"))),
                      _ptr(loss), _ptr(d_pose),
                      MLP(*[_ptr(d_mlp[k]) for k in ("w1", "b1", "w2", "b2")]) if d_mlp else MLP(),
                      Anchors(self.A, *[_ptr(d_anchors[k]) for k in ("pos", "feat", "offsets", "scaling")])
                      if d_anchors else Anchors())
        t = C.c_uint64(0)
        st = self._L.ups_submit(self._h, C.byref(req), C.byref(t))
        if st != UPS_OK:
            raise UpsError(st, "ups_submit rejected the request")
        self._live[t.value] = (targets, loss, d_pose, d_mlp, d_anchors)
        return t.value

    def poll(self, ticket):
        """-> None while pending, else a dict (status, times in ms, batch info)."""
        r = Result()
        st = self._L.ups_poll(self._h, ticket, C.byref(r))
        if st == UPS_PENDING:
            return None
        if st != UPS_OK:
            raise UpsError(st, "unknown ticket")
        self._live.pop(ticket, None)
        return {k: getattr(r, k) for k, _ in Result._fields_}

    def cancel(self, ticket):
        return self._L.ups_cancel(self._h, ticket)

    def wait(self, ticket, timeout_s=120.0):
        import time
        t_end = time.time() + timeout_s
        while True:
            res = self.poll(ticket)
            if res is not None:
                return res
            if time.time() > t_end:
                raise UpsError(5, "request did not finish in time")
            time.sleep(0.0005)

    def wait_idle(self, timeout_s=120.0):
        st = self._L.ups_server_wait_idle(self._h, timeout_s * 1e3)
        if st != UPS_OK:
            raise UpsError(st, "server did not drain in time")

    def set_scene(self, anchors, mlp, timeout_s=120.0):
        """Swap the resident scene (e.g. after ups_anchor_update changed the anchors)."""
        A = int(anchors["pos"].shape[0])
        ca = Anchors(A, _ptr(anchors["pos"]), _ptr(anchors["feat"]), _ptr(anchors["offsets"]),
                     _ptr(anchors["scaling"]))
        cm = MLP(_ptr(mlp["w1"]), _ptr(mlp["b1"]), _ptr(mlp["w2"]), _ptr(mlp["b2"]))
        st = self._L.ups_server_set_scene(self._h, C.byref(ca), C.byref(cm), timeout_s * 1e3)
        if st != UPS_OK:
            raise UpsError(st, "ups_server_set_scene failed")
        self._keep = (anchors, mlp)
        self.A = A

    def last_error(self):
        return self._L.ups_server_last_error(self._h).decode()

    def close(self):
        if getattr(self, "_h", None):
            self._L.ups_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return load().ups_version().decode()


# ----------------------------------------------------------------------------
# conversions from the seeded numpy scenes
# ----------------------------------------------------------------------------

def to_set(g, device="cuda", per_view=False):
    """numpy Gaussians (mean, scale, quat, opacity, color, feat) -> GaussianSet with 1 set
    (or a list/array of V such dicts when per_view)."""
    import torch

    def one(gg):
        n = gg["mean"].shape[0]
        mo = np.concatenate([gg["mean"], gg["opacity"].reshape(n, 1)], 1)
        sc = np.concatenate([gg["scale"], np.zeros((n, 1))], 1)
        co = np.concatenate([gg["color"], np.zeros((n, 1))], 1)
        return mo, sc, gg["quat"], co, gg["feat"]

    parts = [one(gg) for gg in (g if per_view else [g])]
    t = lambda k: torch.tensor(np.stack([p[k] for p in parts]), dtype=torch.float32, device=device).contiguous()
    return GaussianSet(t(0), t(1), t(2), t(3), t(4), per_view)


def anchors_to_device(anc, mlp, device="cuda"):
    import torch
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
    return ({k: t(anc[k]) for k in ("pos", "feat", "offsets", "scaling")},
            {k: t(mlp[k]) for k in ("w1", "b1", "w2", "b2")})


def targets_to_device(tgts, device="cuda"):
    import torch
    cat = lambda k: torch.tensor(np.concatenate([t[k].reshape(-1) for t in tgts]),
                                 dtype=torch.float32, device=device)
    return dict(color=cat("color"), depth=cat("depth"), feat=cat("feat"), weight=cat("weight"))
