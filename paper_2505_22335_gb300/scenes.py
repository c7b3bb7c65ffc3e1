"""Seeded synthetic inputs shaped like the paper's RGB-D SLAM workloads.

This module only draws random numbers and builds camera poses; it holds none
of the render arithmetic, so both the CUDA path and the FP64 oracle may use it.

Shapes follow the experiments section (640x480 TUM/Bonn/ScanNet frames,
1280x720 MoCap frames); the datasets themselves are not used, synthetic scenes
stand in for them:

* plain Gaussians (Eq. 1): means uniform in a 2 m cube centred 2.5 m in front
  of the identity camera, log-uniform scales in [0.005, 0.05] m, random unit
  quaternions, opacity sigmoid(N(0,1)), colours uniform [0,1];
* anchors (Sec. 3.3, "Adaptively Structured Gaussian"): positions in the same
  cube, 32-d features N(0, 0.1^2), K offsets N(0, 0.05^2) m, per-anchor scaling
  log-uniform in [0.01, 0.1];
* MLP weights (Eq. 8-9): Kaiming-uniform from a seed, zero biases;
* keyframe poses on a 3 m arc (radius 2.5 m about the cube centre, +-30 deg),
  jittered by 0.3 m and 10 deg;
* keyframes for the probabilistic anchor map (Eq. 7): a tilted, bumpy depth
  surface 1.5-4 m away with 5 % of the pixels missing, a moving object (a disc
  0.4-0.8 m nearer) marked in the motion mask, and anchors seen from that
  keyframe: half on the surface (depth +- 3 cm), a fifth in the free space in
  front of it, the rest hidden behind it or anywhere in a 6 m box.

All arrays are float64 numpy; callers cast to float32 for the GPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

CUBE_CENTRE = np.array([0.0, 0.0, 2.5])
CUBE_HALF = 1.0


@dataclass
class Camera:
    """Pinhole intrinsics plus the world-to-camera pose T_cw (row-major 4x4)."""
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    T_cw: np.ndarray = field(default_factory=lambda: np.eye(4))
    t_norm: float = 0.5

    def scaled(self, factor: float) -> "Camera":
        """The same pose with intrinsics and resolution scaled (pyramid level)."""
        return Camera(self.fx * factor, self.fy * factor, self.cx * factor,
                      self.cy * factor, int(round(self.width * factor)),
                      int(round(self.height * factor)), self.T_cw.copy(),
                      self.t_norm)


def _rng(seed):
    return np.random.default_rng(seed)


def random_quaternions(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def plain_gaussians(seed: int, n: int, n_feat: int = 0, *, scale_lo=0.005,
                    scale_hi=0.05, half=CUBE_HALF, centre=CUBE_CENTRE):
    """Gaussians given directly (no decode): the plain 3DGS workload."""
    rng = _rng(seed)
    mean = centre + rng.uniform(-half, half, size=(n, 3))
    scale = np.exp(rng.uniform(math.log(scale_lo), math.log(scale_hi), size=(n, 3)))
    quat = random_quaternions(rng, n)
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(size=n)))
    color = rng.uniform(0.0, 1.0, size=(n, 3))
    feat = rng.normal(size=(n, n_feat)) if n_feat else np.zeros((n, 0))
    return dict(mean=mean, scale=scale, quat=quat, opacity=opacity,
                color=color, feat=feat)


def anchors(seed: int, n_anchor: int, k: int, feat_dim: int = 32, *,
            half=CUBE_HALF, centre=CUBE_CENTRE, offset_sigma=0.05,
            feat_sigma=0.1, scaling_lo=0.01, scaling_hi=0.1):
    """Anchor state: position x_v, feature f_v, K offsets, per-anchor scaling."""
    rng = _rng(seed)
    pos = centre + rng.uniform(-half, half, size=(n_anchor, 3))
    feat = rng.normal(0.0, feat_sigma, size=(n_anchor, feat_dim))
    offsets = rng.normal(0.0, offset_sigma, size=(n_anchor, k, 3))
    scaling = np.exp(rng.uniform(math.log(scaling_lo), math.log(scaling_hi),
                                 size=(n_anchor, 3)))
    return dict(pos=pos, feat=feat, offsets=offsets, scaling=scaling)


def mlp_weights(seed: int, k: int, n_feat: int, feat_dim: int = 32,
                hidden: int = 32, bias_sigma: float = 0.0):
    """Weights of the four decode MLPs, Kaiming-uniform with zero biases.

    Layout: W1 is [4*hidden, feat_dim+6] (hidden blocks: opacity, covariance,
    colour, feature); W2 is [K*(11+n_feat), hidden] with output rows grouped as
    opacity (K), covariance (7K: 3 scale + 4 quaternion per Gaussian), colour
    (3K) and feature (K*n_feat); row group g reads hidden block g only.
    """
    rng = _rng(seed)
    d_in = feat_dim + 6
    n_out = k * (11 + n_feat)
    w1 = rng.uniform(-1.0, 1.0, size=(4 * hidden, d_in)) * math.sqrt(6.0 / d_in)
    w2 = rng.uniform(-1.0, 1.0, size=(n_out, hidden)) * math.sqrt(6.0 / hidden)
    b1 = rng.normal(0.0, bias_sigma, size=4 * hidden) if bias_sigma > 0 else np.zeros(4 * hidden)
    b2 = rng.normal(0.0, bias_sigma, size=n_out) if bias_sigma > 0 else np.zeros(n_out)
    return dict(w1=w1, b1=b1, w2=w2, b2=b2)


def _rot(axis, angle):
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis)
    x, y, z = axis
    c, s = math.cos(angle), math.sin(angle)
    C = 1 - c
    return np.array([[c + x * x * C, x * y * C - z * s, x * z * C + y * s],
                     [y * x * C + z * s, c + y * y * C, y * z * C - x * s],
                     [z * x * C - y * s, z * y * C + x * s, c + z * z * C]])


def look_at(position, target):
    """T_cw for a camera at `position` looking at `target` (x right, y down)."""
    fwd = np.asarray(target, float) - np.asarray(position, float)
    fwd /= np.linalg.norm(fwd)
    down_hint = np.array([0.0, 1.0, 0.0])
    right = np.cross(down_hint, fwd)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R_wc = np.stack([right, down, fwd], axis=1)
    T = np.eye(4)
    T[:3, :3] = R_wc.T
    T[:3, 3] = -R_wc.T @ np.asarray(position, float)
    return T


def arc_poses(seed: int, n_views: int, *, radius=2.5, span_deg=30.0,
              jitter_t=0.3, jitter_deg=10.0, centre=CUBE_CENTRE):
    """Keyframe poses on an arc about the cube centre, jittered."""
    rng = _rng(seed)
    poses = []
    for i in range(n_views):
        th = math.radians(-span_deg + 2 * span_deg * (i + 0.5) / n_views)
        pos = centre + radius * np.array([math.sin(th), 0.0, -math.cos(th)])
        # uniform point in a ball of radius jitter_t
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        pos = pos + d * jitter_t * rng.uniform() ** (1.0 / 3.0)
        T = look_at(pos, centre)
        axis = rng.normal(size=3)
        ang = math.radians(rng.uniform(0.0, jitter_deg))
        R_wc = T[:3, :3].T @ _rot(axis, ang)
        T2 = np.eye(4)
        T2[:3, :3] = R_wc.T
        T2[:3, 3] = -R_wc.T @ pos
        poses.append(T2)
    return poses


def cameras(seed: int, n_views: int, width: int, height: int, fx: float,
            fy: float | None = None, *, identity: bool = False,
            t_norm: float = 0.5):
    fy = fx if fy is None else fy
    if identity:
        poses = [np.eye(4) for _ in range(n_views)]
    else:
        poses = arc_poses(seed, n_views)
    return [Camera(fx, fy, width / 2.0, height / 2.0, width, height, T, t_norm)
            for T in poses]


def targets(seed: int, cams, n_feat: int, *, weighted: bool,
            depth_lo=1.5, depth_hi=3.5):
    """Per-view target colour/depth/feature images and per-pixel weights."""
    rng = _rng(seed)
    out = []
    for cam in cams:
        h, w = cam.height, cam.width
        out.append(dict(
            color=rng.uniform(0.0, 1.0, size=(3, h, w)),
            depth=rng.uniform(depth_lo, depth_hi, size=(h, w)),
            feat=rng.normal(size=(n_feat, h, w)),
            weight=(rng.uniform(0.0, 1.0, size=(h, w)) if weighted
                    else np.ones((h, w)))))
    return out


# ----------------------------------------------------------------------------
# Named workloads (sizes of the five benchmark configurations)
# ----------------------------------------------------------------------------

def workload_plain_2k(seed=0):
    """2,000 plain Gaussians, one 160x120 view, identity pose, RGB+depth."""
    g = plain_gaussians(seed, 2000, 0)
    cams = cameras(seed, 1, 160, 120, 150.0, identity=True)
    return g, cams


def workload_anchor(seed, n_anchor, k, n_feat, n_views, width, height, fx,
                    identity=False):
    a = anchors(seed, n_anchor, k)
    m = mlp_weights(seed + 1000, k, n_feat)
    cams = cameras(seed, n_views, width, height, fx, identity=identity)
    return a, m, cams


def keyframe(seed: int, cam: Camera, *, hole_frac=0.05):
    """Depth map [H, W] (0 = missing) and motion mask [H, W] uint8 of one keyframe."""
    rng = _rng(seed)
    H, W = cam.height, cam.width
    yy, xx = np.mgrid[0:H, 0:W] / max(H, W)
    a, b, c = rng.uniform(1.0, 1.5, 3)
    depth = 1.5 + a * xx + 0.5 * b * yy + 0.3 * np.sin(6.0 * c * xx) * np.cos(4.0 * yy)
    depth = np.clip(depth + rng.uniform(0.0, 0.01, (H, W)), 1.5, 4.0)
    cx, cy, r = rng.uniform(0.3, 0.7) * W, rng.uniform(0.3, 0.7) * H, rng.uniform(0.08, 0.15) * max(H, W)
    jj, ii = np.mgrid[0:H, 0:W]
    disc = (ii - cx) ** 2 + (jj - cy) ** 2 < r * r
    depth[disc] -= rng.uniform(0.4, 0.8)
    depth[rng.uniform(size=(H, W)) < hole_frac] = 0.0
    return depth, disc.astype(np.uint8)


def anchor_cloud(seed: int, cam: Camera, depth, n: int, k: int, feat_dim: int = 32):
    """n anchors around the keyframe's surface (positions from the inverse pose,
    float64), with features, offsets, scalings and log-odds U(-2.5, 3.5)."""
    rng = _rng(seed)
    H, W = depth.shape
    T_wc = np.linalg.inv(np.asarray(cam.T_cw, float))
    kind = rng.choice(4, size=n, p=[0.5, 0.2, 0.15, 0.15])
    i = rng.uniform(-0.5, W - 0.5, n)
    j = rng.uniform(-0.5, H - 0.5, n)
    d = depth[np.clip(np.rint(j), 0, H - 1).astype(int), np.clip(np.rint(i), 0, W - 1).astype(int)]
    d = np.where(d > 0, d, 2.5)
    z = np.where(kind == 0, d + rng.uniform(-0.03, 0.03, n),
                 np.where(kind == 1, d * rng.uniform(0.3, 0.9, n), d * rng.uniform(1.1, 1.5, n)))
    Xc = np.stack([(i - cam.cx) / cam.fx * z, (j - cam.cy) / cam.fy * z, z, np.ones(n)])
    pos = (T_wc @ Xc)[:3].T
    box = T_wc[:3, 3] + rng.uniform(-3.0, 3.0, (n, 3))
    pos = np.where((kind == 3)[:, None], box, pos)
    return dict(pos=pos, feat=rng.normal(0.0, 0.1, (n, feat_dim)), offsets=rng.normal(0.0, 0.05, (n, k, 3)),
                scaling=np.exp(rng.uniform(np.log(0.01), np.log(0.1), (n, 3)))), rng.uniform(-2.5, 3.5, n)
