"""Probabilistic anchor update on the GPU (Sec. 3.3, Eq. 7) against the oracle:
both take every decision (pixel of an anchor, hit / miss, voxel of a pixel) in
FP32 with one rounding per operation in the same order, and the rest is copies
and counters, so every output is compared bit for bit: the kept rows and their
order, the log-odds, the inserted anchors, their raster order and the counts."""
import numpy as np
import pytest

import oracle
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu

FIELDS = ("pos", "feat", "offsets", "scaling")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def f32(cam):
    """Camera with intrinsics already in FP32 (the library receives floats)."""
    return scenes.Camera(*(float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy)), cam.width, cam.height,
                         np.asarray(cam.T_cw, np.float32).astype(np.float64), cam.t_norm)


def same(got, ref, what):
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    bad = np.nonzero((got != ref).reshape(len(got), -1).any(axis=1))[0] if len(got) else []
    assert len(bad) == 0, (what, len(bad), bad[:5], got[bad[:3]], ref[bad[:3]])


def run(R, anc, l, cam, depth, motion, capacity, **cfg):
    import torch
    dev = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    ga = {k: dev(anc[k]) for k in FIELDS}
    out, lo, src, cnt = R.anchor_update(ga, dev(l), cam, dev(depth), None if motion is None else dev(motion, torch.uint8),
                                        capacity=capacity, **cfg)
    ref = oracle.anchor_update(anc, l, cam, depth, motion, oracle.AnchorCfg(**cfg), capacity)
    for k in ("n_kept", "n_inserted", "n_dropped", "n_hit", "n_miss"):
        assert cnt[k] == ref[k], (k, cnt[k], ref[k])
    same(src.cpu().numpy(), ref["src"], "src")
    for k in FIELDS:
        same(out[k].cpu().numpy().view(np.uint32), ref[k].view(np.uint32), k)
    same(lo.cpu().numpy().view(np.uint32), ref["logodds"].view(np.uint32), "logodds")
    return {k: out[k].cpu().numpy() for k in FIELDS}, lo.cpu().numpy(), ref


def case(seed, W, H, n, k=4, fx=None):
    cam = f32(scenes.cameras(seed, 1, W, H, fx or 0.9 * W)[0])
    depth, motion = scenes.keyframe(seed, cam)
    anc, l = scenes.anchor_cloud(seed + 1, cam, depth, n, k)
    return cam, {kk: v.astype(np.float32) for kk, v in anc.items()}, l.astype(np.float32), \
        depth.astype(np.float32), motion


def cfg32(**kw):
    """ups_anchor_cfg fields rounded to FP32 the way the library stores them."""
    c = oracle.AnchorCfg(**kw)
    return {f: float(np.float32(getattr(c, f))) for f in c.__dataclass_fields__}


@pytest.mark.parametrize("W,H,n", [(61, 45, 700), (200, 150, 3000)])
def test_ragged_keyframes(W, H, n):
    cam, anc, l, depth, motion = case(W + n, W, H, n)
    R = B.Renderer(n_feat=16, k=4)
    _, _, ref = run(R, anc, l, cam, depth, motion, capacity=n + W * H, **cfg32(voxel=0.02))
    assert ref["n_inserted"] > 50 and ref["n_hit"] > 0 and ref["n_miss"] > 0 and ref["n_kept"] < n


def test_full_keyframe_640x480_100k_anchors():
    cam, anc, l, depth, motion = case(11, 640, 480, 100_000, k=10, fx=600.0)
    R = B.Renderer(n_feat=16, k=10)
    _, _, ref = run(R, anc, l, cam, depth, motion, capacity=200_000, **cfg32())
    assert ref["n_hit"] > 10_000 and ref["n_inserted"] > 0


def test_capacity_motion_none_and_empty_input():
    cam, anc, l, depth, motion = case(5, 96, 64, 400)
    R = B.Renderer(n_feat=16, k=4)
    c = cfg32(voxel=0.02)
    _, _, ref = run(R, anc, l, cam, depth, motion, capacity=400, **c)       # only the pruned rows are free
    assert ref["n_kept"] + ref["n_inserted"] == 400 and ref["n_dropped"] > 0
    _, _, ref2 = run(R, anc, l, cam, depth, None, capacity=407, **c)        # all static: more anchors kept
    assert ref2["n_kept"] > ref["n_kept"] and ref2["n_kept"] + ref2["n_inserted"] == 407
    empty = {k: v[:0] for k, v in anc.items()}
    _, _, ref = run(R, empty, l[:0], cam, depth, motion, capacity=96 * 64, **c)   # insertion only
    assert ref["n_kept"] == 0 and ref["n_inserted"] > 100
    _, _, ref = run(R, anc, l, cam, np.zeros_like(depth), motion, capacity=400, **c)  # nothing observed
    assert ref["n_hit"] == ref["n_miss"] == ref["n_inserted"] == 0


def test_keyframe_sequence_stays_bit_exact():
    cams = [f32(c) for c in scenes.cameras(21, 3, 160, 120, 150.0)]
    R = B.Renderer(n_feat=16, k=4)
    depth0, _ = scenes.keyframe(21, cams[0])
    anc, l = scenes.anchor_cloud(22, cams[0], depth0, 1500, 4)
    anc = {k: v.astype(np.float32) for k, v in anc.items()}
    l = l.astype(np.float32)
    for t, cam in enumerate(cams * 2):
        depth, motion = scenes.keyframe(30 + t, cam)
        anc, l, _ = run(R, anc, l, cam, depth.astype(np.float32), motion, capacity=len(l) + 4000,
                        **cfg32(voxel=0.03))


def test_rejects_bad_arguments():
    import torch
    cam, anc, l, depth, motion = case(7, 32, 24, 50)
    R = B.Renderer(n_feat=16, k=4)
    dev = lambda a: torch.tensor(a, device="cuda")
    ga = {k: dev(anc[k]) for k in FIELDS}
    with pytest.raises(B.UpsError):
        R.anchor_update(ga, dev(l), cam, dev(depth), capacity=10)          # capacity < n
    with pytest.raises(B.UpsError):
        R.anchor_update(ga, dev(l), cam, dev(depth), voxel=0.0)
    # outputs on top of the inputs
    L = B.load()
    import ctypes as C
    ac = B.AnchorCfg()
    L.ups_anchor_cfg_default(C.byref(ac))
    ca = B.Anchors(50, *(B._ptr(ga[k]) for k in FIELDS))
    res = B.AnchorResult()
    st = L.ups_anchor_update(R._h, C.byref(ac), B.make_cameras([cam]), B._ptr(dev(depth)), None, C.byref(ca),
                             B._ptr(dev(l)), C.byref(ca), B._ptr(dev(l)), 50, None, C.byref(res), B._stream())
    assert B.STATUS[st] == "ERR_ARG"


def test_degenerate_keyframes():
    """Every pixel dynamic (no insertion, surface anchors missed), every anchor
    pruned (insertion from row 0), anchors and pixels beyond the voxel index range
    (no voxel held, none inserted), and a voxel larger than the scene."""
    cam, anc, l, depth, motion = case(13, 80, 60, 500)
    R = B.Renderer(n_feat=16, k=4)
    _, _, ref = run(R, anc, l, cam, depth, np.ones_like(motion), capacity=500 + 80 * 60, **cfg32(voxel=0.02))
    assert ref["n_inserted"] == 0 and ref["n_hit"] == 0 and ref["n_miss"] > 0
    _, _, ref = run(R, anc, l, cam, depth, motion, capacity=500 + 80 * 60, **cfg32(voxel=0.02, l_prune=10.0))
    assert ref["n_kept"] == 0 and ref["n_inserted"] > 0
    far = dict(anc)
    far["pos"] = anc["pos"] + np.float32(1e5)
    _, _, ref = run(R, far, l, cam, depth, motion, capacity=500 + 80 * 60, **cfg32(voxel=0.05))
    assert ref["n_hit"] == ref["n_miss"] == 0 and ref["n_inserted"] > 0
    _, _, ref = run(R, anc, l, cam, depth * np.float32(1e5), motion, capacity=500 + 80 * 60,
                    **cfg32(voxel=0.01, margin=0.05))
    assert ref["n_inserted"] == 0   # every back-projected voxel index beyond 2^20
    _, _, ref = run(R, anc, l, cam, depth, motion, capacity=500 + 80 * 60, **cfg32(voxel=50.0, margin=0.05))
    assert ref["n_inserted"] <= 8
