"""Pins of the probabilistic-anchor oracle (Sec. 3.3 "Adaptively Structured
Gaussian", Eq. 7): Eq. 7's closed forms, the log-odds update against Eq. 7
iterated in FP64, the observation model on anchors placed by the inverse pose,
insertion against a brute-force FP64 voxel walk in raster order, pruning,
capacity and clamping; no GPU."""
import math

import numpy as np
import pytest

import oracle
from paper_2505_22335_gb300 import scenes

W, H = 37, 23


def cam_at(seed=0):
    rng = np.random.default_rng(seed)
    T = scenes.look_at(rng.normal(size=3) * 0.3 + np.array([0.1, -0.2, -2.0]), rng.normal(size=3) * 0.1)
    return scenes.Camera(30.0, 28.0, 17.3, 11.6, W, H, T)


def world_of(cam, i, j, z):
    """FP64 world point seen at pixel (i, j) at camera depth z (inverse pose)."""
    Xc = np.array([(i - cam.cx) / cam.fx * z, (j - cam.cy) / cam.fy * z, z, 1.0])
    return (np.linalg.inv(np.asarray(cam.T_cw, float)) @ Xc)[:3]


def empty_anchors(n, F=4, K=2):
    return dict(pos=np.zeros((n, 3), np.float32), feat=np.zeros((n, F), np.float32),
                offsets=np.zeros((n, K, 3), np.float32), scaling=np.ones((n, 3), np.float32))


def test_eq7_closed_forms():
    # two observations of 0.7 on an uninformative prior: 1 / (1 + (3/7)^2) = 49/58
    assert oracle.anchor_posterior(0.7, 0.7, 0.5) == pytest.approx(49 / 58, rel=1e-15)
    # with only the prior behind it, the posterior is the observation itself
    for p, pr in [(0.7, 0.3), (0.4, 0.5), (0.9, 0.8)]:
        assert oracle.anchor_posterior(p, pr, pr) == pytest.approx(p, rel=1e-14)
    # an observation equal to the prior changes nothing
    assert oracle.anchor_posterior(0.3, 0.81, 0.3) == pytest.approx(0.81, rel=1e-14)
    # a hit then a miss of 1 - p_hit on a 0.5 prior cancel
    p = oracle.anchor_posterior(0.7, 0.5, 0.5)
    assert oracle.anchor_posterior(0.3, p, 0.5) == pytest.approx(0.5, rel=1e-14)
    assert oracle.logodds(0.5) == 0.0 and oracle.logodds(0.7) == pytest.approx(math.log(7 / 3))


def one_anchor_at(cam, z, depth, motion=None):
    anc = empty_anchors(1)
    anc["pos"][0] = world_of(cam, 20, 9, z)
    return anc


@pytest.mark.parametrize("p_prior", [0.5, 0.3])
def test_logodds_update_follows_eq7_iterated(p_prior):
    cam = cam_at(1)
    depth = np.full((H, W), 2.0)
    cfg = oracle.AnchorCfg(l_prior=oracle.logodds(p_prior), l_min=-50.0, l_max=50.0, l_prune=-100.0)
    hit = one_anchor_at(cam, 2.0, depth)      # on the surface
    miss = one_anchor_at(cam, 1.0, depth)     # in the free space in front of it
    rng = np.random.default_rng(3)
    l = np.array([oracle.logodds(0.6)], np.float32)
    p = 0.6
    for step in range(40):
        is_hit = rng.uniform() < 0.6
        out = oracle.anchor_update(hit if is_hit else miss, l, cam, depth, None, cfg, capacity=1)
        assert (out["n_hit"], out["n_miss"]) == ((1, 0) if is_hit else (0, 1))
        l = out["logodds"][:1]
        p = oracle.anchor_posterior(0.7 if is_hit else 0.4, p, p_prior)
        assert 1.0 / (1.0 + math.exp(-float(l[0]))) == pytest.approx(p, rel=2e-5, abs=1e-7), step


def test_observation_model_on_placed_anchors():
    cam = cam_at(2)
    depth = np.full((H, W), 2.5)
    depth[5, 30] = 0.0                       # no depth at this pixel
    motion = np.zeros((H, W), np.uint8)
    motion[15, 4] = 1                        # dynamic pixel
    cases = [  # (pixel, camera depth, expected observation)
        ((20, 9), 2.5, 1),        # static surface: hit
        ((3, 17), 2.5 + 0.04, 1),  # inside the surface band
        ((33, 2), 1.2, 2),        # free space in front of the surface: miss
        ((4, 15), 2.5, 2),        # surface of a dynamic pixel: miss
        ((4, 15), 1.0, 2),        # free space in front of a dynamic pixel: miss
        ((11, 20), 3.5, 0),       # behind the surface: occluded
        ((30, 5), 2.5, 0),        # pixel without depth
        ((20, 9), 0.1, 0),        # nearer than near_z
        ((W + 4, 9), 2.5, 0),     # projects right of the image
        ((20, -3), 2.5, 0),       # above the image
    ]
    pos = [world_of(cam, i, j, z) for (i, j), z, _ in cases]
    pos.append(world_of(cam, 20, 9, -2.0))   # behind the camera
    expect = [e for _, _, e in cases] + [0]
    obs = oracle.anchor_observe(np.array(pos), cam, depth, motion, oracle.AnchorCfg())
    assert obs.tolist() == expect
    # the image axes are not exchanged: a transposed lookup would read pixel (9, 20)
    d2 = depth.copy()
    d2[9, 20] = 1.0
    assert oracle.anchor_observe(np.array(pos[:1]), cam, d2, motion, oracle.AnchorCfg()).tolist() == [0]


def boundary_free_depth(cam, depth, voxel, tol=2e-3):
    """Zero the depth of pixels whose FP64 world point lies within tol voxels of a
    voxel face (where FP32 and FP64 could put it in different voxels)."""
    d = depth.copy()
    for j in range(H):
        for i in range(W):
            if d[j, i] > 0:
                x = world_of(cam, i, j, float(np.float32(d[j, i]))) / voxel
                if np.min(np.abs(x - np.round(x))) < tol:
                    d[j, i] = 0.0
    return d


def brute_force_insert(cam, depth, motion, voxel, held, near_z=0.2):
    """Voxels of the static valid pixels in raster order, first pixel kept, minus `held`."""
    seen, out = set(held), []
    for j in range(H):
        for i in range(W):
            D = float(np.float32(depth[j, i]))
            if D > near_z and (motion is None or motion[j, i] == 0):
                q = tuple(int(v) for v in np.floor(world_of(cam, i, j, D) / voxel))
                if q not in seen:
                    seen.add(q)
                    out.append((q, j * W + i))
    return out


def keyframe(seed):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    depth = 2.0 + 0.03 * xx - 0.02 * yy + rng.uniform(0, 0.05, (H, W))
    depth[rng.uniform(size=(H, W)) < 0.1] = 0.0
    motion = ((xx - 25) ** 2 + (yy - 8) ** 2 < 20).astype(np.uint8)
    return depth.astype(np.float32), motion


@pytest.mark.parametrize("seed", [4, 5])
def test_insertion_against_brute_force(seed):
    cam = cam_at(seed)
    cfg = oracle.AnchorCfg(voxel=0.07)
    depth, motion = keyframe(seed)
    depth = boundary_free_depth(cam, depth, cfg.voxel)
    # two anchors already hold voxels of the keyframe (far from every face)
    anc = empty_anchors(3)
    held = []
    for a, (i, j) in enumerate([(6, 4), (10, 19)]):
        x = world_of(cam, i, j, float(depth[j, i]) if depth[j, i] > 0 else 2.0)
        q = np.floor(x / cfg.voxel)
        anc["pos"][a] = (q + 0.5) * cfg.voxel
        held.append(tuple(int(v) for v in q))
    anc["pos"][2] = world_of(cam, 18, 11, -3.0)    # behind the camera: kept, never observed
    l0 = np.zeros(3, np.float32)
    ref = brute_force_insert(cam, depth, motion, cfg.voxel, held)
    out = oracle.anchor_update(anc, l0, cam, depth, motion, cfg, capacity=10_000)
    assert out["n_kept"] == 3 and out["n_inserted"] == len(ref) > 20 and out["n_dropped"] == 0
    assert out["src"][:3].tolist() == [0, 1, 2]
    assert out["src"][3:].tolist() == [-1 - p for _, p in ref]
    centres = np.array([(np.array(q) + 0.5) * cfg.voxel for q, _ in ref])
    assert np.allclose(out["pos"][3:], centres, rtol=0, atol=1e-6)
    assert np.all(out["scaling"][3:] == np.float32(cfg.voxel))
    assert not out["feat"][3:].any() and not out["offsets"][3:].any()
    assert np.all(out["logodds"][3:] == np.float32(cfg.l_prior) + (np.float32(cfg.l_hit) - np.float32(cfg.l_prior)))
    # capacity keeps the raster-first new voxels
    cut = oracle.anchor_update(anc, l0, cam, depth, motion, cfg, capacity=5)
    assert cut["n_inserted"] == 2 and cut["n_dropped"] == len(ref) - 2
    assert cut["src"][3:].tolist() == out["src"][3:5].tolist()
    # the same keyframe again inserts nothing: every static voxel now holds an anchor
    again = oracle.anchor_update({k: out[k] for k in ("pos", "feat", "offsets", "scaling")}, out["logodds"], cam,
                                 depth, motion, cfg, capacity=10_000)
    assert again["n_inserted"] == 0


def test_prune_clamp_and_order():
    cam = cam_at(6)
    depth = np.full((H, W), 2.0, np.float32)
    cfg = oracle.AnchorCfg(l_prune=0.3)
    n = 8
    anc = empty_anchors(n)
    anc["feat"][:] = np.arange(n)[:, None]
    # even rows in free space (miss), odd rows behind the camera (no observation)
    for a in range(n):
        anc["pos"][a] = world_of(cam, 3 + 4 * a, 5 + a, 1.0 if a % 2 == 0 else -1.0)
    l0 = np.array([0.2, 0.2, 0.9, 0.9, 5.0, -5.0, 0.31, 0.29], np.float32)
    out = oracle.anchor_update(anc, l0, cam, np.zeros((H, W), np.float32), None, cfg, capacity=n)
    assert out["n_hit"] == out["n_miss"] == 0 and out["n_inserted"] == 0  # no depth: nothing observed
    assert out["src"].tolist() == [2, 3, 4, 6]          # l >= 0.3 kept, in order, unclamped
    assert np.array_equal(out["logodds"], l0[[2, 3, 4, 6]])
    out = oracle.anchor_update(anc, l0, cam, depth, None, cfg, capacity=n)
    dm = np.float32(cfg.l_miss) - np.float32(cfg.l_prior)
    lm, lx = np.float32(cfg.l_min), np.float32(cfg.l_max)
    # observed rows are clamped after the update (5 - 0.41 comes down to l_max), the others untouched
    exp = np.where(np.arange(n) % 2 == 0, np.minimum(np.maximum(l0 + dm, lm), lx), l0)
    assert exp[4] == lx and exp[5] == np.float32(-5.0)
    assert out["n_miss"] == 4
    keep = np.nonzero(exp >= np.float32(0.3))[0]
    assert out["src"][:len(keep)].tolist() == keep.tolist()
    assert np.array_equal(out["logodds"][:len(keep)], exp[keep])
    assert np.array_equal(out["feat"][:len(keep), 0], keep.astype(np.float32))
    # repeated misses saturate at l_min, repeated hits at l_max
    a1 = empty_anchors(1)
    a1["pos"][0] = world_of(cam, 9, 9, 1.0)
    l = np.zeros(1, np.float32)
    cfg0 = oracle.AnchorCfg(l_prune=-100.0)
    for _ in range(20):
        l = oracle.anchor_update(a1, l, cam, depth, None, cfg0, 1)["logodds"]
    assert l[0] == np.float32(cfg0.l_min)
    a1["pos"][0] = world_of(cam, 9, 9, 2.0)
    for _ in range(20):
        l = oracle.anchor_update(a1, l, cam, depth, None, cfg0, 1)["logodds"]
    assert l[0] == np.float32(cfg0.l_max)


def test_empty_inputs():
    cam = cam_at(7)
    out = oracle.anchor_update(empty_anchors(0), np.zeros(0, np.float32), cam, np.zeros((H, W), np.float32),
                               None, oracle.AnchorCfg(), capacity=0)
    assert out["n_kept"] == out["n_inserted"] == out["n_dropped"] == 0 and out["pos"].shape == (0, 3)
