"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

No GPU.  Each test checks the oracle against something other than itself:
closed forms of a single Gaussian (Eq. 1-3), invariants of front-to-back
blending (Eq. 3: weights plus final transmittance telescope to 1, transmittance
never increases), brute force over all pixels versus the tiled render, library
routines (scipy rotations, numpy stable sort, numpy matmul) in special cases,
and central finite differences for every gradient.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

import oracle
from paper_2505_22335_gb300 import scenes

CFG = oracle.RenderCfg()
BRUTE = oracle.RenderCfg(brute=True)


def cam(fx=100.0, fy=120.0, w=64, h=48, T=None, cx=None, cy=None, t_norm=0.5):
    return scenes.Camera(fx, fy, w / 2 if cx is None else cx, h / 2 if cy is None else cy,
                         w, h, np.eye(4) if T is None else T, t_norm)


def gauss(means, scales, quats=None, opac=None, colors=None, feat=None):
    means = np.atleast_2d(np.asarray(means, float))
    n = means.shape[0]
    scales = np.broadcast_to(np.asarray(scales, float), (n, 3)).copy()
    quats = (np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None
             else np.atleast_2d(np.asarray(quats, float)).copy())
    opac = np.full(n, 0.8) if opac is None else np.asarray(opac, float).reshape(n)
    colors = (np.tile([1.0, 0.5, 0.25], (n, 1)) if colors is None
              else np.atleast_2d(np.asarray(colors, float)).copy())
    feat = np.zeros((n, 0)) if feat is None else np.atleast_2d(np.asarray(feat, float))
    return dict(mean=means, scale=scales, quat=quats, opacity=opac, color=colors, feat=feat)


def render(g, c, cfg=CFG, nf=0):
    pr = oracle.project(g, c, cfg)
    return pr, oracle.render(pr, g, c, cfg, nf)


# ---------------------------------------------------------------------------
# Eq. 1-2: projection closed forms
# ---------------------------------------------------------------------------

def test_isotropic_on_axis_footprint_and_peak():
    c = cam()
    s, z, o = 0.05, 2.0, 0.8
    g = gauss([[0, 0, z]], s, opac=[o])
    pr, img = render(g, c)
    sxx = (c.fx * s / z) ** 2 + 0.3
    syy = (c.fy * s / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [sxx, 0, syy], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(pr["conic"][0], [1 / sxx, 0, 1 / syy], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(pr["uv"][0], [c.cx, c.cy], atol=1e-13)
    k2 = 2 * math.log(255 * o)
    np.testing.assert_allclose(pr["extent"][0], [c.cx - math.sqrt(k2 * sxx), c.cy - math.sqrt(k2 * syy),
                                                 c.cx + math.sqrt(k2 * sxx), c.cy + math.sqrt(k2 * syy)],
                               rtol=1e-13)
    cx, cy = int(c.cx), int(c.cy)
    # peak alpha at the centre pixel, and alpha at radius rho along x
    assert img["color"][0, cy, cx] == pytest.approx(o, abs=1e-14)
    assert img["T"][cy, cx] == pytest.approx(1 - o, abs=1e-14)
    for rho in (1, 3, 6):
        a = o * math.exp(-rho * rho / (2 * sxx))
        assert img["color"][0, cy, cx + rho] == pytest.approx(a, rel=1e-13)
        a = o * math.exp(-rho * rho / (2 * syy))
        assert img["color"][1, cy + rho, cx] == pytest.approx(0.5 * a, rel=1e-13)
    # outside the alpha_min ellipse nothing is blended
    r_out = int(math.ceil(math.sqrt(k2 * sxx))) + 1
    assert img["T"][cy, cx + r_out] == 1.0
    assert img["n_contrib"][cy, cx] == 1


def test_isotropic_rotation_invariance():
    rng = np.random.default_rng(3)
    c = cam()
    base, _ = render(gauss([[0.1, -0.2, 2.5]], 0.04), c)
    for _ in range(5):
        q = rng.normal(size=4) * rng.uniform(0.2, 5)
        pr, _ = render(gauss([[0.1, -0.2, 2.5]], 0.04, quats=[q]), c)
        np.testing.assert_allclose(pr["cov2d"], base["cov2d"], rtol=1e-12)


def test_off_axis_jacobian():
    c = cam()
    x, y, z, s = 0.3, -0.2, 2.0, 0.03
    pr, _ = render(gauss([[x, y, z]], s), c)
    sxx = s * s * (c.fx / z) ** 2 * (1 + x * x / (z * z)) + 0.3
    syy = s * s * (c.fy / z) ** 2 * (1 + y * y / (z * z)) + 0.3
    sxy = s * s * c.fx * c.fy * x * y / z ** 4
    np.testing.assert_allclose(pr["cov2d"][0], [sxx, sxy, syy], rtol=1e-13)
    np.testing.assert_allclose(pr["uv"][0], [c.fx * x / z + c.cx, c.fy * y / z + c.cy], rtol=1e-14)
    assert pr["pcam"][0, 2] == z


def test_quaternion_convention_matches_scipy():
    """Sigma = R S S^T R^T with R the rotation of q = (w, x, y, z)."""
    rng = np.random.default_rng(4)
    c = cam()
    z = 2.0
    for _ in range(6):
        q = rng.normal(size=4)
        s = rng.uniform(0.01, 0.06, size=3)
        pr, _ = render(gauss([[0, 0, z]], s, quats=[q]), c)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = R @ np.diag(s * s) @ R.T
        # on the optical axis J = diag(f/z) on the first two rows
        exp = [(c.fx / z) ** 2 * Sig[0, 0] + 0.3, c.fx * c.fy / z ** 2 * Sig[0, 1],
               (c.fy / z) ** 2 * Sig[1, 1] + 0.3]
        np.testing.assert_allclose(pr["cov2d"][0], exp, rtol=1e-12)
    # 90 deg about z swaps the x/y scales; about x swaps y/z
    s = np.array([0.01, 0.03, 0.05])
    h = math.sqrt(0.5)
    pr, _ = render(gauss([[0, 0, z]], s, quats=[[h, 0, 0, h]]), c)
    np.testing.assert_allclose(pr["cov2d"][0], [(c.fx * s[1] / z) ** 2 + 0.3, 0,
                                               (c.fy * s[0] / z) ** 2 + 0.3], atol=1e-12)
    pr, _ = render(gauss([[0, 0, z]], s, quats=[[h, h, 0, 0]]), c)
    np.testing.assert_allclose(pr["cov2d"][0], [(c.fx * s[0] / z) ** 2 + 0.3, 0,
                                               (c.fy * s[2] / z) ** 2 + 0.3], atol=1e-12)


def test_pose_equals_moving_the_gaussian():
    """Rendering mu with pose T_cw equals rendering (W mu + t) with the identity."""
    rng = np.random.default_rng(5)
    T = scenes.look_at([0.3, -0.2, -0.5], [0.0, 0.1, 2.0])
    W, t = T[:3, :3], T[:3, 3]
    c_pose, c_id = cam(T=T), cam()
    mu = np.array([[0.1, 0.2, 2.2], [-0.3, 0.1, 1.8]])
    q = rng.normal(size=(2, 4))
    s = np.array([[0.02, 0.05, 0.03], [0.04, 0.01, 0.02]])
    g1 = gauss(mu, s, quats=q)
    # the same Gaussian expressed in camera coordinates (scipy composes rotations)
    qc = []
    for qq in q:
        Rm = W @ Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        x, y, z, w = Rotation.from_matrix(Rm).as_quat()
        qc.append([w, x, y, z])
    g2 = gauss((W @ mu.T).T + t, s, quats=qc)
    pr1, im1 = render(g1, c_pose)
    pr2, im2 = render(g2, c_id)
    np.testing.assert_allclose(pr1["cov2d"], pr2["cov2d"], rtol=1e-11)
    np.testing.assert_allclose(pr1["uv"], pr2["uv"], rtol=1e-12)
    np.testing.assert_allclose(im1["color"], im2["color"], atol=1e-12)


def test_culling():
    c = cam()
    g = gauss([[0, 0, 0.1], [0, 0, -1], [5, 0, 2], [0, 0, 2], [0, 0, 2]], 0.03,
              opac=[0.8, 0.8, 0.8, 0.5 / 255, 0.8])
    pr = oracle.project(g, c, CFG)
    assert pr["valid"].tolist() == [0, 0, 0, 0, 1]


# ---------------------------------------------------------------------------
# Eq. 3 / Eq. 10: blending
# ---------------------------------------------------------------------------

def _random_scene(seed, n, nf=0, w=50, h=37):
    rng = np.random.default_rng(seed)
    mean = np.stack([rng.uniform(-0.8, 0.8, n), rng.uniform(-0.6, 0.6, n),
                     rng.uniform(1.5, 3.0, n)], 1)
    g = gauss(mean, np.exp(rng.uniform(math.log(0.01), math.log(0.12), (n, 3))),
              quats=rng.normal(size=(n, 4)), opac=rng.uniform(0.05, 0.99, n),
              colors=rng.uniform(0, 1, (n, 3)), feat=rng.normal(size=(n, nf)))
    return g, cam(fx=40.0, fy=40.0, w=w, h=h)


@pytest.mark.parametrize("brute", [False, True])
def test_weights_plus_final_T_is_one(brute):
    g, c = _random_scene(1, 200)
    g["color"][:] = 1.0
    cfg = oracle.RenderCfg(brute=brute)
    _, img = render(g, c, cfg)
    np.testing.assert_allclose(img["color"][0] + img["T"], 1.0, atol=1e-12)
    assert img["T"].min() >= 1e-4 * (1 - 0.99) - 1e-15


def test_transmittance_never_increases():
    g, c = _random_scene(2, 150)
    _, img = render(g, c, oracle.RenderCfg(t_min=0.0))
    behind = gauss([[0, 0, 3.2]], 0.3, opac=[0.9])
    g2 = {k: np.concatenate([g[k], behind[k]]) for k in g}
    _, img2 = render(g2, c, oracle.RenderCfg(t_min=0.0))
    assert np.all(img2["T"] <= img["T"] + 1e-15)
    assert np.any(img2["T"] < img["T"] - 1e-3)
    assert img["color"].min() >= 0 and img["color"].max() <= 1
    np.testing.assert_array_less(img["depth"], 3.0 * (1 - img["T"]) + 1e-12)


def test_two_gaussian_order():
    c = cam()
    cx, cy = int(c.cx), int(c.cy)
    c1, c2 = [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]
    for (z1, z2) in ((2.0, 2.5), (2.5, 2.0)):
        g = gauss([[0, 0, z1], [0, 0, z2]], 0.05, opac=[0.6, 0.7], colors=[c1, c2])
        _, img = render(g, c)
        a_front, a_back = (0.6, 0.7) if z1 < z2 else (0.7, 0.6)
        col_front, col_back = (c1, c2) if z1 < z2 else (c2, c1)
        exp = a_front * np.array(col_front) + (1 - a_front) * a_back * np.array(col_back)
        np.testing.assert_allclose(img["color"][:, cy, cx], exp, atol=1e-14)
        zf, zb = (z1, z2) if z1 < z2 else (z2, z1)
        assert img["depth"][cy, cx] == pytest.approx(a_front * zf + (1 - a_front) * a_back * zb, abs=1e-14)


def test_early_termination_and_clamp():
    c = cam()
    cx, cy = int(c.cx), int(c.cy)
    n = 20
    g = gauss([[0, 0, 2.0]] * n, 0.05, opac=[0.5] * n, colors=[[1, 1, 1]] * n)
    _, img = render(g, c)
    # 0.5^13 >= 1e-4 > 0.5^14: exactly 13 Gaussians blend at the centre
    assert img["n_contrib"][cy, cx] == 13
    assert img["T"][cy, cx] == pytest.approx(0.5 ** 13, rel=1e-14)
    assert img["color"][0, cy, cx] == pytest.approx(1 - 0.5 ** 13, rel=1e-14)
    g = gauss([[0, 0, 2.0]], 0.05, opac=[0.9999])
    _, img = render(g, c)
    assert img["color"][0, cy, cx] == pytest.approx(0.99, abs=1e-15)


def test_alpha_min_skip():
    c = cam()
    cx, cy = int(c.cx), int(c.cy)
    s, z, o = 0.05, 2.0, 0.8
    sxx = (c.fx * s / z) ** 2 + 0.3
    g = gauss([[0, 0, z]], s, opac=[o])
    _, img = render(g, c)
    for rho in range(1, 20):
        a = o * math.exp(-rho * rho / (2 * sxx))
        exp = a if a >= 1 / 255 else 0.0
        assert img["color"][0, cy, cx + rho] == pytest.approx(exp, abs=1e-15)


@pytest.mark.parametrize("seed,w,h", [(7, 50, 37), (8, 33, 17), (9, 16, 16), (10, 70, 45)])
def test_tiled_equals_brute(seed, w, h):
    """Every pixel with alpha >= alpha_min lies in a tile that lists the Gaussian."""
    g, c = _random_scene(seed, 180, nf=3, w=w, h=h)
    # include Gaussians that straddle or leave the image
    g["mean"][:20, 0] = np.linspace(-1.6, 1.6, 20)
    pr = oracle.project(g, c, CFG)
    a = oracle.render(pr, g, c, CFG, 3)
    b = oracle.render(pr, g, c, BRUTE, 3)
    for k in ("color", "depth", "feat", "T"):
        assert np.array_equal(a[k], b[k]), k


def _q(pr, g, x, y):
    """Quadratic form of Gaussian g at pixel coordinates (x, y) (numpy broadcasting)."""
    a, b, c = pr["conic"][g]
    dx, dy = x - pr["uv"][g, 0], y - pr["uv"][g, 1]
    return a * dx * dx + 2 * b * dx * dy + c * dy * dy


def test_tile_lists_match_stable_sort():
    """Tile lists against independent checks: every tile holding a pixel centre
    with alpha >= alpha_min lists the Gaussian (brute force over pixels); every
    listed tile is in the rect and its box of pixel centres meets the ellipse
    (dense sampling of the box); each list is in ascending (float32 z, id)."""
    g, c = _random_scene(11, 300, w=70, h=45)
    pr = oracle.project(g, c, CFG)
    lst, rng = oracle.tile_lists(pr, c, CFG)
    tx, ty = (c.width + 15) // 16, (c.height + 15) // 16
    listed = [set(lst[rng[t, 0]:rng[t, 1]].tolist()) for t in range(tx * ty)]
    n_dropped = 0
    for gi in range(300):
        if not pr["valid"][gi]:
            assert not any(gi in s for s in listed)
            continue
        k2 = 2 * math.log(g["opacity"][gi] * 255)
        x0, y0, x1, y1 = pr["rect"][gi]
        for t in range(tx * ty):
            ttx, tty = t % tx, t // tx
            in_rect = x0 <= ttx <= x1 and y0 <= tty <= y1
            xs = np.arange(16 * ttx, min(16 * ttx + 16, c.width))
            ys = np.arange(16 * tty, min(16 * tty + 16, c.height))
            if not in_rect:
                assert gi not in listed[t]
                continue
            qpix = _q(pr, gi, xs[None, :].astype(float), ys[:, None].astype(float)).min()
            if qpix <= k2 * (1 - 1e-9):
                assert gi in listed[t], (gi, t)
            if gi in listed[t]:
                xf = np.linspace(xs[0], xs[-1], 8 * (len(xs) - 1) + 1)
                yf = np.linspace(ys[0], ys[-1], 8 * (len(ys) - 1) + 1)
                assert _q(pr, gi, xf[None, :], yf[:, None]).min() <= k2 * 1.01 + 1e-9, (gi, t)
            else:
                n_dropped += 1
    assert n_dropped > 0  # the ellipse test removes rect tiles
    for t in range(tx * ty):
        a = lst[rng[t, 0]:rng[t, 1]]
        key = [(np.float32(pr["pcam"][x, 2]), x) for x in a]
        assert key == sorted(key)
    counts = rng[:, 1] - rng[:, 0]
    assert np.array_equal(rng[:, 0], np.concatenate([[0], np.cumsum(counts)[:-1]]))


def test_elongated_gaussian_lists_only_tiles_it_meets():
    """A long thin Gaussian along the image diagonal: its rect is the full 5 x 5
    tile grid, but the far corners (0, 4) and (4, 0) lie well outside the
    alpha >= alpha_min ellipse and are not listed; the diagonal tiles are."""
    c = cam(fx=100.0, fy=100.0, w=80, h=80)
    rot = Rotation.from_euler("z", 45, degrees=True).as_quat()  # x, y, z, w
    q = [rot[3], rot[0], rot[1], rot[2]]
    g = gauss([[0, 0, 2.0]], [0.8, 0.01, 0.01], quats=[q], opac=[0.9])
    pr = oracle.project(g, c, CFG)
    lst, rng = oracle.tile_lists(pr, c, CFG)
    assert tuple(pr["rect"][0]) == (0, 0, 4, 4)
    listed = {t for t in range(25) if rng[t, 1] > rng[t, 0]}
    for k in range(5):
        assert 5 * k + k in listed
    assert 4 not in listed and 20 not in listed
    assert len(listed) < 25
    # and the render still equals the all-pairs render
    a = oracle.render(pr, g, c, CFG, 0)
    b = oracle.render(pr, g, c, BRUTE, 0)
    for key in ("color", "depth", "T"):
        assert np.array_equal(a[key], b[key]), key


# ---------------------------------------------------------------------------
# Eq. 4 / Eq. 14: loss
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("l2", [False, True])
def test_loss_closed_form_on_constant_images(l2):
    H, W, nf = 5, 7, 2
    img = dict(color=np.full((3, H, W), 0.3), depth=np.full((H, W), 2.0),
               feat=np.full((nf, H, W), -0.5))
    tgt = dict(color=np.full((3, H, W), 0.5), depth=np.full((H, W), 2.5),
               feat=np.full((nf, H, W), 0.5), weight=np.full((H, W), 0.25))
    lc = oracle.LossCfg(lambda_color=0.8, lambda_depth=0.6, lambda_feat=0.4, l2=l2)
    L, gr = oracle.loss_view(img, tgt, lc, nf, norm=float(H * W))
    f = (lambda r: r * r) if l2 else abs
    exp = 0.25 * (0.8 * 3 * f(-0.2) + 0.6 * f(-0.5) + 0.4 * nf * f(-1.0))
    assert L == pytest.approx(exp, rel=1e-14)
    d = (lambda r: 2 * r) if l2 else np.sign
    np.testing.assert_allclose(gr["color"], 0.25 * 0.8 * d(-0.2) / (H * W), rtol=1e-14)
    np.testing.assert_allclose(gr["depth"], 0.25 * 0.6 * d(-0.5) / (H * W), rtol=1e-14)


# ---------------------------------------------------------------------------
# Eq. 8-9: decode
# ---------------------------------------------------------------------------

def test_decode_routing_closed_form():
    """One-hot weights route single inputs to single outputs through each MLP."""
    K, F, Hd, NL = 3, 32, 32, 4
    rng = np.random.default_rng(12)
    A = 5
    anc = dict(pos=rng.uniform(-1, 1, (A, 3)) + [0, 0, 2.5], feat=rng.normal(0, 0.5, (A, F)),
               offsets=rng.normal(0, 0.1, (A, K, 3)), scaling=rng.uniform(0.01, 0.1, (A, 3)))
    nout = K * (11 + NL)
    w1 = np.zeros((4 * Hd, F + 6))
    w2 = np.zeros((nout, Hd))
    b1 = np.zeros(4 * Hd)
    b2 = np.zeros(nout)
    w1[0, F + 3] = 1.0            # opacity hidden 0 <- d_vc
    w1[Hd + 0, F + 0] = 1.0       # covariance hidden 0 <- delta_x
    w1[2 * Hd + 0, F + 4] = 1.0   # colour hidden 0 <- sin(pi t)
    w1[2 * Hd + 1, F + 5] = 1.0   # colour hidden 1 <- cos(pi t)
    w1[3 * Hd + 0, 0] = 1.0       # feature hidden 0 <- f_v[0]
    for k in range(K):
        w2[k, 0] = 1.0                          # o_k = sigmoid(relu(d))
        w2[K + 7 * k + 1, 0] = 1.0              # s_k[1] = l[1] sigmoid(relu(delta_x))
        b2[K + 7 * k + 3] = 1.0                 # q_k = (1, 0, 0, 0)
        w2[8 * K + 3 * k + 2, 0] = 1.0          # c_k[2] = sigmoid(relu(sin pi t))
        w2[8 * K + 3 * k + 0, 1] = 1.0          # c_k[0] = sigmoid(relu(cos pi t))
        w2[11 * K + NL * k + 1, 0] = 2.0        # f_k[1] = 2 softplus(f_v[0])
    mlp = dict(w1=w1, b1=b1, w2=w2, b2=b2)
    centre = np.array([0.4, -0.3, -0.2])
    T = scenes.look_at(centre, [0, 0, 2.5])
    t = 0.3
    c = cam(T=T, t_norm=t)
    out = oracle.decode(anc, mlp, c, K, NL)
    sig = lambda x: 1 / (1 + np.exp(-x))
    relu = lambda x: np.maximum(x, 0)
    for a in range(A):
        r = anc["pos"][a] - centre
        d = np.linalg.norm(r)
        for k in range(K):
            g = a * K + k
            np.testing.assert_allclose(out["mean"][g], anc["pos"][a] + anc["offsets"][a, k], rtol=1e-15)
            assert out["opacity"][g] == pytest.approx(sig(d), rel=1e-13)
            np.testing.assert_allclose(out["scale"][g], anc["scaling"][a] * np.array(
                [0.5, sig(relu(r[0] / d)), 0.5]), rtol=1e-13)
            np.testing.assert_allclose(out["quat"][g], [1, 0, 0, 0], atol=0)
            np.testing.assert_allclose(out["color"][g], [sig(relu(math.cos(math.pi * t))), 0.5,
                                                         sig(relu(math.sin(math.pi * t)))], rtol=1e-13)
            np.testing.assert_allclose(out["feat"][g], [0, 2 * np.log1p(np.exp(anc["feat"][a, 0])), 0, 0],
                                       rtol=1e-13, atol=1e-300)


def test_decode_matches_numpy_matmul():
    """Random weights: the loop oracle equals the same MLP evaluated with numpy matmul."""
    K, NL = 4, 5
    anc = scenes.anchors(13, 7, K)
    mlp = scenes.mlp_weights(14, K, NL, bias_sigma=0.2)
    T = scenes.look_at([0.2, 0.1, -0.3], [0, 0, 2.5])
    c = cam(T=T, t_norm=0.7)
    out = oracle.decode(anc, mlp, c, K, NL)
    oc = -T[:3, :3].T @ T[:3, 3]
    r = anc["pos"] - oc
    d = np.linalg.norm(r, axis=1, keepdims=True)
    x = np.concatenate([anc["feat"], r / d, d, np.full_like(d, math.sin(math.pi * 0.7)),
                        np.full_like(d, math.cos(math.pi * 0.7))], 1)
    z = x @ mlp["w1"].T + mlp["b1"]
    H = 32
    h = np.concatenate([np.maximum(z[:, :3 * H], 0), np.logaddexp(0, z[:, 3 * H:])], 1)
    bounds = [0, K, 8 * K, 11 * K, K * (11 + NL)]
    y = np.concatenate([h[:, g * H:(g + 1) * H] @ mlp["w2"][bounds[g]:bounds[g + 1]].T
                        for g in range(4)], 1) + mlp["b2"]
    sig = lambda v: 1 / (1 + np.exp(-v))
    cov = y[:, K:8 * K].reshape(-1, K, 7)
    np.testing.assert_allclose(out["opacity"], sig(y[:, :K]).ravel(), rtol=1e-12)
    np.testing.assert_allclose(out["scale"], (anc["scaling"][:, None, :] * sig(cov[..., :3])).reshape(-1, 3), rtol=1e-12)
    np.testing.assert_allclose(out["quat"], cov[..., 3:].reshape(-1, 4), rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(out["color"], sig(y[:, 8 * K:11 * K]).reshape(-1, 3), rtol=1e-12)
    np.testing.assert_allclose(out["feat"], y[:, 11 * K:].reshape(-1, NL), rtol=1e-11, atol=1e-13)


# ---------------------------------------------------------------------------
# gradients: central finite differences
# ---------------------------------------------------------------------------

def _fd(f, arr, ana, n_pick, rng, h=1e-6, rtol=1e-5):
    flat = arr.reshape(-1)
    idx = rng.choice(flat.size, size=min(n_pick, flat.size), replace=False)
    num = np.empty(idx.size)
    for j, i in enumerate(idx):
        old = flat[i]
        flat[i] = old + h
        fp = f()
        flat[i] = old - h
        fm = f()
        flat[i] = old
        num[j] = (fp - fm) / (2 * h)
    a = ana.reshape(-1)[idx]
    scale = max(np.linalg.norm(num), 1e-12)
    err = np.linalg.norm(num - a) / scale
    assert err < rtol, (err, num[:6], a[:6])
    assert np.linalg.norm(num) > 0 or np.linalg.norm(a) == 0


def _twist(xi):
    X = np.zeros((4, 4))
    rho, phi = xi[:3], xi[3:]
    X[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    X[:3, 3] = rho
    return expm(X)


def _fd_pose(f, cams, ana, h=1e-6, rtol=1e-5):
    for v, c in enumerate(cams):
        T0 = c.T_cw.copy()
        num = np.empty(6)
        for i in range(6):
            e = np.zeros(6)
            e[i] = h
            c.T_cw = _twist(e) @ T0
            fp = f()
            c.T_cw = _twist(-e) @ T0
            fm = f()
            num[i] = (fp - fm) / (2 * h)
        c.T_cw = T0
        err = np.linalg.norm(num - ana[v]) / max(np.linalg.norm(num), 1e-12)
        assert err < rtol, (v, err, num, ana[v])


SMOOTH = oracle.RenderCfg(alpha_min=0.0, alpha_max=1.0, t_min=0.0, brute=True)


def _fd_cams():
    return [cam(fx=50.0, fy=50.0, w=40, h=32),
            cam(fx=50.0, fy=48.0, w=40, h=32, T=scenes.look_at([0.2, -0.1, 0.1], [0.05, 0.0, 2.0]))]


def _plain_fd_scene(seed, n=12, nf=3):
    rng = np.random.default_rng(seed)
    mean = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(1.6, 2.6, n)], 1)
    g = gauss(mean, np.exp(rng.uniform(math.log(0.04), math.log(0.2), (n, 3))),
              quats=rng.normal(size=(n, 4)), opac=rng.uniform(0.2, 0.9, n),
              colors=rng.uniform(0, 1, (n, 3)), feat=rng.normal(size=(n, nf)))
    cams = _fd_cams()
    tg = scenes.targets(seed + 1, cams, nf, weighted=True, depth_lo=0.0, depth_hi=2.0)
    return g, cams, tg


def _min_margin(cams, fwd_views):
    return min(float(v["img"]["margin"].min()) for v in fwd_views)


@pytest.mark.parametrize("cfg_name,l2", [("smooth", True), ("smooth", False), ("default", False)])
def test_fd_plain_gradients(cfg_name, l2):
    nf = 3
    lc = oracle.LossCfg(lambda_color=0.8, lambda_depth=0.6, lambda_feat=0.4, lambda_scale=0.01, l2=l2)
    cfg = SMOOTH if cfg_name == "smooth" else CFG
    for seed in range(20, 60):
        g, cams, tg = _plain_fd_scene(seed, nf=nf)
        L, out, views, _ = oracle.backward_plain(g, cams, tg, cfg, lc, nf)
        if cfg_name == "smooth" or _min_margin(cams, views) > 1e-3:
            break
    else:
        pytest.fail("no seed with every pair away from the thresholds")
    f = lambda: oracle.forward_plain(g, cams, tg, cfg, lc, nf)
    rng = np.random.default_rng(0)
    for k in ("mean", "scale", "quat", "opacity", "color", "feat"):
        _fd(f, g[k], out[k], 24, rng)
    _fd_pose(f, cams, out["pose"])


def test_fd_transmittance_gradient():
    """dL/dT_final enters the blending backward (objective sum r_p T_p)."""
    g, cams, _ = _plain_fd_scene(3)
    c = cams[1]
    rng = np.random.default_rng(1)
    r = rng.normal(size=(c.height, c.width))
    rc = rng.normal(size=(3, c.height, c.width))

    def f():
        pr = oracle.project(g, c, SMOOTH)
        im = oracle.render(pr, g, c, SMOOTH, 3)
        return float(np.sum(r * im["T"]) + np.sum(rc * im["color"]))

    pr = oracle.project(g, c, SMOOTH)
    g2 = oracle.render_bwd(pr, g, c, SMOOTH, 3, dict(T=r, color=rc))
    g3 = oracle.project_bwd(g, pr, c, SMOOTH, g2)
    _fd(f, g["opacity"], g2["opacity"], 12, rng)
    _fd(f, g["color"], g2["color"], 12, rng)
    _fd(f, g["mean"], g3["mean"], 12, rng)
    _fd(f, g["scale"], g3["scale"], 12, rng)


def _anchor_fd_scene(seed, K=4, nf=3, A=3):
    anc = scenes.anchors(seed, A, K, offset_sigma=0.15, half=0.4, centre=np.array([0.0, 0.0, 2.0]),
                         scaling_lo=0.1, scaling_hi=0.4)
    mlp = scenes.mlp_weights(seed + 1, K, nf, bias_sigma=0.2)
    cams = _fd_cams()
    cams[0].t_norm, cams[1].t_norm = 0.25, 0.6
    tg = scenes.targets(seed + 2, cams, nf, weighted=True, depth_lo=0.0, depth_hi=2.0)
    return anc, mlp, cams, tg


@pytest.mark.parametrize("cfg_name", ["smooth", "default"])
def test_fd_anchor_gradients(cfg_name):
    K, nf = 4, 3
    lc = oracle.LossCfg(lambda_color=1.0, lambda_depth=0.5, lambda_feat=0.3, lambda_scale=0.01)
    cfg = SMOOTH if cfg_name == "smooth" else CFG
    for seed in range(40, 80):
        anc, mlp, cams, tg = _anchor_fd_scene(seed, K, nf)
        L, out, views, _ = oracle.backward_anchor(anc, mlp, cams, tg, cfg, lc, K, nf)
        if cfg_name == "smooth" or _min_margin(cams, views) > 1e-3:
            break
    else:
        pytest.fail("no seed with every pair away from the thresholds")
    f = lambda: oracle.forward_anchor(anc, mlp, cams, tg, cfg, lc, K, nf)
    rng = np.random.default_rng(2)
    for k in ("w1", "b1", "w2", "b2"):
        _fd(f, mlp[k], out[k], 24, rng)
    for k in ("pos", "feat", "offsets", "scaling"):
        _fd(f, anc[k], out[k], 24, rng)
    _fd_pose(f, cams, out["pose"])


def test_decode_tanh_opacity_against_sigmoid_decode():
    """opacity_tanh: o = tanh(y) for the same pre-activation y that the sigmoid decode
    maps to p = sigmoid(y), i.e. o = (p^2 - (1-p)^2) / (p^2 + (1-p)^2); nothing else
    changes."""
    K, NL = 4, 3
    anc = scenes.anchors(21, 9, K)
    mlp = scenes.mlp_weights(22, K, NL, bias_sigma=1.0)
    c = cam(T=scenes.look_at([0.1, -0.2, -0.4], [0, 0, 2.5]), t_norm=0.4)
    s = oracle.decode(anc, mlp, c, K, NL)
    t = oracle.decode(anc, mlp, c, K, NL, opacity_tanh=True)
    p, q = s["opacity"], 1.0 - s["opacity"]
    np.testing.assert_allclose(t["opacity"], (p * p - q * q) / (p * p + q * q), rtol=1e-12, atol=1e-15)
    assert (t["opacity"] < 0).any() and (t["opacity"] > 0).any()
    for k in ("mean", "scale", "quat", "color", "feat"):
        assert np.array_equal(s[k], t[k]), k


def test_fd_anchor_gradients_tanh_opacity():
    """The tanh decode with its o <= 0 Gaussians dropped by the projection: gradients
    of every group against central differences (thresholds off, so the drop at o = 0
    is continuous: such a Gaussian blends with zero alpha)."""
    K, nf = 4, 3
    lc = oracle.LossCfg(lambda_color=1.0, lambda_depth=0.5, lambda_feat=0.3, lambda_scale=0.01)
    anc, mlp, cams, tg = _anchor_fd_scene(44, K, nf)
    mlp["b2"][:K] -= 0.3  # push some opacities below zero
    g = oracle.decode(anc, mlp, cams[0], K, nf, opacity_tanh=True)
    assert (g["opacity"] < 0).any() and (g["opacity"] > 0).any()
    L, out, views, _ = oracle.backward_anchor(anc, mlp, cams, tg, SMOOTH, lc, K, nf, opacity_tanh=True)
    f = lambda: oracle.forward_anchor(anc, mlp, cams, tg, SMOOTH, lc, K, nf, opacity_tanh=True)
    rng = np.random.default_rng(3)
    for k in ("w1", "b1", "w2", "b2"):
        _fd(f, mlp[k], out[k], 24, rng)
    for k in ("pos", "feat", "offsets", "scaling"):
        _fd(f, anc[k], out[k], 16, rng)
    # the opacity rows of b2 in particular (the tanh derivative)
    for i in range(K):
        old = mlp["b2"][i]
        mlp["b2"][i] = old + 1e-6
        lp = f()
        mlp["b2"][i] = old - 1e-6
        lm = f()
        mlp["b2"][i] = old
        assert out["b2"][i] == pytest.approx((lp - lm) / 2e-6, rel=1e-5, abs=1e-9), i
