"""Tile-list cap (ups_config.list_cap).

Blending (Eq. 3 with the t_min stopping reading) reads a tile's depth-ordered
list only until every pixel of the tile has stopped, so keeping the first
list_cap entries of each list changes no pixel as long as every pixel stops
inside the kept prefix; when one does not, the forward rebuilds the lists
without the cap and blends again.  Either way the images must equal the
uncapped render bit for bit (same kernels, same prefix), and the loss and the
backward's per-Gaussian records must equal it up to the order of the atomic
adds.
"""
import numpy as np
import pytest

from gpu_cases import rel_l2, round_cams, round_dict
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


NF = 16


@pytest.fixture(scope="module")
def scene():
    # 60k Gaussians of opacity 0.95 in front of one 160x120 view: tile lists
    # of 626 to 3759 entries whose pixels all stop within the first 263 (the
    # oracle's n_contrib on this scene)
    g = scenes.plain_gaussians(11, 60_000, NF, scale_lo=0.02, scale_hi=0.06)
    g["opacity"] = np.full(60_000, 0.95)
    g = round_dict(g)
    cams = round_cams(scenes.cameras(11, 1, 160, 120, 150.0, identity=True))
    tg = [round_dict(t) for t in scenes.targets(12, cams, NF, weighted=True)]
    return g, cams, tg


def run(scene, cap):
    import torch
    g, cams, tg = scene
    R = B.Renderer(n_feat=NF, k=1, list_cap=cap)
    gs = B.to_set(g)
    img = R.forward(gs, cams)
    loss, dimg = R.loss(img, B.targets_to_device(tg), g=gs)
    R.backward(dimg, B.GRAD_POSE | B.GRAD_GAUSS)
    torch.cuda.synchronize()
    out = dict(img={k: v.cpu().numpy() for k, v in img.items()}, st=R.stats(), loss=float(loss.item()),
               lst=R.copy_buffer(0), rng=R.copy_buffer(2).reshape(-1, 2).astype(np.int64),
               rec=R.copy_buffer(6).astype(np.float64))
    R.close()
    return out


@pytest.fixture(scope="module")
def full(scene):
    return run(scene, -1)


def same_images(a, b):
    for k in ("color", "depth", "feat", "T", "n_contrib"):
        assert np.array_equal(a["img"][k], b["img"][k]), k
    # the loss is a sum of per-block atomic adds: equal up to their order
    assert abs(a["loss"] - b["loss"]) <= 1e-6 * abs(b["loss"])
    assert rel_l2(a["rec"], b["rec"]) < 1e-5


def test_uncapped_lists_are_whole(full):
    st = full["st"]
    assert st["list_refills"] == 0 and st["n_listed"] == st["n_instances"]
    assert np.diff(full["rng"], axis=1).max() > 1000  # long lists: the cap has work to do


def test_cap_keeps_prefixes_and_changes_nothing(scene, full):
    deepest = int(full["img"]["n_contrib"].max())
    cap = 3 * deepest + 64  # every pixel stops well inside the kept prefix
    longest = int(np.diff(full["rng"], axis=1).max())
    assert cap < longest, (cap, longest)
    capd = run(scene, cap)
    st = capd["st"]
    assert st["list_refills"] == 0
    assert st["n_listed"] < st["n_instances"]
    n_full = np.diff(full["rng"], axis=1)[:, 0]
    n_cap = np.diff(capd["rng"], axis=1)[:, 0]
    assert np.array_equal(n_cap, np.minimum(n_full, cap))
    assert int(n_cap.sum()) == st["n_listed"]
    for t in range(len(n_full)):
        a = capd["lst"][capd["rng"][t, 0]:capd["rng"][t, 1]]
        b = full["lst"][full["rng"][t, 0]:full["rng"][t, 0] + n_cap[t]]
        assert np.array_equal(a, b), t
    same_images(capd, full)


def test_short_cap_rebuilds_whole_lists(scene, full):
    capd = run(scene, 2)  # no pixel stops after two Gaussians
    st = capd["st"]
    assert st["list_refills"] == 1
    assert st["n_listed"] == st["n_instances"]
    assert np.array_equal(capd["rng"], full["rng"])
    assert np.array_equal(capd["lst"], full["lst"])
    same_images(capd, full)


def test_default_cap_on_the_dense_scene(scene, full):
    capd = run(scene, 0)  # 0: the default, 1024
    same_images(capd, full)


def test_cap_out_of_range_is_rejected():
    with pytest.raises(B.UpsError):
        B.Renderer(n_feat=NF, k=1, list_cap=40_000)
