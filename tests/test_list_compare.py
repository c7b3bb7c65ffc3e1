"""The full-size tile-list comparison (gpu_cases.compare_tile_lists,
tie_groups, z_error_bound, tile_q_ratio) on hand-made lists, no GPU: it must
accept exactly the differences its rules allow and flag every other one."""
import numpy as np

import oracle
from gpu_cases import CFG, compare_tile_lists, tie_groups, tile_q_ratio, z_error_bound
from paper_2505_22335_gb300 import scenes


def _lists():
    # two tiles; depths chosen so that ids 1 and 2 tie, nothing else does
    z = np.array([1.0, 2.0, 2.0 + 1e-8, 3.0, 4.0, 5.0])
    e = np.full(6, 1e-7)
    lst = np.array([0, 1, 2, 3, 4, 5, 0, 3])
    rng = np.array([[0, 6], [6, 8]])
    return z, e, lst, rng


def test_groups_follow_the_depth_window():
    z, e, lst, rng = _lists()
    grp = tie_groups(lst, rng, z, e)
    # 1 and 2 share a group; tile 1 starts new groups
    assert grp[1] == grp[2] and len(np.unique(grp)) == 7


def test_identical_and_tie_swapped_lists_pass():
    z, e, lst, rng = _lists()
    grp = tie_groups(lst, rng, z, e)
    for gl in (lst.copy(), np.array([0, 2, 1, 3, 4, 5, 0, 3])):
        out = compare_tile_lists(gl, rng, lst, rng, grp, -1)
        assert out["order"] == 0 and out["dup"] == 0 and not out["missing"] and not out["extra"]


def test_untied_swap_missing_duplicate_and_extra_are_flagged():
    z, e, lst, rng = _lists()
    grp = tie_groups(lst, rng, z, e)
    assert compare_tile_lists(np.array([0, 1, 2, 4, 3, 5, 0, 3]), rng, lst, rng, grp, -1)["order"] == 1
    out = compare_tile_lists(np.array([0, 1, 2, 3, 5, 0, 3]), np.array([[0, 5], [5, 7]]), lst, rng, grp, -1)
    assert out["missing"] == [(0, 4)]
    out = compare_tile_lists(np.array([0, 1, 1, 3, 4, 5, 0, 3]), rng, lst, rng, grp, -1)
    assert out["dup"] == 1
    out = compare_tile_lists(np.array([0, 1, 2, 3, 4, 5, 0, 9, 3]), np.array([[0, 6], [6, 9]]), lst, rng, grp, -1)
    assert out["extra"] == [(1, 9)] and out["order"] == 0


def test_capped_prefix_rules():
    z, e, lst, rng = _lists()
    grp = tie_groups(lst, rng, z, e)
    # cap 2 cuts the tie group {1, 2}: either member may be kept
    for keep in (1, 2):
        out = compare_tile_lists(np.array([0, keep, 0, 3]), np.array([[0, 2], [2, 4]]), lst, rng, grp, 2)
        assert out["prefix"] == 0 and out["order"] == 0 and out["cut"] == 2
    # keeping a later entry instead of the first ones is a prefix error
    out = compare_tile_lists(np.array([0, 3, 0, 3]), np.array([[0, 2], [2, 4]]), lst, rng, grp, 2)
    assert out["prefix"] == 1


def test_depth_bound_and_margin_ratio_on_an_oracle_projection():
    g = scenes.plain_gaussians(0, 300, 0)
    cam = scenes.cameras(1, 1, 96, 64, 80.0)[0]
    pr = oracle.project(g, cam, CFG)
    e = z_error_bound(g["mean"], cam.T_cw)
    v = pr["valid"] == 1
    assert np.all(e[v] > 0) and np.all(e[v] < 1e-5 * np.abs(pr["pcam"][v, 2]))
    lst, rng = oracle.tile_lists(pr, cam, CFG)
    tiles = np.repeat(np.arange(len(rng)), rng[:, 1] - rng[:, 0])
    pairs = list(zip(tiles.tolist(), lst.tolist()))
    q, kap = tile_q_ratio(pr, cam, pairs)
    # every listed (tile, Gaussian) has its exact ellipse meeting the tile box
    assert np.all(q <= 1 + 1e-12) and np.all(kap >= 1)
