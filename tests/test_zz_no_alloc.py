"""The allocation-free forward (ups_render_forward_static) against the regular
context-based forward (ups_render_forward), through the C ABI.

This entry point exists for callers that may not allocate GPU memory (a
camera-rate tracking front end inside a fixed memory budget); its scratch is
a static device array of the library.  Two calls in a row must each match the
regular forward within the pixel bar of the parity tests, so a call must not
depend on what the previous call left in the shared array.  The file is named
to be collected last.
"""
import numpy as np
import pytest

from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu

ATOL, RTOL = 1e-5, 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()


def _close(a, b):
    a = a.cpu().numpy().astype(np.float64)
    b = b.cpu().numpy().astype(np.float64)
    assert a.shape == b.shape
    assert np.all(np.abs(a - b) <= ATOL + RTOL * np.abs(b)), float(np.abs(a - b).max())


def _case(g_np, cams, nf):
    import torch
    gs = B.to_set(g_np)
    R = B.Renderer(n_feat=nf, k=1)
    ref = R.forward(gs, cams)
    torch.cuda.synchronize()
    for _ in range(2):
        out = R.alloc_images(cams)
        for v in out.values():
            v.fill_(7)  # stale values must be overwritten
        B.render_forward_static(gs, cams, out, nf)
        torch.cuda.synchronize()
        for k in ("color", "depth", "T") + (("feat",) if nf else ()):
            _close(out[k], ref[k])
        assert torch.equal(out["n_contrib"], ref["n_contrib"])
    R.close()


def test_static_forward_matches_context_forward_plain_2k():
    g, cams = scenes.workload_plain_2k(0)
    _case(g, cams, 0)


def test_static_forward_matches_context_forward_multiview_feat16():
    base = scenes.cameras(7, 3, 100, 70, 90.0)
    cams = [base[0], base[1].scaled(0.5), scenes.Camera(40.0, 40.0, 16.5, 8.5, 33, 17, base[2].T_cw)]
    _case(scenes.plain_gaussians(11, 3000, 16), cams, 16)


def test_static_forward_rejects_oversized_input():
    import torch
    g = scenes.plain_gaussians(1, 70_000, 0)
    cams = scenes.cameras(0, 1, 64, 48, 60.0, identity=True)
    gs = B.to_set(g)
    out = B.Renderer(n_feat=0, k=1).alloc_images(cams)
    with pytest.raises(B.UpsError) as ei:
        B.render_forward_static(gs, cams, out, 0)
    assert ei.value.status == 8 and "65536" in str(ei.value)
    torch.cuda.synchronize()


def test_static_forward_rejects_too_many_tiles():
    import torch
    g = scenes.plain_gaussians(2, 100, 0)
    # 2048 x 1040 pixels = 128 x 65 = 8,320 tiles, above the 8,192 limit
    cams = [scenes.Camera(1000.0, 1000.0, 1024.0, 520.0, 2048, 1040, np.eye(4))]
    gs = B.to_set(g)
    out = B.Renderer(n_feat=0, k=1).alloc_images(cams)
    with pytest.raises(B.UpsError) as ei:
        B.render_forward_static(gs, cams, out, 0)
    assert ei.value.status == 8 and "8192" in str(ei.value)
    torch.cuda.synchronize()


def test_static_forward_instance_overflow_then_normal_call():
    """Large Gaussians close to the camera cover most of the 1,200 tiles of a
    640x480 view: more than 524,288 tile instances.  That limit is known only
    after the projection and the depth sort have written the static array; the
    call must fail with the capacity status, and the next call (a normal scene)
    must still match the context forward, i.e. the half-written array must not
    leak into it."""
    import torch
    cams = scenes.cameras(0, 1, 640, 480, 600.0, identity=True)
    big = scenes.plain_gaussians(3, 3000, 16, scale_lo=0.3, scale_hi=0.6)
    gs = B.to_set(big)
    out = B.Renderer(n_feat=16, k=1).alloc_images(cams)
    with pytest.raises(B.UpsError) as ei:
        B.render_forward_static(gs, cams, out, 16)
    assert ei.value.status == 8 and "524288" in str(ei.value)
    torch.cuda.synchronize()
    base = scenes.cameras(7, 3, 100, 70, 90.0)
    cams2 = [base[0], base[1].scaled(0.5), scenes.Camera(40.0, 40.0, 16.5, 8.5, 33, 17, base[2].T_cw)]
    _case(scenes.plain_gaussians(11, 3000, 16), cams2, 16)
