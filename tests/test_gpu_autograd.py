"""The torch.autograd.Function wrappers: a loss written in torch on the rendered
images back-propagates through the library's hand-written backward, and the
resulting gradients match the FP64 oracle's analytic gradients (2e-3 relative
L2, the parity bar of the backward)."""
import numpy as np
import pytest

import oracle
from gpu_cases import CFG, assert_grad, round_cams, round_dict
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def torch_loss(views, tgts, nf, l2):
    import torch
    P = sum(v["depth"].numel() for v in views)
    L = 0.0
    for v, t in zip(views, tgts):
        w = t["weight"]
        f = (lambda r: r * r) if l2 else torch.abs
        L = L + (w * f(v["color"] - t["color"]).sum(0)).sum() + (w * f(v["depth"] - t["depth"])).sum()
        if nf:
            L = L + (w * f(v["feat"] - t["feat"]).sum(0)).sum()
    return L / P


def dev_targets(tg):
    import torch
    return [{k: torch.tensor(v, dtype=torch.float32, device="cuda") for k, v in t.items()} for t in tg]


def test_autograd_anchor_render_matches_oracle():
    import torch
    from paper_2505_22335_gb300 import autograd as AG
    K, nf = 10, 16
    anc = round_dict(scenes.anchors(31, 500, K))
    mlp = round_dict(scenes.mlp_weights(32, K, nf, bias_sigma=0.05))
    cams = round_cams(scenes.cameras(31, 2, 128, 96, 120.0))
    tg = [round_dict(t) for t in scenes.targets(33, cams, nf, weighted=True)]
    R = B.Renderer(n_feat=nf, k=K)
    ad, md = B.anchors_to_device(anc, mlp)
    for d in (ad, md):
        for v in d.values():
            v.requires_grad_(True)
    xi = torch.zeros(len(cams), 6, device="cuda", requires_grad=True)
    views, _ = AG.render_anchors(R, cams, ad, md, xi)
    loss = torch_loss(views, dev_targets(tg), nf, l2=False)
    loss.backward()
    L, ref, _, _ = oracle.backward_anchor(anc, mlp, cams, tg, CFG, oracle.LossCfg(), K, nf)
    assert abs(float(loss) - L) <= 1e-5 + 1e-4 * abs(L)
    for k in ("w1", "b1", "w2", "b2"):
        assert_grad(k, md[k].grad.cpu().numpy(), ref[k])
    for k in ("pos", "feat", "offsets", "scaling"):
        assert_grad("anchor_" + k, ad[k].grad.cpu().numpy(), ref[k])
    assert_grad("pose", xi.grad.cpu().numpy(), ref["pose"])


def test_autograd_plain_render_l2_matches_oracle():
    import torch
    from paper_2505_22335_gb300 import autograd as AG
    nf = 0
    g = round_dict(scenes.plain_gaussians(41, 1500, nf))
    cams = round_cams(scenes.cameras(41, 2, 96, 72, 90.0))
    tg = [round_dict(t) for t in scenes.targets(42, cams, nf, weighted=True)]
    R = B.Renderer(n_feat=nf, k=1)
    gs = B.to_set(g)
    for t in (gs.mean_opacity, gs.scale, gs.quat, gs.color):
        t.requires_grad_(True)
    xi = torch.zeros(len(cams), 6, device="cuda", requires_grad=True)
    views, _ = AG.render_gaussians(R, cams, gs, xi)
    loss = torch_loss(views, dev_targets(tg), nf, l2=True)
    loss.backward()
    L, ref, _, _ = oracle.backward_plain(g, cams, tg, CFG, oracle.LossCfg(l2=True), nf)
    assert abs(float(loss) - L) <= 1e-5 + 1e-4 * abs(L)
    mo = gs.mean_opacity.grad.cpu().numpy()[0]
    assert_grad("mean", mo[:, :3], ref["mean"])
    assert_grad("opacity", mo[:, 3], ref["opacity"])
    assert_grad("scale", gs.scale.grad.cpu().numpy()[0, :, :3], ref["scale"])
    assert_grad("quat", gs.quat.grad.cpu().numpy()[0], ref["quat"])
    assert_grad("color", gs.color.grad.cpu().numpy()[0, :, :3], ref["color"])
    assert_grad("pose", xi.grad.cpu().numpy(), ref["pose"])


def test_autograd_rejects_stale_graph():
    import torch
    from paper_2505_22335_gb300 import autograd as AG
    g = round_dict(scenes.plain_gaussians(43, 200, 0))
    cams = round_cams(scenes.cameras(43, 1, 48, 40, 50.0))
    R = B.Renderer(n_feat=0, k=1)
    gs = B.to_set(g)
    gs.color.requires_grad_(True)
    v1, _ = AG.render_gaussians(R, cams, gs)
    v2, _ = AG.render_gaussians(R, cams, gs)  # second forward on the same context
    with pytest.raises(RuntimeError, match="another forward"):
        v1[0]["color"].sum().backward()
    v2[0]["color"].sum().backward()
    assert gs.color.grad is not None and torch.isfinite(gs.color.grad).all()
