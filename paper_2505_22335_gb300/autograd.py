"""torch.autograd.Function wrappers of the C-ABI render path.

The forward calls the library's decode and render; the backward calls its
reverse-order blending backward (per-pixel transmittance recomputed by division
from the stored final T, no per-fragment state), the projection backward and
the decode backward.  The camera pose enters as a twist xi (one 6-vector per
view, zeros in the forward): T_cw(xi) = Exp(xi) T_cw, so d loss / d xi is the
pose gradient of tracking.

One Renderer holds the state of one forward; call backward before the next
forward on the same Renderer (an error is raised otherwise).
"""
from __future__ import annotations

import itertools

import torch

from . import binding as B

_token = itertools.count(1)


def _check_alive(renderer, token):
    if getattr(renderer, "_autograd_token", None) != token:
        raise RuntimeError("the Renderer ran another forward since this graph was built; "
                           "use one Renderer per in-flight graph")


def _images(renderer, img, cams):
    """Split the flat library images into per-view tensors [C, H, W]."""
    nf = renderer.n_feat
    outs = []
    P = 0
    for c in cams:
        hw = c.width * c.height
        outs.append(dict(color=img["color"][3 * P:3 * (P + hw)].view(3, c.height, c.width),
                         depth=img["depth"][P:P + hw].view(c.height, c.width),
                         feat=img["feat"][nf * P:nf * (P + hw)].view(nf, c.height, c.width),
                         T=img["T"][P:P + hw].view(c.height, c.width)))
        P += hw
    return outs


class AnchorRender(torch.autograd.Function):
    """(anchor pos, feat, offsets, scaling, w1, b1, w2, b2, xi) -> flat images
    (colour [3P], depth [P], feature [N_l P], final transmittance [P])."""

    @staticmethod
    def forward(ctx, renderer, cams, pos, feat, offsets, scaling, w1, b1, w2, b2, xi):
        anchors = dict(pos=pos.contiguous(), feat=feat.contiguous(), offsets=offsets.contiguous(),
                       scaling=scaling.contiguous())
        mlp = dict(w1=w1.contiguous(), b1=b1.contiguous(), w2=w2.contiguous(), b2=b2.contiguous())
        g = renderer.decode(anchors, mlp, cams)
        img = renderer.forward(g, cams)
        token = next(_token)
        renderer._autograd_token = token
        ctx.renderer, ctx.cams, ctx.token = renderer, cams, token
        ctx.anchors, ctx.mlp, ctx.g = anchors, mlp, g
        ctx.mark_non_differentiable(img["n_contrib"])
        return img["color"], img["depth"], img["feat"], img["T"], img["n_contrib"]

    @staticmethod
    def backward(ctx, g_color, g_depth, g_feat, g_T, _g_nc):
        R = ctx.renderer
        _check_alive(R, ctx.token)
        dL = {}
        for k, v in (("color", g_color), ("depth", g_depth), ("feat", g_feat), ("T", g_T)):
            if v is not None:
                dL[k] = v.contiguous()
        grad, d_pose = R.backward(dL, B.GRAD_ALL)
        d_mlp = {k: torch.zeros_like(v) for k, v in ctx.mlp.items()}
        d_anc = {k: torch.zeros_like(v) for k, v in ctx.anchors.items()}
        R.decode_backward(ctx.anchors, ctx.mlp, ctx.cams, grad, B.GRAD_ALL, d_mlp, d_anc, d_pose)
        R._autograd_token = None
        return (None, None, d_anc["pos"], d_anc["feat"], d_anc["offsets"], d_anc["scaling"],
                d_mlp["w1"], d_mlp["b1"], d_mlp["w2"], d_mlp["b2"], d_pose)


class GaussianRender(torch.autograd.Function):
    """Plain 3DGS: (mean_opacity, scale, quat, colour, feature [1, n, .] float4 records, xi) ->
    flat images.  Gradients are summed over views."""

    @staticmethod
    def forward(ctx, renderer, cams, mean_opacity, scale, quat, color, feat, xi):
        g = B.GaussianSet(mean_opacity.contiguous(), scale.contiguous(), quat.contiguous(),
                          color.contiguous(), feat.contiguous(), False)
        img = renderer.forward(g, cams)
        token = next(_token)
        renderer._autograd_token = token
        ctx.renderer, ctx.token = renderer, token
        ctx.mark_non_differentiable(img["n_contrib"])
        return img["color"], img["depth"], img["feat"], img["T"], img["n_contrib"]

    @staticmethod
    def backward(ctx, g_color, g_depth, g_feat, g_T, _g_nc):
        R = ctx.renderer
        _check_alive(R, ctx.token)
        dL = {}
        for k, v in (("color", g_color), ("depth", g_depth), ("feat", g_feat), ("T", g_T)):
            if v is not None:
                dL[k] = v.contiguous()
        grad, d_pose = R.backward(dL, B.GRAD_POSE | B.GRAD_GAUSS)
        R._autograd_token = None
        return (None, None, grad.mean_opacity, grad.scale, grad.quat, grad.color, grad.feat, d_pose)


def render_anchors(renderer, cams, anchors, mlp, xi=None):
    """Differentiable decode + render; returns per-view image dicts and n_contrib."""
    if xi is None:
        xi = torch.zeros(len(cams), 6, device=anchors["pos"].device, requires_grad=True)
    col, dep, fea, T, nc = AnchorRender.apply(renderer, cams, anchors["pos"], anchors["feat"],
                                              anchors["offsets"], anchors["scaling"], mlp["w1"],
                                              mlp["b1"], mlp["w2"], mlp["b2"], xi)
    return _images(renderer, dict(color=col, depth=dep, feat=fea, T=T), cams), nc


def render_gaussians(renderer, cams, g: B.GaussianSet, xi=None):
    if xi is None:
        xi = torch.zeros(len(cams), 6, device=g.mean_opacity.device, requires_grad=True)
    col, dep, fea, T, nc = GaussianRender.apply(renderer, cams, g.mean_opacity, g.scale, g.quat,
                                                g.color, g.feat, xi)
    return _images(renderer, dict(color=col, depth=dep, feat=fea, T=T), cams), nc
