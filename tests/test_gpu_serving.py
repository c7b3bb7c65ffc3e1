"""Serving: continuous batching over a resident anchor scene.

A request's result (loss, pose gradient, MLP gradient) must be the same when
it runs alone and when it is packed into a batch with other requests, within
the parity bars (pixels/loss 1e-5 + 1e-4 rel, gradients 2e-3 relative L2,
atomic accumulation order being free)."""
import numpy as np
import pytest

from gpu_cases import rel_l2
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu

K, NF = 10, 16


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def scene():
    anc = scenes.anchors(50, 3000, K)
    mlp = scenes.mlp_weights(51, K, NF, bias_sigma=0.05)
    return B.anchors_to_device(anc, mlp)


def pyramid(cam, levels):
    out = []
    for l in range(levels):
        f = 1.0 / (1 << l)
        out.append(scenes.Camera(cam.fx * f, cam.fy * f, cam.cx * f, cam.cy * f, cam.width >> l,
                                 cam.height >> l, cam.T_cw, cam.t_norm))
    return out


def make_request(seed, kind, n_views=3, levels=3, w=160, h=120):
    import torch
    cams = scenes.cameras(seed, n_views if kind == B.MAP else 1, w, h, 150.0)
    views = pyramid(cams[0], levels) if kind == B.TRACK else cams
    tg = B.targets_to_device(scenes.targets(seed + 7, views, NF, weighted=True))
    outs = dict(loss=torch.zeros(1, device="cuda"),
                d_pose=torch.zeros(6 if kind == B.TRACK else 6 * n_views, device="cuda"))
    return dict(kind=kind, cams=cams, views=views, tg=tg, levels=levels, **outs)


def submit(srv, req, mlp_grads=None):
    return srv.submit(req["kind"], req["cams"], req["tg"], req["loss"], req["d_pose"],
                      d_mlp=mlp_grads, levels=req["levels"])


def zero_mlp(md):
    import torch
    return {k: torch.zeros_like(v) for k, v in md.items()}


def test_results_same_alone_and_in_mix(scene):
    import torch
    ad, md = scene
    srv = B.Server(ad, md, n_feat=NF, k=K, slots=2, max_batch_views=32, batching=True)
    track = make_request(1, B.TRACK)
    mapping = make_request(2, B.MAP, n_views=3)
    # alone
    g_alone = zero_mlp(md)
    r1 = srv.wait(submit(srv, track))
    r2 = srv.wait(submit(srv, mapping, g_alone))
    assert r1["status"] == 0 and r2["status"] == 0
    assert r1["batch_requests"] == 1 and r2["batch_requests"] == 1
    alone = dict(tl=track["loss"].item(), tp=track["d_pose"].cpu().numpy().copy(),
                 ml=mapping["loss"].item(), mp=mapping["d_pose"].cpu().numpy().copy(),
                 mg={k: v.cpu().numpy().copy() for k, v in g_alone.items()})
    # in a mix: fill the queue while the GPU is busy so batches pack
    others = [make_request(10 + i, B.TRACK) for i in range(6)] + [make_request(30, B.MAP, n_views=2)]
    g_mix = zero_mlp(md)
    tickets = [submit(srv, o, zero_mlp(md) if o["kind"] == B.MAP else None) for o in others[:3]]
    t_track = submit(srv, track)
    t_map = submit(srv, mapping, g_mix)
    tickets += [submit(srv, o, zero_mlp(md) if o["kind"] == B.MAP else None) for o in others[3:]]
    res = {t: srv.wait(t) for t in tickets + [t_track, t_map]}
    assert all(r["status"] == 0 for r in res.values())
    assert max(r["batch_requests"] for r in res.values()) > 1, "nothing was batched"
    assert abs(track["loss"].item() - alone["tl"]) <= 1e-5 + 1e-4 * abs(alone["tl"])
    assert abs(mapping["loss"].item() - alone["ml"]) <= 1e-5 + 1e-4 * abs(alone["ml"])
    assert rel_l2(track["d_pose"].cpu().numpy(), alone["tp"]) < 2e-3
    assert rel_l2(mapping["d_pose"].cpu().numpy(), alone["mp"]) < 2e-3
    for k in ("w1", "b1", "w2", "b2"):
        assert rel_l2(g_mix[k].cpu().numpy(), alone["mg"][k]) < 2e-3, k
    srv.close()


def test_tracking_request_matches_direct_path(scene):
    """The server's tracking loss and pose gradient equal the direct C-ABI calls
    (decode at the pyramid cameras, forward, loss over all levels, backward)."""
    import torch
    ad, md = scene
    req = make_request(3, B.TRACK)
    srv = B.Server(ad, md, n_feat=NF, k=K, slots=1, batching=True)
    srv.wait(submit(srv, req))
    srv.close()
    R = B.Renderer(n_feat=NF, k=K)
    g = R.decode(ad, md, req["views"])
    img = R.forward(g, req["views"])
    loss, dimg = R.loss(img, req["tg"])
    grad, d_pose = R.backward(dimg, B.GRAD_POSE | B.GRAD_GAUSS)
    R.decode_backward(ad, md, req["views"], grad, B.GRAD_POSE, d_pose=d_pose)
    torch.cuda.synchronize()
    assert abs(req["loss"].item() - loss.item()) <= 1e-5 + 1e-4 * abs(loss.item())
    assert rel_l2(req["d_pose"].cpu().numpy(), d_pose.sum(0).cpu().numpy()) < 2e-3


def test_plain_mode_runs_one_request_per_batch(scene):
    ad, md = scene
    srv = B.Server(ad, md, n_feat=NF, k=K, slots=1, batching=False)
    reqs = [make_request(40 + i, B.TRACK) for i in range(4)]
    ts = [submit(srv, r) for r in reqs]
    res = [srv.wait(t) for t in ts]
    assert all(r["status"] == 0 and r["batch_requests"] == 1 for r in res)
    assert [r["batch_id"] for r in res] == sorted(r["batch_id"] for r in res)
    srv.close()


def test_cancel_and_small_budget_admission(scene):
    ad, md = scene
    srv = B.Server(ad, md, n_feat=NF, k=K, slots=1, batching=True, memory_budget_gb=1e-6)
    reqs = [make_request(60 + i, B.TRACK) for i in range(6)]
    ts = [submit(srv, r) for r in reqs]
    cancelled = srv.cancel(ts[-1])
    res = [srv.wait(t) for t in ts]
    if cancelled == 0:
        assert res[-1]["status"] == 6  # UPS_ERR_CANCELLED
        res = res[:-1]
    assert all(r["status"] == 0 for r in res)
    # a budget smaller than any request admits one request per batch
    assert all(r["batch_requests"] == 1 for r in res)
    srv.wait_idle()
    srv.close()


def test_scene_swap_after_anchor_update(scene):
    """The map changes under the server (a probabilistic anchor update prunes and
    inserts anchors, Eq. 7): after ups_server_set_scene a tracking request renders
    the new scene, equal to the direct calls on it."""
    import torch
    ad, md = scene
    srv = B.Server(ad, md, n_feat=NF, k=K, slots=2, batching=True)
    first = make_request(5, B.TRACK)
    assert srv.wait(submit(srv, first))["status"] == 0
    R = B.Renderer(n_feat=NF, k=K)
    cam = first["cams"][0]
    depth, motion = scenes.keyframe(9, cam)
    lo = torch.zeros(ad["pos"].shape[0], device="cuda")
    new, _, _, cnt = R.anchor_update(ad, lo, cam, torch.tensor(depth, dtype=torch.float32, device="cuda"),
                                     torch.tensor(motion, device="cuda"), capacity=2 * ad["pos"].shape[0],
                                     voxel=0.1, margin=0.1)
    assert cnt["n_inserted"] > 0 and cnt["n_kept"] < ad["pos"].shape[0]
    new = {k: v.contiguous() for k, v in new.items()}
    srv.set_scene(new, md)
    req = make_request(3, B.TRACK)
    assert srv.wait(submit(srv, req))["status"] == 0
    srv.close()
    g = R.decode(new, md, req["views"])
    img = R.forward(g, req["views"])
    loss, dimg = R.loss(img, req["tg"])
    grad, d_pose = R.backward(dimg, B.GRAD_POSE | B.GRAD_GAUSS)
    R.decode_backward(new, md, req["views"], grad, B.GRAD_POSE, d_pose=d_pose)
    torch.cuda.synchronize()
    assert abs(req["loss"].item() - loss.item()) <= 1e-5 + 1e-4 * abs(loss.item())
    assert rel_l2(req["d_pose"].cpu().numpy(), d_pose.sum(0).cpu().numpy()) < 2e-3


def test_served_results_match_oracle():
    """A tracking request (3 pyramid levels of one pose, forward + pose-only
    backward) and a mapping request (3 keyframes, full backward) submitted
    together to the continuous-batching server: each request's loss, pose
    gradient and (mapping) MLP gradient against the FP64 oracle run from the
    same seeded, float32-rounded scene, cameras and targets (loss normalised by
    the request's own pixels, pose gradients of the levels summed)."""
    import torch
    import oracle
    from gpu_cases import CFG, round_cams, round_dict
    anc = round_dict(scenes.anchors(60, 600, K))
    mlp = round_dict(scenes.mlp_weights(61, K, NF, bias_sigma=0.05))
    ad, md = B.anchors_to_device(anc, mlp)
    srv = B.Server(ad, md, n_feat=NF, k=K, slots=2, max_batch_views=16, batching=True)
    cam_t = round_cams(scenes.cameras(62, 1, 160, 120, 150.0))[0]
    levels = pyramid(cam_t, 3)
    tg_t = [round_dict(t) for t in scenes.targets(63, levels, NF, weighted=True)]
    cams_m = round_cams(scenes.cameras(64, 3, 160, 120, 150.0))
    tg_m = [round_dict(t) for t in scenes.targets(65, cams_m, NF, weighted=True)]
    loss_t, pose_t = torch.zeros(1, device="cuda"), torch.zeros(6, device="cuda")
    loss_m, pose_m = torch.zeros(1, device="cuda"), torch.zeros(18, device="cuda")
    g_m = zero_mlp(md)
    t1 = srv.submit(B.TRACK, [cam_t], B.targets_to_device(tg_t), loss_t, pose_t, levels=3)
    t2 = srv.submit(B.MAP, cams_m, B.targets_to_device(tg_m), loss_m, pose_m, d_mlp=g_m)
    r1, r2 = srv.wait(t1), srv.wait(t2)
    assert r1["status"] == 0 and r2["status"] == 0
    torch.cuda.synchronize()
    srv.close()
    lc = oracle.LossCfg()
    L_t, ref_t, _, _ = oracle.backward_anchor(anc, mlp, levels, tg_t, CFG, lc, K, NF)
    L_m, ref_m, _, _ = oracle.backward_anchor(anc, mlp, cams_m, tg_m, CFG, lc, K, NF)
    for L, got in ((L_t, loss_t.item()), (L_m, loss_m.item())):
        assert abs(got - L) <= 1e-5 + 1e-4 * abs(L), (got, L)
    assert rel_l2(pose_t.cpu().numpy(), ref_t["pose"].sum(axis=0)) < 2e-3
    assert rel_l2(pose_m.cpu().numpy().reshape(3, 6), ref_m["pose"]) < 2e-3
    for k in ("w1", "b1", "w2", "b2"):
        assert rel_l2(g_m[k].cpu().numpy(), ref_m[k]) < 2e-3, k
