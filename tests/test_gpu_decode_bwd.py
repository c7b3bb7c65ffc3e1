"""Decode backward (Eq. 8-9 differentiated) on its own: MLP-weight, anchor and
pose gradients for a given dL/d(decoded Gaussians), against the oracle fed the
same dL/dG.

* FP32 path: 2e-3 relative L2 (the gradient bar);
* BF16 tensor-core path (decode_bf16 with decode_bwd_bf16): every operand of the data-path products
  rounded to BF16 (8 significant bits), and the ReLU masks follow the BF16
  hidden pre-activations (as in the BF16 forward), so a hidden unit near zero
  may switch; the stated bound is 5e-2 relative L2 (the measured values are
  printed, and written to bf16_decode_bwd_error.json in $UPS_REPORT_DIR when set);
* rows (anchor, view) span two scratch chunks (262144 rows each) in the large
  case, and the grad masks that need no scratch run too.
"""
import numpy as np
import pytest

import oracle
from gpu_cases import rel_l2, round_cams, round_dict
from paper_2505_22335_gb300 import binding as B
from paper_2505_22335_gb300 import scenes

pytestmark = pytest.mark.gpu

FP32_RTOL = 2e-3
BF16_RTOL = 5e-2


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def random_dG(seed, V, N, nf):
    rng = np.random.default_rng(seed)
    f = lambda *s: rng.standard_normal(s)
    return [round_dict(dict(mean=f(N, 3), opacity=f(N), scale=f(N, 3), quat=f(N, 4), color=f(N, 3),
                            feat=f(N, nf))) for _ in range(V)]


def make_case(seed, A, K, nf, V):
    anc = round_dict(scenes.anchors(seed, A, K))
    mlp = round_dict(scenes.mlp_weights(seed + 1, K, nf, bias_sigma=0.05))
    cams = round_cams(scenes.cameras(seed, V, 320, 240, 300.0))
    dG = random_dG(seed + 2, V, A * K, nf)
    return dict(anc=anc, mlp=mlp, cams=cams, dG=dG, K=K, nf=nf)


def oracle_grads(case, opacity_tanh=False):
    anc, mlp = case["anc"], case["mlp"]
    acc = {k: np.zeros_like(np.asarray(v, dtype=np.float64)) for k, v in
           list(mlp.items()) + [(k, anc[k]) for k in ("pos", "feat", "offsets", "scaling")]}
    acc = {k: np.ascontiguousarray(v) for k, v in acc.items()}
    pose = np.stack([oracle.decode_bwd(anc, mlp, c, case["K"], case["nf"], g, acc, opacity_tanh)
                     for c, g in zip(case["cams"], case["dG"])])
    acc["pose"] = pose
    return acc


def gpu_grads(case, bf16, mask=B.GRAD_ALL, opacity_tanh=False):
    import torch
    # the BF16 case runs the tensor-core data path of the decode backward (decode_bwd_bf16)
    R = B.Renderer(n_feat=case["nf"], k=case["K"], decode_bf16=int(bf16), decode_bwd_bf16=int(bf16),
                   opacity_tanh=int(opacity_tanh))
    ad, md = B.anchors_to_device(case["anc"], case["mlp"])
    dG = B.to_set(case["dG"], per_view=True)
    d_mlp = {k: torch.zeros_like(v) for k, v in md.items()}
    d_anc = {k: torch.zeros_like(v) for k, v in ad.items()}
    d_pose = torch.zeros(len(case["cams"]), 6, device="cuda")
    R.decode_backward(ad, md, case["cams"], dG, mask, d_mlp, d_anc, d_pose)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in d_mlp.items()}
    out.update({k: v.cpu().numpy().astype(np.float64) for k, v in d_anc.items()})
    out["pose"] = d_pose.cpu().numpy().astype(np.float64)
    return out


NAMES = ("w1", "b1", "w2", "b2", "pos", "feat", "offsets", "scaling", "pose")


REPORT = {}


def errors(got, ref, tag=None):
    e = {k: rel_l2(got[k], ref[k]) for k in NAMES}
    if tag:
        import json
        import os
        REPORT[tag] = e
        print(tag, {k: f"{v:.2e}" for k, v in e.items()})
        out_dir = os.environ.get("UPS_REPORT_DIR")
        if out_dir:
            os.makedirs(out_dir, exist_ok=True)
            with open(os.path.join(out_dir, "bf16_decode_bwd_error.json"), "w") as f:
                json.dump(REPORT, f, indent=1)
    return e


@pytest.fixture(scope="module")
def small():
    c = make_case(3, 2000, 10, 16, 3)
    c["ref"] = oracle_grads(c)
    return c


def test_fp32_decode_backward_matches_oracle(small):
    e = errors(gpu_grads(small, bf16=False), small["ref"], "fp32 A=2000 K=10 nf=16 V=3")
    assert all(v < FP32_RTOL for v in e.values()), e


def test_bf16_decode_backward_within_stated_bound(small):
    e = errors(gpu_grads(small, bf16=True), small["ref"], "bf16 A=2000 K=10 nf=16 V=3")
    assert all(v < BF16_RTOL for v in e.values()), e


@pytest.mark.parametrize("nf", [0, 32])
def test_feature_widths(nf):
    c = make_case(4, 700, 7, nf, 2)
    ref = oracle_grads(c)
    for bf16, tol in ((False, FP32_RTOL), (True, BF16_RTOL)):
        e = errors(gpu_grads(c, bf16), ref, f"{'bf16' if bf16 else 'fp32'} A=700 K=7 nf={nf} V=2")
        assert all(v < tol for v in e.values()), (nf, bf16, e)


@pytest.mark.parametrize("mask", [B.GRAD_POSE, B.GRAD_ANCHOR, B.GRAD_MLP])
def test_single_masks(small, mask):
    """Each gradient alone equals its part of the full run; untouched outputs stay zero."""
    got = gpu_grads(small, bf16=False, mask=mask)
    parts = {B.GRAD_POSE: ("pose",), B.GRAD_ANCHOR: ("pos", "feat", "offsets", "scaling"),
             B.GRAD_MLP: ("w1", "b1", "w2", "b2")}[mask]
    for k in NAMES:
        if k in parts:
            assert rel_l2(got[k], small["ref"][k]) < FP32_RTOL, k
        else:
            assert not np.any(got[k]), k


def test_rows_span_two_scratch_chunks():
    """70k anchors x 4 views = 280k rows: two chunks of the weight-gradient scratch."""
    c = make_case(5, 70_000, 10, 16, 4)
    ref = oracle_grads(c)
    e = errors(gpu_grads(c, bf16=False), ref, "fp32 A=70000 K=10 nf=16 V=4")
    assert all(v < FP32_RTOL for v in e.values()), e
    e = errors(gpu_grads(c, bf16=True), ref, "bf16 A=70000 K=10 nf=16 V=4")
    assert all(v < BF16_RTOL for v in e.values()), e


def test_tanh_opacity_decode_backward(small):
    """The tanh opacity decode (o = tanh(y), the Scaffold-GS form): its derivative
    1 - o^2 in both row kernels."""
    ref = oracle_grads(small, opacity_tanh=True)
    e = errors(gpu_grads(small, bf16=False, opacity_tanh=True), ref, "fp32 tanh A=2000 K=10 nf=16 V=3")
    assert all(v < FP32_RTOL for v in e.values()), e
    e = errors(gpu_grads(small, bf16=True, opacity_tanh=True), ref, "bf16 tanh A=2000 K=10 nf=16 V=3")
    assert all(v < BF16_RTOL for v in e.values()), e
    # the opacity rows of the weights do differ from the sigmoid decode's
    assert rel_l2(ref["b2"][:small["K"]], small["ref"]["b2"][:small["K"]]) > 0.1
