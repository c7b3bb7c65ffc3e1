#!/usr/bin/env python
"""Benchmark of the fwd+bwd render path (one JSON line on rank 0).

Workload (default): mapping batch of 100k anchors x K=10 (1M Gaussians), 8
keyframes at 640x480 (fx = fy = 600) on a 3 m arc, RGB + depth + 16-channel
feature map, L1 loss weighted by a per-pixel uncertainty map U[0,1], mean-scale
term 0.01; FP32 decode.  One step = decode -> project -> depth sort -> tile
instances -> tile sort -> ranges -> blend -> loss -> blend backward ->
projection backward -> decode backward (all through the C ABI).

Metric: fwd+bwd Mpixel/s = views x H x W / step time.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU (torchrun): every rank runs an independent replica of the workload
(the path has no exchange step here), time = max over ranks, value = all
ranks' pixels / that time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpixel/s at 1M Gaussians 640x480"
UNIT = "Mpixel/s"

WORKLOADS = {
    # name: anchors, K, n_feat, views, width, height, fx
    "mapping_100k_anchors_x10_8x640x480": dict(A=100_000, K=10, NF=16, V=8, W=640, H=480, fx=600.0),
    "decode_render_10k_anchors_x10_640x480": dict(A=10_000, K=10, NF=16, V=1, W=640, H=480, fx=600.0),
    # smaller case for ncu captures (decoded set 0.26 GB > L2)
    "profile_100k_anchors_x10_2x640x480": dict(A=100_000, K=10, NF=16, V=2, W=640, H=480, fx=600.0),
    # seconds-long case for checks of the JSON contract (the reference arm on CPU)
    "tiny_200_anchors_x4_2x64x48": dict(A=200, K=4, NF=16, V=2, W=64, H=48, fx=80.0),
}
DEFAULT_WORKLOAD = "mapping_100k_anchors_x10_8x640x480"
LAMBDA_SCALE = 0.01


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)),
                    bf16_tflops_sustained=float(d.get("bf16_tflops_sustained", 1700.0)), source="measured")
    return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, bf16_tflops_sustained=1700.0, source="fallback")


# ---------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None,
                    sm_max_mhz=float(max(smax)) if smax else None,
                    reasons=sorted(reasons), samples=len(sm))


# ---------------------------------------------------------------------------
# the workload on the device
# ---------------------------------------------------------------------------

def make_inputs(wl, seed=0):
    from paper_2505_22335_gb300 import scenes
    anc = scenes.anchors(seed, wl["A"], wl["K"])
    mlp = scenes.mlp_weights(seed + 1000, wl["K"], wl["NF"])
    cams = scenes.cameras(seed, wl["V"], wl["W"], wl["H"], wl["fx"], identity=(wl["V"] == 1))
    tg = scenes.targets(seed + 1, cams, wl["NF"], weighted=True)
    return anc, mlp, cams, tg


class Step:
    """Preallocated buffers + one fwd+bwd step through the C ABI."""

    def __init__(self, wl, anc, mlp, cams, tg, device, bf16=False):
        import torch
        from paper_2505_22335_gb300 import binding as B
        self.B = B
        self.wl = wl
        self.cams = cams
        self.R = B.Renderer(n_feat=wl["NF"], k=wl["K"], device=device, decode_bf16=int(bf16))
        self.ad, self.md = B.anchors_to_device(anc, mlp)
        self.tgt = B.targets_to_device(tg)
        V, N = len(cams), wl["A"] * wl["K"]
        self.g = B.GaussianSet.empty(V, N, wl["NF"], True)
        self.img = self.R.alloc_images(cams)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.dimg = dict(color=torch.zeros_like(self.img["color"]), depth=torch.zeros_like(self.img["depth"]),
                         feat=torch.zeros_like(self.img["feat"]))
        self.grad = B.GaussianSet.empty(V, N, wl["NF"], True)
        self.d_pose = torch.zeros(V, 6, dtype=torch.float32, device="cuda")
        self.d_mlp = {k: torch.zeros_like(v) for k, v in self.md.items()}
        self.d_anc = {k: torch.zeros_like(v) for k, v in self.ad.items()}
        self.scale_grad = LAMBDA_SCALE / (3.0 * V * N)

    def run(self):
        B, R = self.B, self.R
        R.decode(self.ad, self.md, self.cams, out=self.g)
        R.forward(self.g, self.cams, out=self.img)
        R.loss(self.img, self.tgt, lambda_scale=LAMBDA_SCALE, g=self.g, loss_out=self.loss,
               grad_out=self.dimg)
        R.backward(self.dimg, B.GRAD_ALL, scale_grad=self.scale_grad, grad=self.grad, d_pose=self.d_pose)
        for v in self.d_mlp.values():
            v.zero_()
        for v in self.d_anc.values():
            v.zero_()
        R.decode_backward(self.ad, self.md, self.cams, self.grad, B.GRAD_ALL, self.d_mlp, self.d_anc,
                          self.d_pose)


def processed_instances(img, cams):
    """Sum over tiles of the longest blended prefix (entries the blend kernels read)."""
    nc = img["n_contrib"].cpu().numpy()
    total = 0
    P = 0
    for c in cams:
        a = nc[P:P + c.width * c.height].reshape(c.height, c.width)
        ty, tx = (c.height + 15) // 16, (c.width + 15) // 16
        pad = np.zeros((ty * 16, tx * 16), a.dtype)
        pad[:c.height, :c.width] = a
        total += int(pad.reshape(ty, 16, tx, 16).max(axis=(1, 3)).sum())
        P += c.width * c.height
    return total


def evaluations(img):
    """Evaluated (pixel, list entry) pairs of the blend: the sum of n_contrib."""
    return int(img["n_contrib"].to(dtype=__import__("torch").int64).sum().item())


def algorithmic(wl, stats, proc_inst, evals=0):
    """Algorithmic bytes (HBM-bound stages) and FP32 flops (ALU-bound stages) per launch.

    Flops count an FMA as 2 and any other arithmetic op (exp included) as 1.
    Blend: per evaluated (pixel, entry) pair 2 (NF + 4) + 12 forward (conic
    quadratic, alpha, weighted colour/depth/features, transmittance) and
    4 NF + 60 backward (alpha recomputed, transmittance by division, feature
    and colour gradients, d alpha, conic / mean / opacity terms).  Decode rows
    (backward, one (anchor, view) row): Z of the four MLPs, Y of the 7 K
    nonlinear outputs, dL/dH through W2 and dL/dx through W1 (36 inputs)."""
    A, K, NF, V = wl["A"], wl["K"], wl["NF"], wl["V"]
    N = A * K
    GV = V * N
    P = stats["n_pixels"]
    I = stats["n_instances"]
    anc_b = 12 + 4 * 32 + 12 * K + 12          # pos, feat, offsets, scaling
    rec3d = 64 + 4 * NF                         # mean|o, scale, quat, colour, features
    n_out = K * (11 + NF)
    row_fwd = 2 * (38 * 128 + 32 * n_out)       # flops per (anchor, view) row
    row_bwd = 2 * (38 * 128 + 7 * K * 32 + 32 * n_out + 36 * 128)
    scratch_row = 4 * (40 + 128 + n_out + 128)  # X, H, dL/dY, dL/dZ per row (feature-major)
    rows = A * V
    inst_b = 16 + 16 + 16 + 4 * NF + 4         # xyzo, conic, colour, features, id
    pix_out = 4 * (3 + 1 + NF + 1) + 4
    passes = lambda bits: (bits + 7) // 8
    return {
        "decode_fwd": dict(bytes=A * anc_b + GV * rec3d, flops=A * V * row_fwd),
        "project": dict(bytes=GV * (48 + 56)),
        "depth_sort": dict(bytes=passes(32 + (math.ceil(math.log2(V)) if V > 1 else 0)) * GV * 32),
        "offsets": dict(bytes=GV * (4 + 4 + 4 + 8)),
        "emit": dict(bytes=GV * 24 + I * 8),
        "tile_sort": dict(bytes=passes(stats["key_bits"]) * I * 20),
        "ranges": dict(bytes=I * 8 + stats["n_tiles"] * 8),
        "composite_fwd": dict(bytes=proc_inst * inst_b + P * pix_out, flops=evals * (2 * (NF + 4) + 12)),
        "loss": dict(bytes=P * 4 * (3 * (3 + 1 + NF) + 1)),
        # gradient records: at most one per read instance receives an atomic add
        "composite_bwd": dict(bytes=proc_inst * (inst_b + 4 * (12 + NF)) + P * (pix_out + 4 * (3 + 1 + NF)),
                              flops=evals * (4 * NF + 60)),
        "project_bwd": dict(bytes=GV * (48 + 4 * (12 + NF) + rec3d)),
        "decode_bwd_rows": dict(bytes=A * anc_b * 2 + GV * rec3d + rows * scratch_row, flops=rows * row_bwd),
        "decode_wgrad": dict(bytes=rows * scratch_row),
    }


ALU_STAGES = {"decode_fwd", "decode_bwd_rows", "composite_fwd", "composite_bwd"}

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a stage's kernel, from
# one ncu capture of that kernel on the named workload: (bytes, capture date, SHA-256 prefix of
# the kernel's source file when it was captured).  Reported as the roofline's `traffic` only while
# the source file still has that hash; any later change of the kernel makes it null (stale).
MEASURED_TRAFFIC = {
    # full ncu captures of one launch on the 2-view profiling workload (1M Gaussians, 2 x 640x480), scaled to the
    # 8-view launch by the list entries the tiles read (384,532 -> 1,618,003; images scale alike, 4x the pixels)
    ("composite_bwd", DEFAULT_WORKLOAD): (301.7e6, "2026-12-04 (2-view capture x 4.21)", "cb96ae212ea91e15"),
    ("composite_fwd", DEFAULT_WORKLOAD): (107.4e6, "2026-12-04 (2-view capture x 4.21)", "cb96ae212ea91e15"),
    # full ncu capture of one 200,000-row launch on the 2-view profiling workload; the 8-view step's 4 launches
    # average the same 200,000 rows, and the traffic is per row (dL/dG read, scratch written)
    ("decode_bwd_rows", DEFAULT_WORKLOAD): (786.9e6, "2026-12-04 (2-view capture, 200k rows = the average launch)",
                                            "ef771be9ad95a383"),
}
STAGE_SOURCE = {"composite_fwd": "composite.cu", "composite_bwd": "composite.cu", "decode_bwd_rows": "decode.cu",
                "decode_fwd": "decode.cu", "decode_wgrad": "wgrad_tc.cu", "project_bwd": "project.cu"}


def source_hash(stage):
    import hashlib
    f = STAGE_SOURCE.get(stage)
    if f is None:
        return None
    with open(os.path.join(ROOT, "paper_2505_22335_gb300", "csrc", f), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def traffic_for(stage, wl_name):
    m = MEASURED_TRAFFIC.get((stage, wl_name))
    if m is None:
        return None, "no ncu capture of this kernel on this workload"
    nbytes, when, sha = m
    if sha != source_hash(stage):
        return None, f"stale: the kernel changed since the {when} capture"
    return nbytes, f"ncu capture of {when} (dram__bytes_read.sum + dram__bytes_write.sum, one launch)"


def run_ours(args, wl_name):
    import torch
    import torch.distributed as dist
    from paper_2505_22335_gb300 import binding as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    wl = WORKLOADS[wl_name]
    anc, mlp, cams, tg = make_inputs(wl, seed=0)
    st = Step(wl, anc, mlp, cams, tg, local, bf16=args.decode_bf16)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        st.run()
    torch.cuda.synchronize()
    stats = st.R.stats()
    st.R.profile_read()  # reset counters
    st.R.profile(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        st.run()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    prof, launches = st.R.profile_read()
    st.R.profile(False)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    pix = sum(c.width * c.height for c in cams)
    value = world * pix / (ms_max / 1e3) / 1e6
    proc = processed_instances(st.img, cams)
    evals = evaluations(st.img)

    # the next rows of the path, timed on their own (not part of the mapping step)
    unc = run_uncertainty(args, st, wl)
    lift = run_lift(args, st, wl)
    ssim = run_ssim(args, st, wl)
    umlp = run_unc_mlp(args, st, wl)
    anch = run_anchor(args, wl, anc, cams[0])

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, st, anc, mlp, tg, world)

    if rank == 0:
        peaks = load_peaks()
        alg = algorithmic(wl, stats, proc, evals)
        stages = {k: dict(ms_per_step=v[0] / args.steps, launches_per_step=v[1] / args.steps)
                  for k, v in prof.items()}
        dom = max(prof, key=lambda k: prof[k][0])
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peaks["sm_count"] = sms
        roof = roofline(dom, alg, prof[dom][0] / args.steps, prof[dom][1] / args.steps, peaks, args.decode_bf16)
        roof["traffic"], roof["traffic_source"] = traffic_for(dom, wl_name)
        # both blend kernels, each against the FP32 pipe and against HBM
        blend = {}
        for stg in ("composite_fwd", "composite_bwd"):
            if stg in prof:
                r = roofline(stg, alg, prof[stg][0] / args.steps, prof[stg][1] / args.steps, peaks)
                h = roofline(stg, alg, prof[stg][0] / args.steps, prof[stg][1] / args.steps, peaks, force_hbm=True)
                tr, trs = traffic_for(stg, wl_name)
                blend[stg] = dict(alu=dict(achieved=r["achieved"], peak=r["peak"], unit=r["unit"], frac=r["frac"],
                                           peak_source=r["peak_source"]),
                                  hbm=dict(achieved=h["achieved"], peak=h["peak"], unit=h["unit"], frac=h["frac"],
                                           peak_source=h["peak_source"]),
                                  avg_launch_ms=r["avg_launch_ms"], traffic=tr, traffic_source=trs)
        cpu = cpu_baseline(wl, anc, mlp, cams, tg) if not args.no_cpu else None
        serving = None
        if not args.no_serving and world == 1 and wl_name == DEFAULT_WORKLOAD:
            del st
            torch.cuda.empty_cache()
            serving = measure_serving(args.serve_seconds)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (bf16 decode GEMMs)" if args.decode_bf16 else "f32",
            "data": "synthetic (seeded anchors, MLP weights, arc poses, targets)",
            "config": {"workload": wl_name, "anchors": wl["A"], "k": wl["K"], "gaussians": wl["A"] * wl["K"],
                       "views": wl["V"], "width": wl["W"], "height": wl["H"], "n_feat": wl["NF"],
                       "decode": "bf16 tensor cores (tcgen05), fp32 accumulate" if args.decode_bf16 else "fp32",
                       "loss": "weighted l1 + 0.01 mean scale",
                       "l2_policy": "inputs larger than L2 (decoded set alone is %.2f GB per step)"
                                    % (wl["V"] * wl["A"] * wl["K"] * (64 + 4 * wl["NF"]) / 1e9),
                       "parallelism": f"replicas x{world}"},
            "gaussians_per_s": round(world * wl["V"] * wl["A"] * wl["K"] / (ms_max / 1e3), 1),
            "gpu_launches": int(launches),
            "clocks": clk,
            "roofline": roof,
            "blend_rooflines": blend,
            "stages": stages,
            "counters": dict(stats, processed_instances=proc, evaluations=evals),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "serving": serving,
            "next_rows": {"tracking_uncertainty": dict(unc, peak=round(peaks["hbm_gbs"], 1),
                                                       frac=round(unc["achieved_gbs"] / peaks["hbm_gbs"], 4),
                                                       peak_source=peaks["source"]),
                          "feature_lifting": dict(lift, **lift_peak(lift, peaks, sms)),
                          "dssim": dict(ssim, peak=round(peaks["hbm_gbs"], 1),
                                        frac=round(ssim["achieved_gbs"] / peaks["hbm_gbs"], 4),
                                        peak_source=peaks["source"]),
                          "uncertainty_mlp": dict(umlp, peak=round(alu_peak(peaks), 2),
                                                  frac=round(umlp["achieved_tflops"] / alu_peak(peaks), 4),
                                                  peak_source=f"derived: {sms} SMs x 128 FP32 lanes x 2 x max SM clock"),
                          "anchor_update": dict(anch, peak=round(peaks["hbm_gbs"], 1),
                                                frac=round(anch["achieved_gbs"] / peaks["hbm_gbs"], 4),
                                                peak_source=peaks["source"])},
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def lift_peak(lift, peaks, sms):
    """Roofline denominator of the lifting call: the measured sustained BF16
    tensor rate where its products run on the tensor cores, else the derived
    FP32 rate."""
    if lift["bound"] == "tensor":
        p = peaks["bf16_tflops_sustained"]
        return dict(peak=round(p, 1), frac=round(lift["achieved_tflops"] / p, 4),
                    peak_source=f"{peaks['source']} (BF16 dense, sustained)")
    p = alu_peak(peaks)
    return dict(peak=round(p, 2), frac=round(lift["achieved_tflops"] / p, 4),
                peak_source=f"derived: {sms} SMs x 128 FP32 lanes x 2 x max SM clock")


def alu_peak(peaks):
    """FP32 FMA peak in TFLOP/s: SMs (from the device properties) x 128 FP32
    lanes x 2 flops x the maximum SM clock."""
    return peaks["sm_count"] * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12


def roofline(stage, alg, stage_ms, launches, peaks, bf16=False, force_hbm=False):
    """Roofline of one stage: its algorithmic work per step over its time per step
    (stages of several launches, e.g. chunked decode backward, are taken whole)."""
    a = alg.get(stage, {})
    common = dict(kernel=stage, traffic=None, stage_ms=round(stage_ms, 4),
                  avg_launch_ms=round(stage_ms / max(launches, 1), 4), algorithmic_bytes=a.get("bytes"))
    if bf16 and not force_hbm and stage == "decode_fwd" and "flops" in a:
        # BF16 operands on the tcgen05 tensor cores; timed inside a long step (the decode
        # backward's data path stays FP32 on the CUDA cores in this configuration)
        peak = peaks["bf16_tflops_sustained"]
        ach = a["flops"] / (stage_ms / 1e3) / 1e12
        return dict(common, bound="tensor", achieved=round(ach, 3), peak=round(peak, 1), unit="TFLOP/s",
                    frac=round(ach / peak, 4), peak_source=peaks["source"] + " (bf16, sustained)",
                    algorithmic_flops=a["flops"])
    if stage in ALU_STAGES and "flops" in a and not force_hbm:
        peak = alu_peak(peaks)
        ach = a["flops"] / (stage_ms / 1e3) / 1e12
        return dict(common, bound="alu", achieved=round(ach, 3), peak=round(peak, 2), unit="TFLOP/s",
                    frac=round(ach / peak, 4),
                    peak_source=f"derived: {peaks['sm_count']} SMs (device properties) x 128 FP32 lanes x 2 x "
                                f"max SM clock {peaks['sm_max_mhz']:.0f} MHz",
                    algorithmic_flops=a["flops"])
    ach = a.get("bytes", 0) / (stage_ms / 1e3) / 1e9
    return dict(common, bound="hbm", achieved=round(ach, 1), peak=peaks["hbm_gbs"], unit="GB/s",
                frac=round(ach / peaks["hbm_gbs"], 4), peak_source=peaks["source"])


def run_uncertainty(args, st, wl):
    """Tracking uncertainty (Eq. 6 residual, Eq. 15 sigma^2 = 2R, motion mask) of
    the last step's rendered views against the targets, through the public API:
    CUDA events over repeated launches on the launch stream (inputs of
    ~0.4 GB, larger than L2).  Algorithmic bytes per pixel: the rendered colour,
    depth, T and N_l features and the target colour, depth and features read
    once (the 3x3 depth window through L1), R, sigma^2 (float) and the mask
    (byte) written."""
    import torch
    img = dict(color=st.img["color"], depth=st.img["depth"], feat=st.img["feat"], T=st.img["T"])
    out = dict(R=torch.empty_like(img["depth"]), sigma2=torch.empty_like(img["depth"]),
               motion=torch.empty(img["depth"].shape, dtype=torch.uint8, device=img["depth"].device))
    for _ in range(3):
        st.R.tracking_uncertainty(img, st.tgt, out=out)
    n = max(10, args.steps)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        st.R.tracking_uncertainty(img, st.tgt, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    NF = wl["NF"]
    pix = wl["V"] * wl["W"] * wl["H"]
    bpp = 4 * ((3 + 1 + 1 + NF) + (3 + 1 + NF)) + 4 + 4 + 1
    return dict(ms=round(ms, 4), pixels=pix, bytes_per_pixel=bpp, bound="hbm",
                achieved_gbs=round(pix * bpp / (ms / 1e3) / 1e9, 1), unit="GB/s",
                motion_frac=round(float(out["motion"].float().mean().item()), 4))


def run_lift(args, st, wl, n_h=384, patch=14):
    """Feature lifting F_m and distillation loss L_d (Eq. 11-12), forward and
    backward (weight and feature-map gradients) on the last step's rendered
    feature map against a seeded synthetic DINO patch grid (n_h = 384, patch
    14), through the public API; CUDA events over repeated calls.  Algorithmic
    FLOPs are those of the reduced form the library computes (the same loss and
    gradients without the n_h-wide F^): per pixel the first layer and its two
    backward products (3 x 2 N_l 128), H M and the Gram of b H (2 x 2 128^2),
    the per-pixel cosine, dL/dZ and per-patch sums (~3.5k, counted as 14 x 2 x
    128); per patch W2^T g and the D G^T product (2 x 2 128 n_h).  The full form
    (F^ materialised) would be 2 (N_l 128 + 128 n_h) + 2 (2 128 n_h + 2 N_l 128)
    per pixel; both are reported."""
    import torch
    NF = wl["NF"]
    gen = torch.Generator(device="cuda").manual_seed(3)
    grids = sum(-(-wl["H"] // patch) * -(-wl["W"] // patch) for _ in range(wl["V"])) * n_h
    dino = torch.randn(grids, generator=gen, device="cuda")
    mlp = dict(w1=torch.randn(128, NF, generator=gen, device="cuda") * 0.3,
               b1=torch.randn(128, generator=gen, device="cuda") * 0.1,
               w2=torch.randn(n_h, 128, generator=gen, device="cuda") * 0.1,
               b2=torch.randn(n_h, generator=gen, device="cuda") * 0.1)
    dmlp = {k: torch.zeros_like(v) for k, v in mlp.items()}
    dfeat = torch.zeros_like(st.img["feat"])
    loss = torch.zeros(1, device="cuda")
    call = lambda: st.R.feature_lift(st.img["feat"], dino, mlp, n_h=n_h, patch=patch, scale=0.4, d_mlp=dmlp,
                                     d_feat=dfeat, loss_out=loss)
    for _ in range(3):
        call()
    n = max(5, args.steps // 2)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    pix = wl["V"] * wl["W"] * wl["H"]
    patches = wl["V"] * -(-wl["H"] // patch) * -(-wl["W"] // patch)
    flops = pix * (3 * 2 * NF * 128 + 2 * 2 * 128 * 128 + 14 * 2 * 128) + patches * 2 * 2 * 128 * n_h
    # at N_l = 16 on the tensor cores: Z = W1 F~, dW1 = dZ F~^T, M H and the Gram of b H
    tensor = pix * (2 * 2 * NF * 128 + 2 * 2 * 128 * 128) if NF == 16 else 0
    full = 2 * (NF * 128 + 128 * n_h) + 2 * (2 * 128 * n_h + 2 * NF * 128)
    return dict(ms=round(ms, 4), pixels=pix, n_h=n_h, algorithmic_flops=flops, full_form_flops_per_pixel=full,
                tensor_core_flops=tensor, bound="tensor" if tensor else "alu",
                achieved_tflops=round(flops / (ms / 1e3) / 1e12, 2), unit="TFLOP/s",
                loss=round(float(loss.item()), 6),
                gemm="reduced form: one fused kernel over all views' patch cells (per-pixel work on chip; at N_l = 16 "
                     "Z = W1 F~ as 3xTF32 and M H, the Gram of b H and dW1 as 3xBF16 tcgen05 MMAs with FP32 "
                     "accumulation, dF~ and the per-pixel terms FP32 on the CUDA cores), hand-written FP32 GEMMs for "
                     "the per-patch and weight-sized products; the split operands make the tensor pipe run about 3x "
                     "the algorithmic count of its products, and the kernel is held by shared-memory wavefronts and "
                     "the MMA round trips rather than by a pipe")


def run_ssim(args, st, wl):
    """The D-SSIM term of Eq. 4, forward and backward (gradient added to a
    colour-gradient buffer), on the last step's rendered colour against the
    target colour, through the public API; CUDA events over repeated calls.
    Algorithmic bytes per channel-pixel: the forward reads both images and
    writes the three window-term maps, the backward reads those maps and both
    images and updates the gradient: 48 B."""
    import torch
    d = torch.zeros_like(st.img["color"])
    loss = torch.zeros(1, device="cuda")
    call = lambda: st.R.ssim_loss(st.img["color"], st.tgt["color"], scale=0.2, d_color=d, loss_out=loss)
    for _ in range(3):
        call()
    n = max(10, args.steps)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    cpx = 3 * wl["V"] * wl["W"] * wl["H"]
    return dict(ms=round(ms, 4), channel_pixels=cpx, bytes_per_channel_pixel=48, bound="hbm",
                achieved_gbs=round(cpx * 48 / (ms / 1e3) / 1e9, 1), unit="GB/s", loss=round(float(loss.item()), 6))


def run_unc_mlp(args, st, wl, n_h=384, patch=14):
    """Uncertainty MLP F_u and L_u (Eq. 5, Eq. 13) with its gradient, on a seeded
    synthetic DINO patch grid and residual map of the bench batch, through the
    public API; CUDA events over repeated calls.  Bound by FP32 arithmetic (9 B
    of pixel traffic against ~2.9 kFLOP per pixel).  Algorithmic FLOPs: per
    pixel the 128 first-layer values interpolated from 4 patches (2 * 4 * 128),
    the output dot (2 * 128), dW2 (2 * 128), dh (128) and its share of the four
    corners (2 * 4 * 128) and db1 (128); per patch the two 128 x n_h products
    (2 * 2 * 128 * n_h)."""
    import torch
    gen = torch.Generator(device="cuda").manual_seed(4)
    grids = sum(-(-wl["H"] // patch) * -(-wl["W"] // patch) for _ in range(wl["V"])) * n_h
    dino = torch.randn(grids, generator=gen, device="cuda")
    Rm = torch.rand(st.img["depth"].shape, generator=gen, device="cuda")
    mlp = dict(w1=torch.randn(128, n_h, generator=gen, device="cuda") * 0.1,
               b1=torch.randn(128, generator=gen, device="cuda") * 0.1,
               w2=torch.randn(128, generator=gen, device="cuda") * 0.2,
               b2=torch.full((1,), 0.2, device="cuda"))
    dm = {k: torch.zeros_like(v) for k, v in mlp.items()}
    loss = torch.zeros(1, device="cuda")
    out = dict(sigma=torch.empty_like(Rm), motion=torch.empty(Rm.shape, dtype=torch.uint8, device="cuda"))
    call = lambda: st.R.uncertainty_mlp(dino, Rm, mlp, n_h=n_h, patch=patch, d_mlp=dm, out=out, loss_out=loss)
    for _ in range(3):
        call()
    n = max(10, args.steps)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    pix = wl["V"] * wl["W"] * wl["H"]
    patches = wl["V"] * -(-wl["H"] // patch) * -(-wl["W"] // patch)
    flops = pix * (2 * 4 * 128 + 2 * 128 + 2 * 128 + 128 + 2 * 4 * 128 + 128) + patches * 4 * 128 * n_h
    return dict(ms=round(ms, 4), pixels=pix, n_h=n_h, algorithmic_flops=flops, bound="alu",
                achieved_tflops=round(flops / (ms / 1e3) / 1e12, 3), unit="TFLOP/s",
                note="first layer per DINO patch (exact by linearity), per-pixel rest on CUDA cores")


def run_anchor(args, wl, anc, cam):
    """Probabilistic anchor update (Eq. 7) with pruning and insertion: the bench
    batch's anchors against one seeded synthetic keyframe of view 0 (scenes.keyframe:
    depth surface with holes and a moving disc), through the public API; the
    device time of the call's kernels from the library's stage events (the call
    ends with one synchronisation that reads the counts back), and the host wall
    time per call.  Algorithmic bytes: every input anchor row read once (pos,
    feature, offsets, scaling, log-odds), every kept row written with its source
    index, every keyframe pixel's depth and motion read, every new row written."""
    import torch
    from paper_2505_22335_gb300 import binding as B
    from paper_2505_22335_gb300 import scenes
    R = B.Renderer(n_feat=wl["NF"], k=wl["K"])
    depth, motion = scenes.keyframe(7, cam)
    t = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    ga = {k: t(anc[k]) for k in ("pos", "feat", "offsets", "scaling")}
    lo = t(np.random.default_rng(8).uniform(-2.5, 3.5, wl["A"]))
    dd, mm = t(depth), t(motion, torch.uint8)
    call = lambda: R.anchor_update(ga, lo, cam, dd, mm, capacity=wl["A"] * 2)
    for _ in range(3):
        call()
    R.profile_read()
    R.profile(True)
    n = max(10, args.steps)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(n):
        _, _, _, cnt = call()
    wall = (time.perf_counter() - w0) / n * 1e3
    prof, launches = R.profile_read()
    R.profile(False)
    ms = prof["anchor_update"][0] / n
    row = 4 * (3 + 32 + 3 * wl["K"] + 3 + 1)  # pos, feature (32), offsets, scaling, log-odds
    P = cam.width * cam.height
    nbytes = wl["A"] * row + cnt["n_kept"] * (row + 4) + P * 5 + cnt["n_inserted"] * (row + 4)
    R.close()
    return dict(ms=round(ms, 4), wall_ms_per_call=round(wall, 4), launches_per_call=launches / n,
                anchors=wl["A"], pixels=P, counts=cnt, algorithmic_bytes=nbytes, bound="hbm",
                achieved_gbs=round(nbytes / (ms / 1e3) / 1e9, 1), unit="GB/s")


def run_e2e(args, st, anc, mlp, tg, world):
    """Same step through the public API, inputs copied from pinned host memory
    and the loss + pose gradient read back, every step, inside the timed region.
    The inputs are double-buffered on the device: while step i runs on the
    compute stream, a copy stream brings step i + 1's inputs into the other
    buffer set (after step i - 1, the last user of that set, has finished)."""
    import torch
    host = {}
    for k in ("pos", "feat", "offsets", "scaling"):
        host["a_" + k] = torch.tensor(np.ascontiguousarray(anc[k]), dtype=torch.float32).pin_memory()
    for k in ("w1", "b1", "w2", "b2"):
        host["m_" + k] = torch.tensor(np.ascontiguousarray(mlp[k]), dtype=torch.float32).pin_memory()
    for k in ("color", "depth", "feat", "weight"):
        host["t_" + k] = torch.tensor(np.concatenate([t[k].reshape(-1) for t in tg]),
                                      dtype=torch.float32).pin_memory()
    out_loss = torch.zeros(1, dtype=torch.float32).pin_memory()
    out_pose = torch.zeros(st.d_pose.shape, dtype=torch.float32).pin_memory()
    sets = []
    for si in range(2):
        ad = st.ad if si == 0 else {k: v.clone() for k, v in st.ad.items()}
        md = st.md if si == 0 else {k: v.clone() for k, v in st.md.items()}
        tgt = st.tgt if si == 0 else {k: (v.clone() if v is not None else None) for k, v in st.tgt.items()}
        dev = {}
        for k in host:
            pre, name = k.split("_", 1)
            dev[k] = ad[name] if pre == "a" else md[name] if pre == "m" else tgt[name]
        sets.append(dict(ad=ad, md=md, tgt=tgt, dev=dev))
    h2d = sum(v.numel() * 4 for v in host.values())
    d2h = out_loss.numel() * 4 + out_pose.numel() * 4
    stream = torch.cuda.current_stream()
    copy = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]

    def put(si, after=None):
        with torch.cuda.stream(copy):
            if after is not None:
                copy.wait_event(after)
            for k, v in host.items():
                sets[si]["dev"][k].copy_(v, non_blocking=True)
            copied[si].record(copy)

    def steps(n):
        put(0)
        for i in range(n):
            si = i & 1
            stream.wait_event(copied[si])
            if i + 1 < n:
                put(si ^ 1, done[si ^ 1] if i >= 1 else None)
            st.ad, st.md, st.tgt = sets[si]["ad"], sets[si]["md"], sets[si]["tgt"]
            st.run()
            out_loss.copy_(st.loss, non_blocking=True)
            out_pose.copy_(st.d_pose, non_blocking=True)
            done[si].record(stream)

    steps(max(2, args.warmup // 2))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n = max(3, args.steps // 2)
    e0.record(stream)
    steps(n)
    e1.record(stream)
    torch.cuda.synchronize()
    st.ad, st.md, st.tgt = sets[0]["ad"], sets[0]["md"], sets[0]["tgt"]
    ms = e0.elapsed_time(e1) / n
    pix = sum(c.width * c.height for c in st.cams)
    return dict(value=round(world * pix / (ms / 1e3) / 1e6, 3), unit=UNIT, h2d_bytes_per_step=int(h2d),
                d2h_bytes_per_step=int(d2h), ms_per_step=round(ms, 4), steps=n,
                pipeline="inputs double-buffered: step i+1's host-to-device copy overlaps step i")


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg / reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(wl, anc, mlp, cams, tg, window):
    """FP64 oracle fwd+bwd of one view (optionally a centred window of it) with
    every anchor decoded; returns (pixels, seconds)."""
    import oracle
    from paper_2505_22335_gb300 import scenes
    c = cams[0]
    t = tg[0]
    if window is not None:
        ww, hh = window
        x0, y0 = (c.width - ww) // 2, (c.height - hh) // 2
        c = scenes.Camera(c.fx, c.fy, c.cx - x0, c.cy - y0, ww, hh, c.T_cw, c.t_norm)
        t = {k: (v[..., y0:y0 + hh, x0:x0 + ww]) for k, v in t.items()}
    t0 = time.perf_counter()
    oracle.backward_anchor(anc, mlp, [c], [t], oracle.RenderCfg(),
                           oracle.LossCfg(lambda_scale=LAMBDA_SCALE), wl["K"], wl["NF"])
    return c.width * c.height, time.perf_counter() - t0


def cpu_baseline(wl, anc, mlp, cams, tg):
    import oracle
    pix, sec = oracle_sample(wl, anc, mlp, cams, tg, None)
    return dict(value=round(pix / sec / 1e6, 5), unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                sample=f"one {cams[0].width}x{cams[0].height} view of the {wl['V']}-view batch, all "
                       f"{wl['A']} anchors decoded, FP64 fwd+bwd ({sec:.1f} s)")


def run_reference(args, wl_name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[wl_name]
    anc, mlp, cams, tg = make_inputs(wl, seed=0)
    n = args.steps + args.warmup
    window = (640, 480) if n <= 12 else (320, 240) if n <= 30 else (160, 120)
    window = (min(window[0], wl["W"]), min(window[1], wl["H"]))
    for _ in range(args.warmup):
        oracle_sample(wl, anc, mlp, cams, tg, window)
    tot_pix, tot_s = 0, 0.0
    for _ in range(args.steps):
        p, s = oracle_sample(wl, anc, mlp, cams, tg, window)
        tot_pix += p
        tot_s += s
    value = tot_pix / tot_s / 1e6
    sample = (f"{window[0]}x{window[1]} centre window of one view of the {wl['V']}-view batch per step, "
              f"all {wl['A']} anchors decoded, FP64 fwd+bwd")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * tot_s / args.steps, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_name, "anchors": wl["A"], "k": wl["K"], "views": wl["V"],
                       "width": wl["W"], "height": wl["H"], "n_feat": wl["NF"]},
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# serving mix: plain FIFO path vs continuous batching
# ---------------------------------------------------------------------------

SERVE = dict(A=500_000, K=10, NF=16, W=640, H=480, fx=600.0, track_rate=30.0, map_rate=5.0,
             levels=3, map_views=(4, 8))


def serving_schedule(seconds, seed=2, load=1.0):
    """Open-loop arrival schedule: (time_s, kind, n_views) sorted by time;
    `load` multiplies both arrival rates."""
    rng = np.random.default_rng(seed)
    ev = []
    for kind, rate in ((0, SERVE["track_rate"] * load), (1, SERVE["map_rate"] * load)):
        t = rng.exponential(1.0 / rate)
        while t < seconds:
            nv = 1 if kind == 0 else int(rng.integers(SERVE["map_views"][0], SERVE["map_views"][1] + 1))
            ev.append((t, kind, nv))
            t += rng.exponential(1.0 / rate)
    ev.sort()
    return ev


def run_serving(args):
    torch_line = measure_serving(args.serve_seconds)
    print(json.dumps(dict({"metric": "serving mix: fwd+bwd Mpixel/s and tracking p50/p99 latency, plain vs served",
                           "value": torch_line["served_mpix_per_s_saturated"], "unit": "Mpixel/s", "n_gpus": 1,
                           "higher_is_better": True, "dtype": "f32 (bf16 decode GEMMs)", "data": "synthetic"},
                          **torch_line)))


SATURATION_LOAD = 4.0     # arrival rates x4: more work offered than either path can finish
SATURATION_SECONDS = 3.0


def measure_serving(seconds):
    """The serving mix on one GPU, both paths on the same open-loop schedules:
    'plain' = one request per launch, FIFO, one slot; 'served' = continuous
    batching over two slots.
    * at the mix's own rates (30 tracking + 5 mapping requests/s) for
      `seconds`: p50/p99 latency (completion - scheduled arrival) per class;
    * at SATURATION_LOAD x those rates for SATURATION_SECONDS: more is offered
      than either path finishes, so completed pixels / makespan is each path's
      capacity in Mpixel/s (a schedule below capacity would show the offered
      load for both)."""
    import torch
    from paper_2505_22335_gb300 import binding as B
    from paper_2505_22335_gb300 import scenes
    torch.cuda.set_device(0)
    c = SERVE
    anc = scenes.anchors(0, c["A"], c["K"])
    mlp = scenes.mlp_weights(1000, c["K"], c["NF"])
    ad, md = B.anchors_to_device(anc, mlp)
    # request inputs from small pools (contents do not change the work)
    rng = np.random.default_rng(3)
    poses = scenes.arc_poses(4, 16)
    def cam(i):
        return scenes.Camera(c["fx"], c["fx"], c["W"] / 2, c["H"] / 2, c["W"], c["H"], poses[i % 16],
                             float(rng.uniform()))
    def pyr(cm):
        return [scenes.Camera(cm.fx / 2 ** l, cm.fy / 2 ** l, cm.cx / 2 ** l, cm.cy / 2 ** l, cm.width >> l,
                              cm.height >> l, cm.T_cw, cm.t_norm) for l in range(c["levels"])]
    track_tg = [B.targets_to_device(scenes.targets(10 + i, pyr(cam(i)), c["NF"], weighted=True)) for i in range(4)]
    map_tg = {nv: B.targets_to_device(scenes.targets(20 + nv, [cam(j) for j in range(nv)], c["NF"], weighted=True))
              for nv in range(c["map_views"][0], c["map_views"][1] + 1)}
    pix_track = sum((c["W"] >> l) * (c["H"] >> l) for l in range(c["levels"]))
    q = lambda a, p: round(float(np.percentile(np.array(a), p)), 2) if a else None

    def run_schedule(srv, submit, sched):
        lat = {0: [], 1: []}
        pending = {}
        t0 = time.perf_counter()
        done_pix = 0
        i = 0
        last_end = t0
        while i < len(sched) or pending:
            now = time.perf_counter() - t0
            while i < len(sched) and sched[i][0] <= now:
                ta, kind, nv = sched[i]
                t_sub = time.perf_counter()
                tk = submit(i, kind, nv)
                pending[tk] = (ta, kind, nv, t_sub)
                i += 1
            for tk in list(pending):
                res = srv.poll(tk)
                if res is None:
                    continue
                ta, kind, nv, t_sub = pending.pop(tk)
                # completion in this clock: submit time + (server end - server submit)
                t_end = (t_sub - t0) + (res["end_ms"] - res["submit_ms"]) / 1e3
                lat[kind].append((t_end - ta) * 1e3)
                done_pix += pix_track if kind == 0 else nv * c["W"] * c["H"]
                last_end = max(last_end, t0 + t_end)
            time.sleep(0.0002)
        wall = last_end - t0 - sched[0][0]
        return dict(mpix_per_s=round(done_pix / wall / 1e6, 2), tracking_p50_ms=q(lat[0], 50),
                    tracking_p99_ms=q(lat[0], 99), mapping_p50_ms=q(lat[1], 50), mapping_p99_ms=q(lat[1], 99),
                    requests=len(lat[0]) + len(lat[1]), makespan_s=round(wall, 3))

    scheds = dict(rate=serving_schedule(seconds), saturated=serving_schedule(SATURATION_SECONDS, seed=5,
                                                                           load=SATURATION_LOAD))
    out = {}
    for mode in ("plain", "served"):
        srv = B.Server(ad, md, n_feat=c["NF"], k=c["K"], slots=1 if mode == "plain" else 2,
                       max_batch_views=24, batching=(mode == "served"), memory_budget_gb=120.0,
                       decode_bf16=1)
        pool = [dict(loss=torch.zeros(1, device="cuda"), pose=torch.zeros(6 * 8, device="cuda"),
                     mlp={k: torch.zeros_like(v) for k, v in md.items()}) for _ in range(64)]
        def submit(i, kind, nv, cams=None):
            o = pool[i % len(pool)]
            if kind == 0:
                cm = cam(i)
                return srv.submit(B.TRACK, [cm], track_tg[i % 4], o["loss"], o["pose"], levels=c["levels"])
            cms = [cam(i + j) for j in range(nv)]
            return srv.submit(B.MAP, cms, map_tg[nv], o["loss"], o["pose"], d_mlp=o["mlp"])
        # warm-up: every request shape once
        for i, (kind, nv) in enumerate([(0, 1)] + [(1, v) for v in map_tg]):
            srv.wait(submit(1000 + i, kind, nv))
        srv.wait_idle()
        torch.cuda.synchronize()
        out[mode] = {name: run_schedule(srv, submit, sc) for name, sc in scheds.items()}
        srv.close()
    del ad, md, track_tg, map_tg
    torch.cuda.empty_cache()
    plain, served = out["plain"], out["served"]
    better = (served["saturated"]["mpix_per_s"] > plain["saturated"]["mpix_per_s"]
              and served["rate"]["tracking_p99_ms"] < plain["rate"]["tracking_p99_ms"])
    return {"config": {"workload": f"serving_mix_{c['A'] // 1000}k_anchors_x{c['K']}",
                       "tracking": f"{c['track_rate']}/s, {c['levels']} pyramid levels from {c['W']}x{c['H']}, "
                                   f"fwd + pose-only bwd",
                       "mapping": f"{c['map_rate']}/s, {c['map_views'][0]}-{c['map_views'][1]} keyframes "
                                  f"{c['W']}x{c['H']}, full bwd",
                       "decode": "bf16 tensor cores", "arrivals": "open-loop Poisson",
                       "rate_schedule": f"the mix's rates for {seconds} s (seed 2): latency",
                       "saturated_schedule": f"{SATURATION_LOAD:g}x the rates for {SATURATION_SECONDS:g} s (seed 5): "
                                             f"capacity, completed pixels / makespan",
                       "latency": "completion - scheduled arrival"},
            "plain": plain, "served": served,
            "served_mpix_per_s_saturated": served["saturated"]["mpix_per_s"],
            "plain_mpix_per_s_saturated": plain["saturated"]["mpix_per_s"],
            "served_beats_plain_in_mpix_and_tracking_p99": bool(better)}


def run_only(args):
    """One part of the bench on its own, for profiler captures: no timed step,
    no JSON contract line (prints a short JSON summary)."""
    import torch
    torch.cuda.set_device(0)
    wl = WORKLOADS[args.workload]
    anc, mlp, cams, tg = make_inputs(wl, seed=0)
    if args.only == "anchor_update":
        res = run_anchor(args, wl, anc, cams[0])
    else:
        st = Step(wl, anc, mlp, cams, tg, 0, bf16=args.decode_bf16)
        for _ in range(args.warmup):
            st.run()
        torch.cuda.synchronize()
        res = dict(tracking_uncertainty=run_uncertainty(args, st, wl), feature_lifting=run_lift(args, st, wl),
                   dssim=run_ssim(args, st, wl), uncertainty_mlp=run_unc_mlp(args, st, wl))
    print(json.dumps(dict(only=args.only, workload=args.workload, result=res)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--decode-bf16", action="store_true",
                    help="decode MLP GEMMs in BF16 on the tensor cores (FP32 accumulation)")
    ap.add_argument("--serving", action="store_true",
                    help="serving mix (500k anchors resident): plain FIFO path vs continuous batching")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--no-serving", action="store_true",
                    help="leave the serving-mix comparison out of the default line")
    ap.add_argument("--only", choices=["anchor_update", "next_rows"], default=None,
                    help="run only one part (for profiler captures): the anchor update on the default "
                         "workload's anchors, or the next-row entry points on one step's images")
    args = ap.parse_args()
    if args.only:
        from paper_2505_22335_gb300 import build as _b
        _b.build()
        run_only(args)
        return
    if args.serving:
        from paper_2505_22335_gb300 import build as _b
        _b.build()
        run_serving(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        import oracle
        oracle.build()
        run_reference(args, args.workload)
        return
    from paper_2505_22335_gb300 import build as _b
    _b.build()
    import oracle
    oracle.build()
    run_ours(args, args.workload)


if __name__ == "__main__":
    main()
