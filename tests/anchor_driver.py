"""Driver of the anchor-update kernel profile (profiles/anchor_update_100k_anchors_640x480.md): the
probabilistic anchor update (Eq. 7, prune, insert) of 100,000 seeded anchors (k = 10) against one
seeded synthetic 640x480 keyframe, three calls.  Run from the repository root on a GPU; not a test."""
import sys

import numpy as np
import torch

sys.path.insert(0, ".")
from paper_2505_22335_gb300 import binding as B, scenes

cam = scenes.cameras(0, 8, 640, 480, 600.0)[0]  # view 0 of the mapping bench batch
anc = scenes.anchors(0, 100_000, 10)
depth, motion = scenes.keyframe(7, cam)
t = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
ga = {k: t(anc[k]) for k in ("pos", "feat", "offsets", "scaling")}
lo = t(np.random.default_rng(8).uniform(-2.5, 3.5, 100_000))
R = B.Renderer(n_feat=16, k=10)
for _ in range(3):
    _, _, _, cnt = R.anchor_update(ga, lo, cam, t(depth), t(motion, torch.uint8), capacity=200_000)
torch.cuda.synchronize()
print("ok", cnt)
