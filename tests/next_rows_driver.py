"""Driver of the next-row kernel profile (profiles/next_rows_kernels_8x640x480.md): one forward on
eight 640x480 views, then the tracking uncertainty, D-SSIM, uncertainty MLP and feature lifting
entry points twice, on seeded synthetic inputs.  Run from the repository root on a GPU; not a test."""
import sys, torch
sys.path.insert(0, "."); sys.path.insert(0, "tests")
from paper_2505_22335_gb300 import binding as B, scenes
from gpu_cases import round_cams
cams = round_cams(scenes.cameras(0, 8, 640, 480, 600.0))
R = B.Renderer(n_feat=16, k=1)
img = R.forward(B.to_set(scenes.plain_gaussians(0, 2000, 16)), cams)
img["T"].zero_()  # every pixel covered: the residual reads everything
P = 8 * 640 * 480
g = torch.Generator(device="cuda").manual_seed(0)
tgt = dict(color=torch.rand(3 * P, generator=g, device="cuda"), depth=torch.rand(P, generator=g, device="cuda") + 1,
           feat=torch.randn(16 * P, generator=g, device="cuda"))
nh, patch = 384, 14
dino = torch.randn(8 * 35 * 46 * nh, generator=g, device="cuda")
lm = dict(w1=torch.randn(128, 16, device="cuda") * 0.3, b1=torch.zeros(128, device="cuda"),
          w2=torch.randn(nh, 128, device="cuda") * 0.1, b2=torch.zeros(nh, device="cuda"))
um = dict(w1=torch.randn(128, nh, device="cuda") * 0.1, b1=torch.zeros(128, device="cuda"),
          w2=torch.randn(128, device="cuda") * 0.2, b2=torch.full((1,), 0.2, device="cuda"))
dl = {k: torch.zeros_like(v) for k, v in lm.items()}
du = {k: torch.zeros_like(v) for k, v in um.items()}
dcol = torch.zeros(3 * P, device="cuda")
dfe = torch.zeros(16 * P, device="cuda")
for _ in range(2):
    out = R.tracking_uncertainty(img, tgt)
    R.ssim_loss(img["color"], tgt["color"], d_color=dcol)
    R.uncertainty_mlp(dino, out["R"], um, n_h=nh, patch=patch, d_mlp=du)
    R.feature_lift(img["feat"], dino, lm, n_h=nh, patch=patch, d_mlp=dl, d_feat=dfe)
torch.cuda.synchronize()
print("ok")
