// Training-free tracking uncertainty (Sec. 3.4 "Tracking"): the multi-modal
// residual R of Eq. 6 per pixel of the rendered views, and the per-pixel
// minimiser of Eq. 15, 1/2 (R / sigma^2 + log sigma), which is sigma^2 = 2R;
// the motion mask 2 sigma^2 > 1 is then R > 1/4.
//
//   R = (T < t_mask) (lc |C~ - C|_1 + ld |D~ - B(D)| + lf min(1, 1 - cos(F, F~)))
//
// T is the final transmittance (Eq. 3's T~ read as transmittance, so the mask
// keeps covered pixels), |.|_1 sums the three colour channels, B is the 3x3
// box filter of the target depth (the mean over the window's pixels inside
// the view) and cos = 0 when either feature vector is zero.
//
// One thread per pixel, views along grid.y: HBM-bound (reads the rendered
// images and the targets once, the 3x3 depth window through L1).
#include "common.cuh"

namespace ups {

namespace {

template <int NF>
__global__ void __launch_bounds__(256) k_uncertainty(ViewTable vt, float lc, float ld, float lf, float t_mask,
                                                     const float *__restrict__ color, const float *__restrict__ depth,
                                                     const float *__restrict__ feat, const float *__restrict__ T,
                                                     const float *__restrict__ t_color,
                                                     const float *__restrict__ t_depth,
                                                     const float *__restrict__ t_feat, float *__restrict__ R_out,
                                                     float *__restrict__ sigma2_out,
                                                     uint8_t *__restrict__ motion_out) {
    const DevView &cam = vt.v[blockIdx.y];
    const int W = cam.W, H = cam.H;
    const size_t HW = (size_t)W * H;
    const size_t P = (size_t)cam.pix_off;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= HW) return;
    const int y = (int)(p / (size_t)W), x = (int)(p - (size_t)y * W);
    float R = 0.f;
    if (T[P + p] < t_mask) {
        float rc = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) rc += fabsf(color[3 * P + c * HW + p] - t_color[3 * P + c * HW + p]);
        // 3x3 box filter of the target depth over the window's in-view pixels
        float bs = 0.f;
        int bn = 0;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int yy = y + dy, xx = x + dx;
                if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                    bs += t_depth[P + (size_t)yy * W + xx];
                    ++bn;
                }
            }
        const float rd = fabsf(depth[P + p] - bs / (float)bn);
        float rf = 0.f;
        if (NF > 0) {
            float dot = 0.f, na = 0.f, nb = 0.f;
#pragma unroll
            for (int c = 0; c < NF; ++c) {
                const float a = t_feat[NF * P + c * HW + p], b = feat[NF * P + c * HW + p];
                dot = fmaf(a, b, dot);
                na = fmaf(a, a, na);
                nb = fmaf(b, b, nb);
            }
            const float cs = na > 0.f && nb > 0.f ? dot * rsqrtf(na) * rsqrtf(nb) : 0.f;
            rf = fminf(1.f, 1.f - cs);
        }
        R = lc * rc + ld * rd + lf * rf;
    }
    if (R_out) R_out[P + p] = R;
    if (sigma2_out) sigma2_out[P + p] = 2.f * R;
    if (motion_out) motion_out[P + p] = R > 0.25f ? 1 : 0;
}

}  // namespace

cudaError_t launch_uncertainty(const ViewTable &vt, int n_feat, int max_hw, float lc, float ld, float lf,
                               float t_mask, const ups_images &img, const ups_targets &tgt, float *R, float *sigma2,
                               uint8_t *motion, cudaStream_t st) {
    if (vt.n <= 0 || max_hw <= 0) return cudaSuccess;
    dim3 grid((max_hw + 255) / 256, vt.n), block(256);
#define UPS_UNC(NFV)                                                                                         \
    k_uncertainty<NFV><<<grid, block, 0, st>>>(vt, lc, ld, lf, t_mask, img.color, img.depth, img.feat, img.T, \
                                               tgt.color, tgt.depth, tgt.feat, R, sigma2, motion)
    switch (n_feat) {
        case 0: UPS_UNC(0); break;
        case 16: UPS_UNC(16); break;
        case 32: UPS_UNC(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef UPS_UNC
    return cudaGetLastError();
}

}  // namespace ups
