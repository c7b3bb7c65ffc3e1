// Uncertainty MLP F_u and its loss L_u (Sec. 3.3 "Uncertainty Prediction for
// Mapping", Eq. 5, Eq. 13; App. "MLP Implementation Details"):
//   sigma_p = SoftPlus(w2 . ReLU(W1 F_p + b1) + b2)   (1x1 conv -> ReLU -> 1x1
//   conv -> SoftPlus, hidden 128, one output), F_p the DINO feature of pixel
//   p bilinearly upsampled from the patch grid, and
//   L_u = (1 / P) sum_p [R_p / (2 sigma_p^2) + lambda log sigma_p]   (Eq. 5),
// with the gradient flowing only into F_u's parameters (the mapping and
// uncertainty gradient flows are kept apart, Sec. 3.3).
//
// The first layer is linear, so W1 F_p = sum_c a_c(p) (W1 g_c) over the
// pixel's four patch corners g_c with bilinear weights a_c(p): it runs once
// per patch (Zp = G W1^T, a small GEMM in plain FP32: the pedantic compute
// type keeps the library from reduced-precision tensor paths), and every pixel interpolates
// 128 values instead of 384.  Backward, dW1 = sum_p dh_p F_p^T = D^T G with
// D_patch = sum over (pixel, corner) pairs landing on the patch of a_c(p)
// dh_p, so the second small GEMM runs on patches too.
//
// The pixel kernel: one CTA per cell of pixels that share their four corner
// patches, one warp per pixel at a time, each lane owning 4 of the 128 hidden
// units; the per-lane sums (dW2, db1, D of the four corners) are reduced over
// the CTA and added once.
#include <algorithm>

#include "common.cuh"

namespace ups {

namespace {

constexpr int kUH = 128;     // hidden units
constexpr int kUWarps = 4;   // warps per cell CTA

__device__ __forceinline__ float softplus_f(float x) { return x > 20.f ? x : log1pf(__expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.f / (1.f + __expf(-x)); }

// first patch index along an axis of n pixels whose bilinear position
// floor(clamp((x + 0.5) / patch - 0.5, 0, np - 1)) is at least i
__device__ __forceinline__ int cell_start(int i, int patch) {
    // (x + 0.5) / patch - 0.5 >= i  <=>  x >= i * patch + (patch - 1) / 2
    return i == 0 ? 0 : (int)ceilf((float)i * patch + 0.5f * (float)(patch - 1) - 1e-4f);
}

// grid: (cells_x, cells_y) of one view; cell (i, j) = the pixels whose
// floor(u) = i and floor(v) = j (u, v their clamped grid positions).
__global__ void __launch_bounds__(32 * kUWarps) k_unc_cells(
    int W, int H, int wp, int hp, int patch, const float *__restrict__ Zp, const float *__restrict__ b1,
    const float *__restrict__ w2, const float *__restrict__ b2, const float *__restrict__ R, float lambda, float g,
    float *__restrict__ loss, float *__restrict__ sigma_out, uint8_t *__restrict__ motion_out,
    float *__restrict__ d_b1, float *__restrict__ d_w2, float *__restrict__ d_b2, float *__restrict__ D) {
    __shared__ __align__(16) float zc[4][kUH];  // the four corner patches' W1 g
    __shared__ float red[kUWarps][6][kUH];  // per-warp sums: d_w2, d_b1, D[4]
    __shared__ float sred[kUWarps][2];      // loss, d_b2
    const int ci = blockIdx.x, cj = blockIdx.y;
    const int x0 = min(ci, wp - 1), y0 = min(cj, hp - 1);
    const int x1 = min(x0 + 1, wp - 1), y1 = min(y0 + 1, hp - 1);
    const int corner[4] = {y0 * wp + x0, y0 * wp + x1, y1 * wp + x0, y1 * wp + x1};
    for (int i = threadIdx.x; i < 4 * kUH; i += blockDim.x) zc[i / kUH][i % kUH] = Zp[(size_t)corner[i / kUH] * kUH + i % kUH];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // pixel range of the cell (the last cell along an axis runs to the border)
    const int xs = cell_start(ci, patch), xe = ci + 1 >= wp ? W : min(W, cell_start(ci + 1, patch));
    const int ys = cell_start(cj, patch), ye = cj + 1 >= hp ? H : min(H, cell_start(cj + 1, patch));
    const int nx = max(0, xe - xs), npx = nx * max(0, ye - ys);
    float bb1[4], ww2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        bb1[k] = b1[4 * lane + k];
        ww2[k] = w2[4 * lane + k];
    }
    const float bb2 = b2[0];
    float a_dw2[4] = {0.f, 0.f, 0.f, 0.f}, a_db1[4] = {0.f, 0.f, 0.f, 0.f};
    float a_D[4][4] = {};
    float a_loss = 0.f, a_db2 = 0.f;
    const float inv2p = 1.f / (float)(2 * patch);
    // the warp's pixels q = w, w + kUWarps, ... in row-major order over the cell,
    // their coordinates stepped from the first
    int y = ys + (nx > 0 ? w / nx : 0), x = xs + (nx > 0 ? w % nx : 0);
    for (int q = w; q < npx; q += kUWarps) {
        // bilinear weight u - x0 = ((2x + 1) - (2 x0 + 1) patch) / (2 patch): an exact
        // integer numerator, one rounding (u itself is ~45 at 640 px, where a float
        // ulp would already move the weight by 4e-6); clamped positions give 0
        // (and at the far edge x1 == x0)
        const float ax = fminf(fmaxf((float)(2 * x + 1 - (2 * x0 + 1) * patch) * inv2p, 0.f), 1.f);
        const float ay = fminf(fmaxf((float)(2 * y + 1 - (2 * y0 + 1) * patch) * inv2p, 0.f), 1.f);
        const float a[4] = {(1.f - ax) * (1.f - ay), ax * (1.f - ay), (1.f - ax) * ay, ax * ay};
        float z[4], h[4], part = 0.f;
        const float4 z0 = *reinterpret_cast<const float4 *>(&zc[0][4 * lane]);
        const float4 z1 = *reinterpret_cast<const float4 *>(&zc[1][4 * lane]);
        const float4 z2v = *reinterpret_cast<const float4 *>(&zc[2][4 * lane]);
        const float4 z3 = *reinterpret_cast<const float4 *>(&zc[3][4 * lane]);
        const float c0[4] = {z0.x, z0.y, z0.z, z0.w}, c1[4] = {z1.x, z1.y, z1.z, z1.w};
        const float c2[4] = {z2v.x, z2v.y, z2v.z, z2v.w}, c3[4] = {z3.x, z3.y, z3.z, z3.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            z[k] = bb1[k] + a[0] * c0[k] + a[1] * c1[k] + a[2] * c2[k] + a[3] * c3[k];
            h[k] = fmaxf(z[k], 0.f);
            part = fmaf(ww2[k], h[k], part);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const float z2 = part + bb2;
        const float s = softplus_f(z2);
        const size_t p = (size_t)y * W + x;
        const float r = R[p];
        // L_u = R / (2 s^2) + lambda log s;  dL_u/ds = -R / s^3 + lambda / s = (lambda - R / s^2) / s
        const float is = 1.f / s;
        const float ds = g * is * (lambda - r * is * is);
        const float dz2 = ds * sigmoid_f(z2);
        if (lane == 0) {
            a_loss += r / (2.f * s * s) + lambda * logf(s);
            a_db2 += dz2;
            if (sigma_out) sigma_out[p] = s;
            if (motion_out) motion_out[p] = 2.f * s * s > 1.f ? 1 : 0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a_dw2[k] = fmaf(dz2, h[k], a_dw2[k]);
            const float dh = z[k] > 0.f ? dz2 * ww2[k] : 0.f;
            a_db1[k] += dh;
#pragma unroll
            for (int c = 0; c < 4; ++c) a_D[c][k] = fmaf(a[c], dh, a_D[c][k]);
        }
        x += kUWarps;
        while (x >= xe) {
            x -= nx;
            ++y;
        }
    }
    // reduce over the CTA's warps, then one atomic per value
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        red[w][0][4 * lane + k] = a_dw2[k];
        red[w][1][4 * lane + k] = a_db1[k];
#pragma unroll
        for (int c = 0; c < 4; ++c) red[w][2 + c][4 * lane + k] = a_D[c][k];
    }
    if (lane == 0) {
        sred[w][0] = a_loss;
        sred[w][1] = a_db2;
    }
    __syncthreads();
    if (npx == 0) return;
    for (int i = threadIdx.x; i < 6 * kUH; i += blockDim.x) {
        const int t = i / kUH, j = i % kUH;
        float s = 0.f;
#pragma unroll
        for (int ww = 0; ww < kUWarps; ++ww) s += red[ww][t][j];
        if (t == 0) {
            if (d_w2) atomicAdd(d_w2 + j, s);
        } else if (t == 1) {
            if (d_b1) atomicAdd(d_b1 + j, s);
        } else if (D) {
            atomicAdd(D + (size_t)corner[t - 2] * kUH + j, s);
        }
    }
    if (threadIdx.x == 0) {
        float l = 0.f, b = 0.f;
        for (int ww = 0; ww < kUWarps; ++ww) {
            l += sred[ww][0];
            b += sred[ww][1];
        }
        atomicAdd(loss, g * l);
        if (d_b2) atomicAdd(d_b2, b);
    }
}

}  // namespace

size_t unc_scratch_floats(int max_patches) { return (size_t)2 * max_patches * kUH; }

// One view: sigma, motion mask, loss and the F_u gradients (accumulated; any
// gradient pointer may be null).  grid: the view's patch grid [hp][wp][nh];
// R, sigma, motion: the view's pixels; scratch: unc_scratch_floats(hp * wp).
cudaError_t unc_view(int num_sms, cudaStream_t st, int W, int H, int nh, int patch, const float *grid, int wp,
                     int hp, const float *R, const float *w1, const float *b1, const float *w2, const float *b2,
                     float lambda, float g, float *loss, float *d_w1, float *d_b1, float *d_w2, float *d_b2,
                     float *sigma, uint8_t *motion, float *scratch, int *launches) {
    const int np = wp * hp;
    float *Zp = scratch;                     // [np][128]  W1 g of every patch
    float *D = scratch + (size_t)np * kUH;   // [np][128]  interpolation-weighted dL/dh per patch
    cudaError_t e;
    // Zp (column-major [128 x np]) = W1 [128 x nh] G^T
    if ((e = gemm_f32(st, true, false, kUH, np, nh, 1.f, w1, nh, grid, nh, 0.f, Zp, kUH, num_sms, launches)) != cudaSuccess) return e;
    if (d_w1 && (e = cudaMemsetAsync(D, 0, (size_t)np * kUH * sizeof(float), st)) != cudaSuccess) return e;
    k_unc_cells<<<dim3(wp, hp), 32 * kUWarps, 0, st>>>(W, H, wp, hp, patch, Zp, b1, w2, b2, R, lambda, g, loss, sigma,
                                                       motion, d_b1, d_w2, d_b2, d_w1 ? D : nullptr);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // dW1 (column-major [nh x 128], i.e. [128][nh] row-major) += G^T D
    if (d_w1 && (e = gemm_f32(st, false, true, nh, kUH, np, 1.f, grid, nh, D, kUH, 1.f, d_w1, nh, num_sms, launches)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

}  // namespace ups
