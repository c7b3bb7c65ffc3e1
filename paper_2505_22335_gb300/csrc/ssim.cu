// The D-SSIM term of the geometric loss (Eq. 4): scale (1 - SSIM(C~, C)), each
// pixel's (1 - S) weighted by an optional per-pixel weight (the mask of Eq. 14),
// SSIM (Wang et al.) per colour channel of every view with an 11 x 11
// Gaussian window (sigma 1.5, weights summing to 1), C1 = 0.01^2, C2 = 0.03^2
// (data range 1), zero padding, averaged over channels and pixels.
//
// With the window moments mu_x, mu_y, E[x^2], E[y^2], E[xy] of pixel p:
//   A1 = 2 mu_x mu_y + C1, A2 = 2 (E[xy] - mu_x mu_y) + C2,
//   B1 = mu_x^2 + mu_y^2 + C1, B2 = E[x^2] - mu_x^2 + E[y^2] - mu_y^2 + C2,
//   S = A1 A2 / (B1 B2)
// and dS_p/dx_q = w(q - p) (G_mu + 2 x_q G_xx + y_q G_xy)(p) with
//   G_mu = S (2 mu_y / A1 - 2 mu_y / A2 - 2 mu_x / B1 + 2 mu_x / B2),
//   G_xx = -S / B2,  G_xy = 2 S / A2,
// so the backward correlates the three G maps with the (symmetric) window.
//
// Two launches (forward, backward) over all (view, channel) planes, 32 x 16
// output tiles: the input tile with its 5-pixel halo is staged in shared
// memory, a horizontal then a vertical 11-tap pass form the window sums.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace ups {

namespace {

constexpr int kR = 5;                 // window radius
constexpr int kTX = 32, kTY = 16;     // output tile
constexpr int kIX = kTX + 2 * kR, kIY = kTY + 2 * kR;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

__constant__ float c_win[2 * kR + 1];  // 1-D Gaussian window, sums to 1

// the (view, channel) planes of one call: blockIdx.z selects the plane
constexpr int kMaxPlanes = 3 * UPS_MAX_VIEWS;
struct Planes {
    int n;
    int W[kMaxPlanes], H[kMaxPlanes];
    size_t off[kMaxPlanes];   // offset of the plane's pixel 0 in the colour arrays
    size_t goff[kMaxPlanes];  // offset of its window-term maps in G (3 maps of W * H)
    size_t woff[kMaxPlanes];  // offset of its view's pixel 0 in the weight map
};
struct Plane {
    int W, H;
    size_t off, goff, woff;
};
__device__ __forceinline__ Plane plane_of(const Planes &t) {
    const int z = blockIdx.z;
    return Plane{t.W[z], t.H[z], t.off[z], t.goff[z], t.woff[z]};
}

// horizontal then vertical window sums of NQ staged quantities
template <int NQ>
__device__ __forceinline__ void window_sums(const float (&in)[NQ][kIY][kIX], float (&hs)[NQ][kIY][kTX],
                                           float (&out)[2][NQ]) {
    const int tid = threadIdx.x;
    for (int i = tid; i < kIY * kTX; i += blockDim.x) {
        const int r = i / kTX, cx = i - r * kTX;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * kR; ++k) s = fmaf(c_win[k], in[q][r][cx + k], s);
            hs[q][r][cx] = s;
        }
    }
    __syncthreads();
    // each thread: outputs (tid % 32, tid / 32) and (tid % 32, tid / 32 + 8)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int ox = tid & (kTX - 1), oy = (tid >> 5) + 8 * h;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * kR; ++k) s = fmaf(c_win[k], hs[q][oy + k][ox], s);
            out[h][q] = s;
        }
    }
}

__global__ void __launch_bounds__(256) k_ssim_fwd(const Planes pt, const float *__restrict__ x,
                                                  const float *__restrict__ y, const float *__restrict__ weight,
                                                  float *__restrict__ Gall, float g, float *__restrict__ loss) {
    __shared__ float in[5][kIY][kIX];
    __shared__ float hs[5][kIY][kTX];
    const Plane pl = plane_of(pt);
    if ((int)blockIdx.x * kTX >= pl.W || (int)blockIdx.y * kTY >= pl.H) return;  // grid sized for the largest plane
    float *G = Gall + pl.goff;
    const size_t gstride = (size_t)pl.W * pl.H;
    const int x0 = blockIdx.x * kTX - kR, y0 = blockIdx.y * kTY - kR;
    for (int i = threadIdx.x; i < kIY * kIX; i += blockDim.x) {
        const int r = i / kIX, cx = i - r * kIX;
        const int gx = x0 + cx, gy = y0 + r;
        float a = 0.f, b = 0.f;
        if (gx >= 0 && gx < pl.W && gy >= 0 && gy < pl.H) {
            a = x[pl.off + (size_t)gy * pl.W + gx];
            b = y[pl.off + (size_t)gy * pl.W + gx];
        }
        in[0][r][cx] = a;
        in[1][r][cx] = b;
        in[2][r][cx] = a * a;
        in[3][r][cx] = b * b;
        in[4][r][cx] = a * b;
    }
    __syncthreads();
    float m[2][5];
    window_sums<5>(in, hs, m);
    float term = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int px = blockIdx.x * kTX + (threadIdx.x & (kTX - 1));
        const int py = blockIdx.y * kTY + (threadIdx.x >> 5) + 8 * h;
        if (px >= pl.W || py >= pl.H) continue;
        const float mx = m[h][0], my = m[h][1];
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * (m[h][4] - mx * my) + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = (m[h][2] - mx * mx) + (m[h][3] - my * my) + kC2;
        const float S = (A1 * A2) / (B1 * B2);
        const size_t lp = (size_t)py * pl.W + px;  // the G maps are per plane
        const float wp = weight ? weight[pl.woff + lp] : 1.f;
        term += wp * (1.f - S);
        G[lp] = wp * S * (2.f * my / A1 - 2.f * my / A2 - 2.f * mx / B1 + 2.f * mx / B2);
        G[gstride + lp] = wp * (-S / B2);
        G[2 * gstride + lp] = wp * (2.f * S / A2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += red[w];
        atomicAdd(loss, g * t);
    }
}

// dx_q += -g (w * G_mu + 2 x_q w * G_xx + y_q w * G_xy)(q)
__global__ void __launch_bounds__(256) k_ssim_bwd(const Planes pt, const float *__restrict__ x,
                                                  const float *__restrict__ y, const float *__restrict__ Gall,
                                                  float g, float *__restrict__ dx) {
    __shared__ float in[3][kIY][kIX];
    __shared__ float hs[3][kIY][kTX];
    const Plane pl = plane_of(pt);
    if ((int)blockIdx.x * kTX >= pl.W || (int)blockIdx.y * kTY >= pl.H) return;
    const float *G = Gall + pl.goff;
    const size_t gstride = (size_t)pl.W * pl.H;
    const int x0 = blockIdx.x * kTX - kR, y0 = blockIdx.y * kTY - kR;
    for (int i = threadIdx.x; i < kIY * kIX; i += blockDim.x) {
        const int r = i / kIX, cx = i - r * kIX;
        const int gx = x0 + cx, gy = y0 + r;
        const bool ok = gx >= 0 && gx < pl.W && gy >= 0 && gy < pl.H;
        const size_t lp = (size_t)(ok ? gy : 0) * pl.W + (ok ? gx : 0);
#pragma unroll
        for (int q = 0; q < 3; ++q) in[q][r][cx] = ok ? G[q * gstride + lp] : 0.f;
    }
    __syncthreads();
    float m[2][3];
    window_sums<3>(in, hs, m);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int px = blockIdx.x * kTX + (threadIdx.x & (kTX - 1));
        const int py = blockIdx.y * kTY + (threadIdx.x >> 5) + 8 * h;
        if (px >= pl.W || py >= pl.H) continue;
        const size_t p = pl.off + (size_t)py * pl.W + px;
        dx[p] -= g * (m[h][0] + 2.f * x[p] * m[h][1] + y[p] * m[h][2]);
    }
}

}  // namespace

cudaError_t ssim_set_window() {
    float w[2 * kR + 1], s = 0.f;
    for (int k = -kR; k <= kR; ++k) s += (w[k + kR] = std::exp(-(float)(k * k) / (2.f * 1.5f * 1.5f)));
    for (float &v : w) v /= s;
    return cudaMemcpyToSymbol(c_win, w, sizeof(w));
}

// Every colour plane of the views in one launch per direction: adds g w (1 - S)
// over all planes to *loss and, if dx, its derivative to dx (w: the per-pixel
// weight of the view's pixels, 1 when null).  G: scratch of 3 x (sum
// of the planes' pixels) floats.
cudaError_t launch_ssim(const ViewTable &vt, const float *x, const float *y, const float *weight, float *G, float g,
                        float *loss, float *dx, cudaStream_t st) {
    Planes pt{};
    int maxw = 0, maxh = 0;
    size_t goff = 0;
    for (int v = 0; v < vt.n; ++v)
        for (int ch = 0; ch < 3; ++ch) {
            const int i = pt.n++;
            pt.W[i] = vt.v[v].W;
            pt.H[i] = vt.v[v].H;
            const size_t HW = (size_t)pt.W[i] * pt.H[i];
            pt.off[i] = 3 * (size_t)vt.v[v].pix_off + ch * HW;
            pt.goff[i] = goff;
            pt.woff[i] = (size_t)vt.v[v].pix_off;
            goff += 3 * HW;
            maxw = std::max(maxw, pt.W[i]);
            maxh = std::max(maxh, pt.H[i]);
        }
    if (pt.n == 0) return cudaSuccess;
    const dim3 grid((maxw + kTX - 1) / kTX, (maxh + kTY - 1) / kTY, pt.n), blk(256);
    k_ssim_fwd<<<grid, blk, 0, st>>>(pt, x, y, weight, G, g, loss);
    if (dx) k_ssim_bwd<<<grid, blk, 0, st>>>(pt, x, y, G, g, dx);
    return cudaGetLastError();
}

}  // namespace ups
