// Feature lifting F_m and the distillation loss L_d (Sec. 3.3, Eq. 11, Eq. 12;
// App. "MLP Implementation Details"): the rendered N_l-channel feature map F~
// goes through a per-pixel (1x1 convolution) MLP N_l -> 128 -> ReLU -> N_h to
// F^, compared by cosine with the DINO feature F of the pixel, bilinearly
// upsampled from the view's patch grid (Sec. 3.2):
//   L_d = (1 / P) sum_p (1 - cos(F_p, F^_p)),   cos = 0 where a vector is 0.
//
// F^ = W2 H + b2 is never formed.  F_p = sum_k w_k g_{c_k} over the four patch
// vectors around p, so with E = G W2 (row c: W2^T g_c), s = G b2, M = W2^T W2,
// u = W2^T b2 and e_p = sum_k w_k E_{c_k}:
//   F^_p . F_p = H_p . e_p + sum_k w_k s_{c_k}
//   |F^_p|^2   = H_p . (M H_p) + 2 u . H_p + |b2|^2
//   |F_p|^2    = w^T Gram(g_{c_0..3}) w        (Gram per cell of the patch grid)
// and with dL/dF^_p = a_p F_p + b_p F^_p (a_p = -g / (|F| |F^|),
// b_p = g cos / |F^|^2):
//   dL/dH_p = a_p e_p + b_p (M H_p + u)
//   dW2 = G^T D + W2 (sum_p b_p H_p H_p^T) + b2 (sum_p b_p H_p)^T,
//         D_c = sum of a_p w_k H_p over the (p, k) with c_k = c
//   db2 = G^T alpha + W2 sum_p b_p H_p + b2 sum_p b_p,  alpha_c = sum a_p w_k.
// Every per-pixel quantity is 128 wide: ~80 kFLOP per pixel instead of
// ~310 k, and no N_h-wide per-pixel array.
//
// The pixel-sized products (F~ W1^T, H M, (bH)^T H and the two backward
// products with W1) run as cuBLAS TF32 GEMMs on the planar image layout
// (channel c of pixel p at [c * HW + p] is a column-major HW x C matrix); the
// small per-patch and weight-sized ones in FP32 (pedantic); one kernel per
// cell of pixels sharing their four patches does the cosine, the loss, dL/dZ
// and the per-patch sums.
#include "common.cuh"

namespace ups {

namespace {

constexpr int kLiftHidden = 128;

__global__ void k_bias_relu(float *__restrict__ z, const float *__restrict__ b, size_t HW) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= HW) return;
    float *row = z + (size_t)blockIdx.y * HW;
    row[p] = fmaxf(row[p] + b[blockIdx.y], 0.f);
}

// out[r] += sum_p m[r * HW + p]: blockIdx.y = row, blockIdx.x = a chunk of
// kSumChunk pixels, one atomic per block
constexpr int kSumChunk = 8192;
__global__ void __launch_bounds__(256) k_row_sums(const float *__restrict__ m, size_t HW, float *__restrict__ out) {
    const float *row = m + (size_t)blockIdx.y * HW;
    const size_t p0 = (size_t)blockIdx.x * kSumChunk;
    const size_t p1 = min(HW, p0 + kSumChunk);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    size_t p = p0 + threadIdx.x;
    for (; p + 768 < p1; p += 1024) {
        s0 += row[p];
        s1 += row[p + 256];
        s2 += row[p + 512];
        s3 += row[p + 768];
    }
    for (; p < p1; p += 256) s0 += row[p];
    float s = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(out + blockIdx.y, t);
    }
}

// first pixel index along an axis whose clamped bilinear position
// floor(clamp((x + 0.5) / patch - 0.5, 0, n - 1)) is at least i
__device__ __forceinline__ int cell_start(int i, int patch) {
    // (x + 0.5) / patch - 0.5 >= i  <=>  x >= i * patch + (patch - 1) / 2
    return i == 0 ? 0 : (int)ceilf((float)i * patch + 0.5f * (float)(patch - 1) - 1e-4f);
}

// Gram matrix of the four corner patches of every cell (x0, y0) of the grid
// (x1 = min(x0 + 1, wp - 1), y1 likewise): gram[cell][10] = g00.g00, g00.g01,
// g00.g10, g00.g11, g01.g01, g01.g10, g01.g11, g10.g10, g10.g11, g11.g11.
// One warp per cell.
__global__ void __launch_bounds__(256) k_cell_gram(const float *__restrict__ grid, int wp, int hp, int nh,
                                                   float *__restrict__ gram) {
    const int cell = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (cell >= wp * hp) return;
    const int y0 = cell / wp, x0 = cell - y0 * wp;
    const int x1 = min(x0 + 1, wp - 1), y1 = min(y0 + 1, hp - 1);
    const float *g[4] = {grid + ((size_t)y0 * wp + x0) * nh, grid + ((size_t)y0 * wp + x1) * nh,
                         grid + ((size_t)y1 * wp + x0) * nh, grid + ((size_t)y1 * wp + x1) * nh};
    float d[10] = {};
    for (int o = lane; o < nh; o += 32) {
        const float v0 = g[0][o], v1 = g[1][o], v2 = g[2][o], v3 = g[3][o];
        d[0] = fmaf(v0, v0, d[0]);
        d[1] = fmaf(v0, v1, d[1]);
        d[2] = fmaf(v0, v2, d[2]);
        d[3] = fmaf(v0, v3, d[3]);
        d[4] = fmaf(v1, v1, d[4]);
        d[5] = fmaf(v1, v2, d[5]);
        d[6] = fmaf(v1, v3, d[6]);
        d[7] = fmaf(v2, v2, d[7]);
        d[8] = fmaf(v2, v3, d[8]);
        d[9] = fmaf(v3, v3, d[9]);
    }
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        float v = d[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) gram[(size_t)cell * 10 + i] = v;
    }
}

constexpr int kCellThreads = 256;

// One CTA per cell (ci, cj) of pixels that share their four patches.  Phase 1,
// a thread per pixel: the cosine from H, MH = M H, e and the cell's Gram; the
// loss; dL/dZ written over MH; b H written to bH; a w_k kept in shared memory.
// Phase 2, a thread per hidden unit (two halves of the pixels): D of the four
// corners.  Per-CTA sums of a w_k, b and the loss go out with one atomic each.
// Dynamic shared memory: 4 * npx_max floats (npx_max >= pixels of any cell).
__global__ void __launch_bounds__(kCellThreads) k_lift_cells(
    int W, int H, int wp, int hp, int patch, int npx_max, const float *__restrict__ Hm, float *__restrict__ MH,
    float *__restrict__ bH, const float *__restrict__ E, const float *__restrict__ s, const float *__restrict__ u,
    const float *__restrict__ beta, const float *__restrict__ gram, const float *__restrict__ weight, float g0,
    float *__restrict__ loss, float *__restrict__ D, float *__restrict__ alpha, float *__restrict__ sb) {
    extern __shared__ float aw[];  // [4][npx_max]
    __shared__ float sE[4][kLiftHidden], sU[kLiftHidden], sS[4], sG[10];
    __shared__ float red[kCellThreads / 32][6];
    __shared__ float part[4][kLiftHidden];
    const int ci = blockIdx.x, cj = blockIdx.y;
    const int x0 = ci, y0 = cj;
    const int x1 = min(x0 + 1, wp - 1), y1 = min(y0 + 1, hp - 1);
    const int corner[4] = {y0 * wp + x0, y0 * wp + x1, y1 * wp + x0, y1 * wp + x1};
    const int tid = threadIdx.x;
    for (int i = tid; i < 4 * kLiftHidden; i += kCellThreads)
        sE[i / kLiftHidden][i % kLiftHidden] = E[(size_t)corner[i / kLiftHidden] * kLiftHidden + i % kLiftHidden];
    if (tid < kLiftHidden) sU[tid] = u[tid];
    if (tid < 4) sS[tid] = s[corner[tid]];
    if (tid < 10) sG[tid] = gram[(size_t)(y0 * wp + x0) * 10 + tid];
    __syncthreads();
    const int xs = cell_start(ci, patch), xe = ci + 1 >= wp ? W : min(W, cell_start(ci + 1, patch));
    const int ys = cell_start(cj, patch), ye = cj + 1 >= hp ? H : min(H, cell_start(cj + 1, patch));
    const int nx = max(0, xe - xs), npx = nx * max(0, ye - ys);
    const size_t HW = (size_t)W * H;
    const float bt = *beta;
    const float inv2p = 1.f / (float)(2 * patch);
    float t_al[4] = {0.f, 0.f, 0.f, 0.f}, t_sb = 0.f, t_term = 0.f;
    for (int q = tid; q < npx; q += kCellThreads) {
        const int y = ys + q / nx, x = xs + q % nx;
        const size_t p = (size_t)y * W + x;
        // bilinear weights from exact integer numerators (clamped positions give 0;
        // at the far edge x1 == x0 and the two weights add up)
        const float ax = fminf(fmaxf((float)(2 * x + 1 - (2 * x0 + 1) * patch) * inv2p, 0.f), 1.f);
        const float ay = fminf(fmaxf((float)(2 * y + 1 - (2 * y0 + 1) * patch) * inv2p, 0.f), 1.f);
        const float w[4] = {(1.f - ax) * (1.f - ay), ax * (1.f - ay), (1.f - ax) * ay, ax * ay};
        float dot = 0.f, hmh = 0.f, uh = 0.f;
#pragma unroll 4
        for (int j = 0; j < kLiftHidden; ++j) {
            const float h = Hm[(size_t)j * HW + p], mh = MH[(size_t)j * HW + p];
            const float ej = w[0] * sE[0][j] + w[1] * sE[1][j] + w[2] * sE[2][j] + w[3] * sE[3][j];
            dot = fmaf(h, ej, dot);
            hmh = fmaf(h, mh, hmh);
            uh = fmaf(sU[j], h, uh);
        }
        dot += w[0] * sS[0] + w[1] * sS[1] + w[2] * sS[2] + w[3] * sS[3];
        const float nF2 = w[0] * w[0] * sG[0] + w[1] * w[1] * sG[4] + w[2] * w[2] * sG[7] + w[3] * w[3] * sG[9] +
                          2.f * (w[0] * w[1] * sG[1] + w[0] * w[2] * sG[2] + w[0] * w[3] * sG[3] +
                                 w[1] * w[2] * sG[5] + w[1] * w[3] * sG[6] + w[2] * w[3] * sG[8]);
        const float nFh2 = hmh + 2.f * uh + bt;
        const bool ok = nF2 > 0.f && nFh2 > 0.f;
        const float wpx = weight ? weight[p] : 1.f;  // per-pixel weight (the mask of Eq. 14)
        const float g = g0 * wpx;
        const float inv = ok ? rsqrtf(nF2) * rsqrtf(nFh2) : 0.f;
        const float cs = dot * inv;
        t_term += wpx * (1.f - cs);
        const float a = -g * inv, b = ok ? g * cs / nFh2 : 0.f;
#pragma unroll 4
        for (int j = 0; j < kLiftHidden; ++j) {
            const size_t o = (size_t)j * HW + p;
            const float h = Hm[o];
            const float ej = w[0] * sE[0][j] + w[1] * sE[1][j] + w[2] * sE[2][j] + w[3] * sE[3][j];
            const float dh = a * ej + b * (MH[o] + sU[j]);
            MH[o] = h > 0.f ? dh : 0.f;  // dL/dZ (ReLU derivative)
            bH[o] = b * h;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            aw[k * npx_max + q] = a * w[k];
            t_al[k] += a * w[k];
        }
        t_sb += b;
    }
    // per-CTA sums
    float v[6] = {t_al[0], t_al[1], t_al[2], t_al[3], t_sb, t_term};
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    if ((tid & 31) == 0)
#pragma unroll
        for (int i = 0; i < 6; ++i) red[tid >> 5][i] = v[i];
    __syncthreads();
    if (npx == 0) return;
    if (tid < 6) {
        float t = 0.f;
        for (int w8 = 0; w8 < kCellThreads / 32; ++w8) t += red[w8][tid];
        if (tid < 4)
            atomicAdd(alpha + corner[tid], t);
        else if (tid == 4)
            atomicAdd(sb, t);
        else
            atomicAdd(loss, g0 * t);
    }
    // D of the four corners: thread (half, j) sums its half of the pixels
    const int j = tid & (kLiftHidden - 1), half = tid >> 7;
    float P[4] = {0.f, 0.f, 0.f, 0.f};
    for (int q = half; q < npx; q += 2) {
        const int y = ys + q / nx, x = xs + q % nx;
        const float h = Hm[(size_t)j * HW + (size_t)y * W + x];
#pragma unroll
        for (int k = 0; k < 4; ++k) P[k] = fmaf(aw[k * npx_max + q], h, P[k]);
    }
    if (half == 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) part[k][j] = P[k];
    __syncthreads();
    if (half == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(D + (size_t)corner[k] * kLiftHidden + j, P[k] + part[k][j]);
}

// y[i] += x[i] * (*c)
__global__ void k_axpy_dev(int n, const float *__restrict__ x, const float *__restrict__ c, float *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fmaf(x[i], *c, y[i]);
}

size_t round64(size_t n) { return (n + 63) & ~size_t(63); }

// scratch of one view, in floats
struct LiftLayout {
    size_t Hm, MH, bH, E, s, M, u, beta, gram, D, alpha, hb, sb, Gb, total;
};
LiftLayout lift_layout(size_t hw, size_t np) {
    LiftLayout L{};
    size_t o = 0;
    auto take = [&](size_t n) {
        const size_t at = o;
        o += round64(n);
        return at;
    };
    L.Hm = take(kLiftHidden * hw);
    L.MH = take(kLiftHidden * hw);
    L.bH = take(kLiftHidden * hw);
    L.E = take(kLiftHidden * np);
    L.s = take(np);
    L.M = take(kLiftHidden * kLiftHidden);
    L.u = take(kLiftHidden);
    L.beta = take(1);
    L.gram = take(10 * np);
    // D, alpha, hb, sb: one run, cleared per view
    L.D = o;
    L.alpha = L.D + kLiftHidden * np;
    L.hb = L.alpha + np;
    L.sb = L.hb + kLiftHidden;
    o = L.sb + 64;
    L.Gb = take(kLiftHidden * kLiftHidden);
    L.total = o;
    return L;
}

}  // namespace

size_t lift_scratch_floats(size_t max_hw, size_t max_np) { return lift_layout(max_hw, max_np).total; }

// largest pixel count of a cell of the patch grid: a cell spans at most
// 1.5 patch + 1 pixels along an axis (the first one), or the whole view
int lift_cell_pixels(int patch) {
    const int m = (3 * patch) / 2 + 2;
    return m * m;
}

// One view: forward, loss and backward.  feat / d_feat: the view's planes
// [nf][HW]; grid: its patch grid [hp][wp][nh]; weight: its per-pixel weights
// (null: 1); scratch: lift_scratch_floats(HW, hp * wp) floats.
// d_w1 [128][nf], d_b1 [128], d_w2 [nh][128], d_b2 [nh] and d_feat are
// accumulated (may be null: that gradient is skipped).
cudaError_t lift_view(int num_sms, cudaStream_t st, int W, int H, int nf, int nh, int patch, const float *feat,
                      const float *grid, int wp, int hp, const float *w1, const float *b1, const float *w2,
                      const float *b2, float g, const float *weight, float *loss, float *d_w1, float *d_b1,
                      float *d_w2, float *d_b2, float *d_feat, float *scratch, int *launches) {
    const int HW = W * H, np = wp * hp;
    const int NH = kLiftHidden;
    const LiftLayout L = lift_layout((size_t)HW, (size_t)np);
    float *Hm = scratch + L.Hm;  // [128][HW] hidden (post-ReLU)
    float *MH = scratch + L.MH;  // [128][HW] M H, then dL/dZ
    float *bH = scratch + L.bH;  // [128][HW] b_p H_p
    float *E = scratch + L.E, *sv = scratch + L.s, *M = scratch + L.M, *u = scratch + L.u, *beta = scratch + L.beta;
    float *gram = scratch + L.gram, *D = scratch + L.D, *alpha = scratch + L.alpha, *hb = scratch + L.hb;
    float *sb = scratch + L.sb, *Gb = scratch + L.Gb;
    const dim3 blk(256);
    const unsigned gx = (unsigned)((HW + 255) / 256);
    cudaError_t e;
    // per patch and weight-sized: E = G W2 ([np][128]), s = G b2, M = W2^T W2, u = W2^T b2, beta = |b2|^2
    if ((e = gemm_f32(st, false, false, NH, np, nh, 1.f, w2, NH, grid, nh, 0.f, E, NH, num_sms, launches)) != cudaSuccess) return e;
    if ((e = gemm_f32(st, true, false, np, 1, nh, 1.f, grid, nh, b2, nh, 0.f, sv, np, num_sms, launches)) != cudaSuccess) return e;
    if ((e = gemm_f32(st, false, true, NH, NH, nh, 1.f, w2, NH, w2, NH, 0.f, M, NH, num_sms, launches)) != cudaSuccess) return e;
    if ((e = gemm_f32(st, false, false, NH, 1, nh, 1.f, w2, NH, b2, nh, 0.f, u, NH, num_sms, launches)) != cudaSuccess) return e;
    if ((e = gemm_f32(st, true, false, 1, 1, nh, 1.f, b2, nh, b2, nh, 0.f, beta, 1, num_sms, launches)) != cudaSuccess) return e;
    k_cell_gram<<<(unsigned)((np + 7) / 8), blk, 0, st>>>(grid, wp, hp, nh, gram);
    if ((e = cudaMemsetAsync(D, 0, (L.sb + 1 - L.D) * sizeof(float), st)) != cudaSuccess) return e;
    // H = relu(F~ W1^T + b1); MH = H M
    if ((e = gemm_f32(st, false, false, HW, NH, nf, 1.f, feat, HW, w1, nf, 0.f, Hm, HW, num_sms, launches)) != cudaSuccess) return e;
    k_bias_relu<<<dim3(gx, NH), blk, 0, st>>>(Hm, b1, (size_t)HW);
    if ((e = gemm_f32(st, false, false, HW, NH, NH, 1.f, Hm, HW, M, NH, 0.f, MH, HW, num_sms, launches)) != cudaSuccess) return e;
    const int npx_max = lift_cell_pixels(patch);
    k_lift_cells<<<dim3(wp, hp), kCellThreads, (size_t)4 * npx_max * sizeof(float), st>>>(
        W, H, wp, hp, patch, npx_max, Hm, MH, bH, E, sv, u, beta, gram, weight, g, loss, D, alpha, sb);
    *launches += 3;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    float *dZ = MH;
    const unsigned sum_blocks = (unsigned)((HW + kSumChunk - 1) / kSumChunk);
    if (d_w2 || d_b2) {
        k_row_sums<<<dim3(sum_blocks, NH), blk, 0, st>>>(bH, (size_t)HW, hb);
        ++*launches;
    }
    if (d_w2) {
        // dW2 ([nh][128] row-major = column-major 128 x nh) += D^T-side: D G, Gb W2, hb b2^T
        if ((e = gemm_f32(st, true, false, NH, NH, HW, 1.f, bH, HW, Hm, HW, 0.f, Gb, NH, num_sms, launches)) != cudaSuccess) return e;
        if ((e = gemm_f32(st, false, true, NH, nh, np, 1.f, D, NH, grid, nh, 1.f, d_w2, NH, num_sms, launches)) != cudaSuccess)
            return e;
        if ((e = gemm_f32(st, false, false, NH, nh, NH, 1.f, Gb, NH, w2, NH, 1.f, d_w2, NH, num_sms, launches)) != cudaSuccess)
            return e;
        if ((e = gemm_f32(st, false, true, NH, nh, 1, 1.f, hb, NH, b2, nh, 1.f, d_w2, NH, num_sms, launches)) != cudaSuccess)
            return e;
    }
    if (d_b2) {
        // db2 += G^T alpha + W2 hb + b2 sum_p b_p
        if ((e = gemm_f32(st, false, false, nh, 1, np, 1.f, grid, nh, alpha, np, 1.f, d_b2, nh, num_sms, launches)) != cudaSuccess)
            return e;
        if ((e = gemm_f32(st, true, false, nh, 1, NH, 1.f, w2, NH, hb, NH, 1.f, d_b2, nh, num_sms, launches)) != cudaSuccess)
            return e;
        k_axpy_dev<<<(unsigned)((nh + 255) / 256), blk, 0, st>>>(nh, b2, sb, d_b2);
        ++*launches;
    }
    if (d_b1) {
        k_row_sums<<<dim3(sum_blocks, NH), blk, 0, st>>>(dZ, (size_t)HW, d_b1);
        ++*launches;
    }
    // dW1 += F~^T dZ ([nf x 128] column-major = [128][nf] row-major)
    if (d_w1 && (e = gemm_f32(st, true, false, nf, NH, HW, 1.f, feat, HW, dZ, HW, 1.f, d_w1, nf, num_sms, launches)) != cudaSuccess)
        return e;
    // dF~ += dZ W1
    if (d_feat && (e = gemm_f32(st, false, true, HW, nf, NH, 1.f, dZ, HW, w1, nf, 1.f, d_feat, HW, num_sms, launches)) != cudaSuccess)
        return e;
    return cudaGetLastError();
}

}  // namespace ups
