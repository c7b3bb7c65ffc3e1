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
// Every pixel-sized product (F~ W1^T, M H, the Gram of b H over pixels and
// the two backward products with W1) runs inside one fused kernel over the
// cells of pixels that share their four patches: the 128-wide per-pixel
// quantities stay on chip, and the kernel also does the cosine, the loss,
// dL/dZ and the per-patch sums.  At N_l = 16 that is k_lift_tc (the products
// but dF~ on the tensor cores, below), at N_l = 32 the all-FP32 k_lift_fused.
// The per-patch and weight-sized products are FP32 GEMMs (gemm.cu).
#include <cstddef>

#include "common.cuh"
#include "umma.cuh"

namespace ups {

namespace {

constexpr int kLiftHidden = 128;

// first pixel index along an axis whose clamped bilinear position
// floor(clamp((x + 0.5) / patch - 0.5, 0, n - 1)) is at least i
__device__ __forceinline__ int cell_start(int i, int patch) {
    // (x + 0.5) / patch - 0.5 >= i  <=>  x >= i * patch + (patch - 1) / 2
    return i == 0 ? 0 : (int)ceilf((float)i * patch + 0.5f * (float)(patch - 1) - 1e-4f);
}

// The cells of all views' patch grids, numbered view after view (cell c of
// view v = patch c of its grid; the grids are concatenated in view order):
// view of global cell `cell`, its grid size and the view's first cell.
struct CellView {
    int v, wp, hp, base;
};
__device__ __forceinline__ CellView cell_view(const ViewTable &vt, int patch, int cell) {
    CellView r{0, 0, 0, 0};
    int base = 0;
    for (int v = 0; v < vt.n; ++v) {
        const int wp = (vt.v[v].W + patch - 1) / patch, hp = (vt.v[v].H + patch - 1) / patch;
        if (cell < base + wp * hp || v == vt.n - 1) {
            r = CellView{v, wp, hp, base};
            break;
        }
        base += wp * hp;
    }
    return r;
}

// Gram matrix of the four corner patches of every cell (x0, y0) of the grid
// (x1 = min(x0 + 1, wp - 1), y1 likewise): gram[cell][10] = g00.g00, g00.g01,
// g00.g10, g00.g11, g01.g01, g01.g10, g01.g11, g10.g10, g10.g11, g11.g11.
// One warp per cell.
__global__ void __launch_bounds__(256) k_cell_gram(ViewTable vt, int patch, int n_cells, const float *__restrict__ grid,
                                                   int nh, float *__restrict__ gram) {
    const int cell = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (cell >= n_cells) return;
    const CellView cv = cell_view(vt, patch, cell);
    const int wp = cv.wp, hp = cv.hp;
    const int local = cell - cv.base;
    const int y0 = local / wp, x0 = local - y0 * wp;
    const int x1 = min(x0 + 1, wp - 1), y1 = min(y0 + 1, hp - 1);
    const float *vg = grid + (size_t)cv.base * nh;
    const float *g[4] = {vg + ((size_t)y0 * wp + x0) * nh, vg + ((size_t)y0 * wp + x1) * nh,
                         vg + ((size_t)y1 * wp + x0) * nh, vg + ((size_t)y1 * wp + x1) * nh};
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

// ---------------------------------------------------------------------------
// fused per-cell kernel: everything 128 wide stays in shared memory
// ---------------------------------------------------------------------------
//
// Persistent CTAs (256 threads) walk the cells of the patch grid; a cell's
// pixels share their four corner patches and go through in chunks of kFC:
//   Z = W1 F~ + b1, H = relu(Z)           (hidden-major Hh and pixel-major Hp)
//   MH = M H                               (8 hidden x 4 pixels per thread)
//   per pixel: H.e_p, u.H, H.MH -> cos, the loss, a_p, b_p
//   dZ = (a e_p + b (MH + u)) relu'(Z)     (over Hh), b H (pixel-major bHp)
//   Gram += (bH)^T H                        (registers, upper 8x8 blocks only)
//   dF~ = W1^T dZ, dW1 += dZ F~^T, db1 += sum dZ, hb += sum b H,
//   D of the four corners += sum a w_k H
// Gram, hb, db1 and dW1 go out with one atomic per value and CTA at the end,
// D and alpha per cell.  FP32 fmaf throughout.
constexpr int kFC = 64;                 // pixels per chunk
constexpr int kFT = 256;                // threads
constexpr int kHP = kFC + 4;            // row stride of hidden-major arrays
constexpr int kPP = kLiftHidden + 4;    // row stride of pixel-major arrays

template <int NF>
struct FusedSmem {
    float M[kLiftHidden][kLiftHidden];   // symmetric W2^T W2
    float W1T[NF][kLiftHidden];          // W1 transposed
    float b1[kLiftHidden], u[kLiftHidden];
    float E[4][kLiftHidden];             // W2^T g of the cell's four corners
    float Fc[NF][kHP];                   // F~ of the chunk, channel-major
    float Hh[kLiftHidden][kHP];          // H, then dZ (hidden-major)
    float Hp[kFC][kPP];                  // H (pixel-major)
    float bHp[kFC][kPP];                 // b_p H_p (pixel-major)
    float red[16][kFC][3];               // partial H.e, u.H, H.MH per hidden block
    float w4[kFC][4];                    // bilinear weights of the chunk's pixels
    float ab[kFC][2];                    // a_p, b_p
    float aw[4][kFC];                    // a_p w_k(p)
    float Dpart[4][kLiftHidden];
    float sS[4], sG[10];
    int pix[kFC];                        // pixel index in the view, -1: none
};

size_t fused_smem_bytes(int nf) {
    return nf == 32 ? sizeof(FusedSmem<32>) : sizeof(FusedSmem<16>);
}

template <int NF>
__global__ void __launch_bounds__(kFT, 1) k_lift_fused(
    ViewTable vt, int n_cells, int patch, const float *__restrict__ feat_all, const float *__restrict__ w1,
    const float *__restrict__ b1, const float *__restrict__ Mg, const float *__restrict__ E,
    const float *__restrict__ s, const float *__restrict__ u, const float *__restrict__ beta,
    const float *__restrict__ gram, const float *__restrict__ weight_all, float g0, float *__restrict__ loss,
    float *__restrict__ D, float *__restrict__ alpha, float *__restrict__ sb, float *__restrict__ hb_out,
    float *__restrict__ Gb, float *__restrict__ d_w1, float *__restrict__ d_b1, float *__restrict__ d_feat_all) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<NF> &S = *reinterpret_cast<FusedSmem<NF> *>(smem_raw);
    const int tid = threadIdx.x;
    for (int i = tid; i < kLiftHidden * kLiftHidden; i += kFT) (&S.M[0][0])[i] = Mg[i];
    for (int i = tid; i < kLiftHidden * NF; i += kFT) {
        const int j = i / NF, c = i - j * NF;
        S.W1T[c][j] = w1[i];
    }
    if (tid < kLiftHidden) {
        S.b1[tid] = b1[tid];
        S.u[tid] = u[tid];
    }
    const float bt = *beta;
    const float inv2p = 1.f / (float)(2 * patch);
    // thread blocks: A = 8 hidden x 4 pixels; G = 8 x 8 of the Gram
    const int jb = tid >> 4, pb = tid & 15;
    const int j0 = jb * 8, p0 = pb * 4;
    // the Gram is symmetric: threads 0..135 own the 136 upper 8x8 blocks
    // (row-major over the block triangle), so whole warps share the work
    int gbi = 0, gt = tid;
    while (gbi < 16 && gt >= 16 - gbi) {
        gt -= 16 - gbi;
        ++gbi;
    }
    const bool gram_on = tid < 136;
    const int gi0 = (gram_on ? gbi : 0) * 8, gj0 = (gram_on ? gbi + gt : 0) * 8;
    f2 G2[4][8];  // Gram rows (x, x + 1) packed for fma.rn.f32x2
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) G2[x][y] = 0ull;
    float hb[8], db1[8];
#pragma unroll
    for (int x = 0; x < 8; ++x) hb[x] = db1[x] = 0.f;
    // dW1: thread (8 hidden of block jb) x (channels c = pb, pb + 16 for NF = 32)
    constexpr int NC = NF / 16;
    float dw1[8][NC];
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < NC; ++y) dw1[x][y] = 0.f;
    float t_loss = 0.f, t_sb = 0.f;
    for (int cell = blockIdx.x; cell < n_cells; cell += gridDim.x) {
        // the cell's view, its images and its four corner patches (global patch indices)
        const CellView cv = cell_view(vt, patch, cell);
        const int wp = cv.wp, hp = cv.hp, W = vt.v[cv.v].W, H = vt.v[cv.v].H;
        const size_t HW = (size_t)W * H, P = (size_t)vt.v[cv.v].pix_off;
        const float *feat = feat_all + (size_t)NF * P;
        float *d_feat = d_feat_all ? d_feat_all + (size_t)NF * P : nullptr;
        const float *weight = weight_all ? weight_all + P : nullptr;
        const int local = cell - cv.base;
        const int cj = local / wp, ci = local - cj * wp;
        const int x0 = ci, y0 = cj;
        const int x1 = min(x0 + 1, wp - 1), y1 = min(y0 + 1, hp - 1);
        const int corner[4] = {cv.base + y0 * wp + x0, cv.base + y0 * wp + x1, cv.base + y1 * wp + x0,
                               cv.base + y1 * wp + x1};
        const int xs = cell_start(ci, patch), xe = ci + 1 >= wp ? W : min(W, cell_start(ci + 1, patch));
        const int ys = cell_start(cj, patch), ye = cj + 1 >= hp ? H : min(H, cell_start(cj + 1, patch));
        const int nx = max(0, xe - xs), npx = nx * max(0, ye - ys);
        __syncthreads();  // the previous cell's shared data is no longer read
        for (int i = tid; i < 4 * kLiftHidden; i += kFT)
            S.E[i / kLiftHidden][i % kLiftHidden] = E[(size_t)corner[i / kLiftHidden] * kLiftHidden + i % kLiftHidden];
        if (tid < 4) S.sS[tid] = s[corner[tid]];
        if (tid < 10) S.sG[tid] = gram[(size_t)cell * 10 + tid];
        for (int i = tid; i < 4 * kLiftHidden; i += kFT) (&S.Dpart[0][0])[i] = 0.f;
        float al[4] = {0.f, 0.f, 0.f, 0.f};  // sum a w_k over the cell (threads < kFC)
        for (int q0 = 0; q0 < npx; q0 += kFC) {
            __syncthreads();
            // chunk pixels, bilinear weights, F~
            if (tid < kFC) {
                const int q = q0 + tid;
                int pidx = -1;
                float w[4] = {0.f, 0.f, 0.f, 0.f};
                if (q < npx) {
                    const int y = ys + q / nx, x = xs + q % nx;
                    pidx = y * W + x;
                    const float ax = fminf(fmaxf((float)(2 * x + 1 - (2 * x0 + 1) * patch) * inv2p, 0.f), 1.f);
                    const float ay = fminf(fmaxf((float)(2 * y + 1 - (2 * y0 + 1) * patch) * inv2p, 0.f), 1.f);
                    w[0] = (1.f - ax) * (1.f - ay);
                    w[1] = ax * (1.f - ay);
                    w[2] = (1.f - ax) * ay;
                    w[3] = ax * ay;
                }
                S.pix[tid] = pidx;
#pragma unroll
                for (int k = 0; k < 4; ++k) S.w4[tid][k] = w[k];
            }
            __syncthreads();
            for (int i = tid; i < NF * kFC; i += kFT) {
                const int c = i / kFC, p = i - c * kFC;
                const int pidx = S.pix[p];
                S.Fc[c][p] = pidx >= 0 ? feat[(size_t)c * HW + pidx] : 0.f;
            }
            __syncthreads();
            // Z and H (block A)
            {
                // hidden pairs (x, x + 1) packed for fma.rn.f32x2 (each half rounded as a scalar fmaf)
                f2 z2[4][4];
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) z2[x][y] = f2_make(S.b1[j0 + 2 * x], S.b1[j0 + 2 * x + 1]);
#pragma unroll 4
                for (int c = 0; c < NF; ++c) {
                    const ulonglong2 wa = *reinterpret_cast<const ulonglong2 *>(&S.W1T[c][j0]);
                    const ulonglong2 wb = *reinterpret_cast<const ulonglong2 *>(&S.W1T[c][j0 + 4]);
                    const float4 f = *reinterpret_cast<const float4 *>(&S.Fc[c][p0]);
                    const f2 wv[4] = {wa.x, wa.y, wb.x, wb.y};
                    const f2 fv[4] = {f2_make(f.x, f.x), f2_make(f.y, f.y), f2_make(f.z, f.z), f2_make(f.w, f.w)};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) z2[x][y] = f2_fma(wv[x], fv[y], z2[x][y]);
                }
                float z[8][4];
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) f2_split(z2[x][y], z[2 * x][y], z[2 * x + 1][y]);
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const float4 h4 = make_float4(fmaxf(z[x][0], 0.f), fmaxf(z[x][1], 0.f), fmaxf(z[x][2], 0.f),
                                                  fmaxf(z[x][3], 0.f));
                    *reinterpret_cast<float4 *>(&S.Hh[j0 + x][p0]) = h4;
                    S.Hp[p0][j0 + x] = h4.x;
                    S.Hp[p0 + 1][j0 + x] = h4.y;
                    S.Hp[p0 + 2][j0 + x] = h4.z;
                    S.Hp[p0 + 3][j0 + x] = h4.w;
                }
            }
            __syncthreads();
            // MH (block A), then the per-pixel partial dot products
            float mh[8][4];
            {
                f2 m2[4][4];  // hidden pairs (x, x + 1) for fma.rn.f32x2
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) m2[x][y] = 0ull;
#pragma unroll 4
                for (int k = 0; k < kLiftHidden; ++k) {
                    const ulonglong2 ma = *reinterpret_cast<const ulonglong2 *>(&S.M[k][j0]);
                    const ulonglong2 mb = *reinterpret_cast<const ulonglong2 *>(&S.M[k][j0 + 4]);
                    const float4 h = *reinterpret_cast<const float4 *>(&S.Hh[k][p0]);
                    const f2 mv[4] = {ma.x, ma.y, mb.x, mb.y};
                    const f2 hv2[4] = {f2_make(h.x, h.x), f2_make(h.y, h.y), f2_make(h.z, h.z), f2_make(h.w, h.w)};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) m2[x][y] = f2_fma(mv[x], hv2[y], m2[x][y]);
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) f2_split(m2[x][y], mh[2 * x][y], mh[2 * x + 1][y]);
            }
            float hv[8][4], ev[8][4];
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const float4 h = *reinterpret_cast<const float4 *>(&S.Hh[j0 + x][p0]);
                hv[x][0] = h.x;
                hv[x][1] = h.y;
                hv[x][2] = h.z;
                hv[x][3] = h.w;
            }
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const float4 w = *reinterpret_cast<const float4 *>(&S.w4[p0 + y][0]);
                float de = 0.f, du = 0.f, dm = 0.f;
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const int j = j0 + x;
                    ev[x][y] = w.x * S.E[0][j] + w.y * S.E[1][j] + w.z * S.E[2][j] + w.w * S.E[3][j];
                    de = fmaf(hv[x][y], ev[x][y], de);
                    du = fmaf(S.u[j], hv[x][y], du);
                    dm = fmaf(hv[x][y], mh[x][y], dm);
                }
                S.red[jb][p0 + y][0] = de;
                S.red[jb][p0 + y][1] = du;
                S.red[jb][p0 + y][2] = dm;
            }
            __syncthreads();
            // per pixel: cosine, loss, a_p, b_p
            if (tid < kFC) {
                const int p = tid;
                float de = 0.f, du = 0.f, dm = 0.f;
                for (int b = 0; b < 16; ++b) {
                    de += S.red[b][p][0];
                    du += S.red[b][p][1];
                    dm += S.red[b][p][2];
                }
                const float *w = S.w4[p];
                const float dot = de + w[0] * S.sS[0] + w[1] * S.sS[1] + w[2] * S.sS[2] + w[3] * S.sS[3];
                const float nF2 = w[0] * w[0] * S.sG[0] + w[1] * w[1] * S.sG[4] + w[2] * w[2] * S.sG[7] +
                                  w[3] * w[3] * S.sG[9] +
                                  2.f * (w[0] * w[1] * S.sG[1] + w[0] * w[2] * S.sG[2] + w[0] * w[3] * S.sG[3] +
                                         w[1] * w[2] * S.sG[5] + w[1] * w[3] * S.sG[6] + w[2] * w[3] * S.sG[8]);
                const float nFh2 = dm + 2.f * du + bt;
                float a = 0.f, b = 0.f;
                const int pidx = S.pix[p];
                if (pidx >= 0) {
                    const bool ok = nF2 > 0.f && nFh2 > 0.f;
                    const float wpx = weight ? weight[pidx] : 1.f;
                    const float g = g0 * wpx;
                    const float inv = ok ? rsqrtf(nF2) * rsqrtf(nFh2) : 0.f;
                    const float cs = dot * inv;
                    t_loss += wpx * (1.f - cs);
                    a = -g * inv;
                    b = ok ? g * cs / nFh2 : 0.f;
                    t_sb += b;
                }
                S.ab[p][0] = a;
                S.ab[p][1] = b;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    S.aw[k][p] = a * w[k];
                    al[k] += a * w[k];
                }
            }
            __syncthreads();
            // dZ over Hh, b H to bHp, db1 and hb sums (block A)
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const float a = S.ab[p0 + y][0], b = S.ab[p0 + y][1];
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const int j = j0 + x;
                    const float dh = fmaf(a, ev[x][y], b * (mh[x][y] + S.u[j]));
                    const float dz = hv[x][y] > 0.f ? dh : 0.f;
                    S.Hh[j][p0 + y] = dz;
                    S.bHp[p0 + y][j] = b * hv[x][y];
                    db1[x] += dz;
                    hb[x] = fmaf(b, hv[x][y], hb[x]);
                }
            }
            __syncthreads();
            // Gram (upper 8x8 blocks), D of the corners, dF~, dW1
            if (gram_on) {
#pragma unroll 2
                for (int p = 0; p < kFC; ++p) {
                    const ulonglong2 ba = *reinterpret_cast<const ulonglong2 *>(&S.bHp[p][gi0]);
                    const ulonglong2 bb = *reinterpret_cast<const ulonglong2 *>(&S.bHp[p][gi0 + 4]);
                    const float4 ha = *reinterpret_cast<const float4 *>(&S.Hp[p][gj0]);
                    const float4 hc = *reinterpret_cast<const float4 *>(&S.Hp[p][gj0 + 4]);
                    const f2 bv[4] = {ba.x, ba.y, bb.x, bb.y};
                    const float hvv[8] = {ha.x, ha.y, ha.z, ha.w, hc.x, hc.y, hc.z, hc.w};
#pragma unroll
                    for (int y = 0; y < 8; ++y) {
                        const f2 h2 = f2_make(hvv[y], hvv[y]);
#pragma unroll
                        for (int x = 0; x < 4; ++x) G2[x][y] = f2_fma(bv[x], h2, G2[x][y]);
                    }
                }
            }
            {
                // D: thread (hidden j, half of the pixels)
                const int j = tid & (kLiftHidden - 1), half = tid >> 7;
                float Dk[4] = {0.f, 0.f, 0.f, 0.f};
                for (int p = half; p < kFC; p += 2) {
                    const float h = S.Hp[p][j];
#pragma unroll
                    for (int k = 0; k < 4; ++k) Dk[k] = fmaf(S.aw[k][p], h, Dk[k]);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) atomicAdd(&S.Dpart[k][j], Dk[k]);
            }
            {
                // dF~ = W1^T dZ: thread (channel, 4 pixels); NF x kFC outputs
                for (int o = tid; o < NF * (kFC / 4); o += kFT) {
                    const int c = o / (kFC / 4), pq = (o - c * (kFC / 4)) * 4;
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
                    for (int j = 0; j < kLiftHidden; ++j) {
                        const float wv = S.W1T[c][j];
                        const float4 dz = *reinterpret_cast<const float4 *>(&S.Hh[j][pq]);
                        acc[0] = fmaf(wv, dz.x, acc[0]);
                        acc[1] = fmaf(wv, dz.y, acc[1]);
                        acc[2] = fmaf(wv, dz.z, acc[2]);
                        acc[3] = fmaf(wv, dz.w, acc[3]);
                    }
                    if (d_feat)
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            const int pidx = S.pix[pq + y];
                            if (pidx >= 0) d_feat[(size_t)c * HW + pidx] += acc[y];
                        }
                }
            }
            // dW1 += dZ F~^T: thread (8 hidden of block jb) x channels pb (+16)
#pragma unroll 2
            for (int pq = 0; pq < kFC; pq += 4) {
                float4 fz[NC];
#pragma unroll
                for (int y = 0; y < NC; ++y) fz[y] = *reinterpret_cast<const float4 *>(&S.Fc[pb + 16 * y][pq]);
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const float4 dz = *reinterpret_cast<const float4 *>(&S.Hh[j0 + x][pq]);
#pragma unroll
                    for (int y = 0; y < NC; ++y)
                        dw1[x][y] = fmaf(dz.x, fz[y].x, fmaf(dz.y, fz[y].y, fmaf(dz.z, fz[y].z, fmaf(dz.w, fz[y].w, dw1[x][y]))));
                }
            }
        }
        __syncthreads();
        // the cell's D rows and alpha
        for (int i = tid; i < 4 * kLiftHidden; i += kFT) {
            const int k = i / kLiftHidden, j = i - k * kLiftHidden;
            if (npx > 0) atomicAdd(D + (size_t)corner[k] * kLiftHidden + j, S.Dpart[k][j]);
        }
        if (tid < kFC && npx > 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(alpha + corner[k], al[k]);
    }
    // the CTA's sums
    if (gram_on)
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 8; ++y) {
                float g0v, g1v;
                f2_split(G2[x][y], g0v, g1v);
                const float gv[2] = {g0v, g1v};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = gi0 + 2 * x + h, j = gj0 + y;
                    if (i <= j) {
                        atomicAdd(Gb + (size_t)i * kLiftHidden + j, gv[h]);
                        if (i != j) atomicAdd(Gb + (size_t)j * kLiftHidden + i, gv[h]);
                    }
                }
            }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        float h = hb[x], d = db1[x];
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {  // the 16 threads of block jb are lanes 16 (jb & 1) ..
            h += __shfl_xor_sync(0xffffffffu, h, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if (pb == 0) {
            atomicAdd(hb_out + j0 + x, h);
            if (d_b1) atomicAdd(d_b1 + j0 + x, d);
        }
        if (d_w1)
#pragma unroll
            for (int y = 0; y < NC; ++y) atomicAdd(d_w1 + (size_t)(j0 + x) * NF + pb + 16 * y, dw1[x][y]);
    }
    float v2[2] = {t_loss, t_sb};
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v2[i] += __shfl_xor_sync(0xffffffffu, v2[i], o);
    if ((tid & 31) == 0) {
        atomicAdd(loss, g0 * v2[0]);
        atomicAdd(sb, v2[1]);
    }
}

// ---------------------------------------------------------------------------
// fused per-cell kernel with the per-pixel products on the tensor cores
// ---------------------------------------------------------------------------
//
// The walk of k_lift_fused (N_l = 16) in chunks of 64 pixels, with every
// per-pixel product but dF~ as tcgen05 MMAs accumulating in FP32 in TMEM:
// Z = W1 F~ in 3xTF32 (x = hi + lo, hi = tf32(x), lo = tf32(x - hi); its sign
// decides ReLU', which a BF16 split flips too often), M H, the Gram of b H and
// dW1 = dZ F~^T in 3xBF16 (hi = bf16(x), lo = bf16(x - hi); about 1e-5
// relative per product), each as hi*hi + hi*lo + lo*hi.  dF~ = W1^T dZ and the
// per-pixel terms run in FP32 on the CUDA cores.
//   TMEM columns [0, 64): Z, then M H of the chunk (lane = hidden unit, column = pixel)
//   TMEM columns [64, 80): dW1, accumulated over all of the CTA's chunks
//   TMEM columns [128, 256): the Gram, likewise
//   TMEM columns [256, 384): M hi, lo; [384, 448): H hi, lo; [448, 512): dZ hi, lo (A operands)
// Thread 0 issues the Z and M H MMAs (`mh_bar` completes each), thread kGramTid
// the Gram and dW1 MMAs (`g_bar` completes them, waited at the next chunk).  A
// warp reads TMEM lanes 32 (w % 4) .. + 31, so thread (warp w, lane i) owns
// hidden unit j = 32 (w % 4) + i and the chunk's pixels 32 (w / 4) .. + 31 from
// Z on, keeping H of them in registers; per-pixel sums over hidden units are
// reduce-scattered over the warp's lanes and added over the four warps of a
// pixel half.  H reaches M H's B operand in the MN-major layout straight from
// the registers; a chunk's global inputs arrive by cp.async a chunk ahead.
namespace lt {
constexpr int kP = 64;       // pixels per chunk
constexpr int kT = 256;      // threads
constexpr int kHS = kP + 4;  // row stride of the FP32 hidden-major arrays
// TMEM columns; the A operands (M, and H as the Gram's A) sit in TMEM as BF16
// pairs (row = lane), so the MMAs read only their B operands from shared memory
constexpr uint32_t kTmemCols = 512, cMH = 0, cG = 128, cMhi = 256, cMlo = 320, cHAhi = 384, cHAlo = 416;
// dW1 accumulator (16 columns) and dZ as its A operand (BF16 hi / lo pairs)
constexpr uint32_t cDW = 64, cDZhi = 448, cDZlo = 480;
// BF16 B operand tiles in shared memory (byte offsets): H of M H (MN-major), b H of
// the Gram (K-major, no swizzle)
constexpr int oHBhi = 0, oHBlo = 16384;        // H [128 k][64 p] (B of M H)
constexpr int oBHhi = 32768, oBHlo = 49152;    // b H [128 i][64 p] (B of the Gram)
constexpr int kOpBytes = 65536;
constexpr int kWait = 1 << 22;
constexpr int kGramTid = 128;  // issues the Gram and dW1 MMAs
// M H's B operand H (K = 128 hidden units x N = 64 pixels) in the MN-major layout
// without swizzle: core matrices of 8 hidden rows x 8 pixels (16 bytes per row, 128
// bytes each), 8 along N then 16 along K, so that a thread writes its hidden unit's
// pixels from registers; the descriptor takes LBO = 1024 (the stride between core
// matrices along K) and SBO = 128 (along N), a K step of 16 hidden units advances the
// start by 2048 bytes, and the instruction descriptor's B-major bit selects MN-major.
__device__ __forceinline__ uint32_t hb_mn_offset(int j, int p) {
    return (uint32_t)((j >> 3) * 1024 + (p >> 3) * 128 + (j & 7) * 16 + (p & 7) * 2);
}
__device__ __forceinline__ uint64_t desc_strides(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;
}
}  // namespace lt

struct LiftTcSmem {  // after the operand tiles (1 KB aligned); the arrays read as
                     // 16-byte vectors come first, at 16-byte multiples
    float Hh[kLiftHidden][lt::kHS];  // dZ (hidden-major), for dF~
    float W1A[2][kLiftHidden * 16];  // W1 as TF32 hi / lo, K-major [128 hidden][16 channels] (A of Z)
    float FcN[2][lt::kP * 16];       // F~ as TF32 hi / lo, K-major [64 pixels][16 channels] (B of Z)
    float W1r[kLiftHidden][16];      // W1 (hidden-major rows)
    float b1[kLiftHidden], u[kLiftHidden];
    // a chunk's global inputs, two buffers (chunk parity), filled a chunk ahead
    float E[2][4][kLiftHidden];      // W2^T g of the cell's four corners
    float Fc[2][16][lt::kHS];        // F~ of the chunk, channel-major
    float dF0[2][16][lt::kP];        // dL/dF~ accumulated before this call, channel-major
    float w4[lt::kP][4];             // bilinear weights of the chunk's pixels
    float ab[lt::kP][2];             // a_p, b_p
    float aw[lt::kP][4];             // a_p w_k(p)
    float Dpart[4][kLiftHidden];
    float red[4][lt::kP][2];         // partial H.e, H.(M H + 2 u) per 32 hidden units
    uint32_t FcT[2][512];            // F~ as BF16 hi / lo, K-major [16 channels][64 pixels] (B of dW1)
    float wpx[2][lt::kP];            // loss weights of the chunk's pixels
    float sS[2][4], sG[2][12];       // s of the corners, the cell's corner Gram (10 used)
    int pix[lt::kP];                 // pixel index in the view, -1: none
    int vwp[UPS_MAX_VIEWS], vhp[UPS_MAX_VIEWS], vbase[UPS_MAX_VIEWS];  // each view's patch grid, first cell
    uint64_t mh_bar, g_bar;
    uint32_t tmem_base;
    int abort_flag;
};
static_assert(offsetof(LiftTcSmem, Hh) == 0 && offsetof(LiftTcSmem, W1A) % 16 == 0 &&
                  offsetof(LiftTcSmem, FcN) % 16 == 0 &&
                  offsetof(LiftTcSmem, W1r) % 16 == 0 && offsetof(LiftTcSmem, FcT) % 16 == 0 &&
                  offsetof(LiftTcSmem, E) % 16 == 0 && offsetof(LiftTcSmem, Fc) % 16 == 0 &&
                  offsetof(LiftTcSmem, dF0) % 16 == 0 &&
                  offsetof(LiftTcSmem, w4) % 16 == 0 && offsetof(LiftTcSmem, ab) % 8 == 0 &&
                  offsetof(LiftTcSmem, mh_bar) % 8 == 0,
              "vector, bulk-copy and mbarrier alignment of the lifting kernel's shared arrays");

// Pixel rectangle of cell `cell` of the patch grids (the pixels whose four
// nearest patch centres are its corners) and its view, from the per-view grid
// table in shared memory (the same numbering as cell_view).
struct CellGeo {
    int v, W, wp, hp, base, x0, y0, xs, ys, nx, npx;
    size_t HW, P;
};
__device__ __forceinline__ CellGeo cell_geo(const LiftTcSmem &S, const ViewTable &vt, int patch, int cell) {
    int v = 0;
    while (v + 1 < vt.n && cell >= S.vbase[v + 1]) ++v;
    const CellView cv{v, S.vwp[v], S.vhp[v], S.vbase[v]};
    CellGeo g;
    g.v = cv.v;
    g.wp = cv.wp;
    g.hp = cv.hp;
    g.base = cv.base;
    g.W = vt.v[cv.v].W;
    const int H = vt.v[cv.v].H;
    g.HW = (size_t)g.W * H;
    g.P = (size_t)vt.v[cv.v].pix_off;
    const int local = cell - cv.base;
    g.y0 = local / cv.wp;
    g.x0 = local - g.y0 * cv.wp;
    g.xs = cell_start(g.x0, patch);
    const int xe = g.x0 + 1 >= cv.wp ? g.W : min(g.W, cell_start(g.x0 + 1, patch));
    g.ys = cell_start(g.y0, patch);
    const int ye = g.y0 + 1 >= cv.hp ? H : min(H, cell_start(g.y0 + 1, patch));
    g.nx = max(0, xe - g.xs);
    g.npx = g.nx * max(0, ye - g.ys);
    return g;
}
// corner k of the cell (bit 0: next column, bit 1: next row, clamped to the grid)
__device__ __forceinline__ int cell_corner(const CellGeo &g, int k) {
    const int x = (k & 1) ? min(g.x0 + 1, g.wp - 1) : g.x0, y = (k & 2) ? min(g.y0 + 1, g.hp - 1) : g.y0;
    return g.base + y * g.wp + x;
}

// Asynchronous global-to-shared copies (cp.async): 4 bytes, zero-filled and
// nothing read where !valid; 16 bytes; groups committed and waited per thread.
__device__ __forceinline__ void cp_async4(void *dst, const float *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(umma::smem_addr(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const float *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(umma::smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issues the copies of chunk (cell, q0)'s global inputs into buffer B (all
// kT threads call it): F~ and dL/dF~ accumulated before the call (thread t:
// pixel t % kP, channels t / kP + 4 r), the loss weights (t < kP), and the
// cell's corner rows of E, s and its Gram.  Pixels past the cell's end read
// nothing and hold 0.
__device__ __forceinline__ void lift_chunk_issue(LiftTcSmem &S, int B, const ViewTable &vt, int patch, int cell,
                                                 int q0, const float *__restrict__ feat_all,
                                                 const float *__restrict__ d_feat_all,
                                                 const float *__restrict__ weight_all, const float *__restrict__ E,
                                                 const float *__restrict__ s, const float *__restrict__ gram, int tid) {
    using namespace lt;
    const CellGeo g = cell_geo(S, vt, patch, cell);
    {
        const int p = tid & (kP - 1), q = q0 + p;
        const bool in = q < g.npx;
        const int yq = in ? q / g.nx : 0;
        const size_t pidx = in ? (size_t)(g.ys + yq) * g.W + g.xs + (q - yq * g.nx) : 0;
        const float *feat = feat_all + (size_t)16 * g.P;
        const float *df = d_feat_all ? d_feat_all + (size_t)16 * g.P : nullptr;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int c = (tid / kP) + 4 * r;
            cp_async4(&S.Fc[B][c][p], feat + (size_t)c * g.HW + pidx, in);
            if (df) cp_async4(&S.dF0[B][c][p], df + (size_t)c * g.HW + pidx, in);
        }
        if (weight_all && tid < kP) cp_async4(&S.wpx[B][p], weight_all + g.P + pidx, in);
    }
    if (tid < 128) {
        const int k = tid >> 5, j4 = 4 * (tid & 31);
        cp_async16(&S.E[B][k][j4], E + (size_t)cell_corner(g, k) * kLiftHidden + j4);
    } else if (tid < 132) {
        cp_async4(&S.sS[B][tid - 128], s + cell_corner(g, tid - 128), true);
    } else if (tid < 142) {
        cp_async4(&S.sG[B][tid - 132], gram + (size_t)cell * 10 + (tid - 132), true);
    }
}

size_t lift_tc_smem_bytes() { return (size_t)lt::kOpBytes + sizeof(LiftTcSmem) + 1024; }

// hi and lo BF16 pairs of (a, b), a at the lower address
__device__ __forceinline__ void split2_bf16(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// 4 values as one 16-byte core-matrix row of the TF32 hi and of the lo tile
// (hi = tf32(x), lo = tf32(x - hi))
__device__ __forceinline__ void put4_tf32(float *hi, float *lo, uint32_t off, float4 v) {
    float4 h, l;
    h.x = umma::tf32_hi(v.x);
    h.y = umma::tf32_hi(v.y);
    h.z = umma::tf32_hi(v.z);
    h.w = umma::tf32_hi(v.w);
    l.x = umma::tf32_hi(v.x - h.x);
    l.y = umma::tf32_hi(v.y - h.y);
    l.z = umma::tf32_hi(v.z - h.z);
    l.w = umma::tf32_hi(v.w - h.w);
    *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(hi) + off) = h;
    *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(lo) + off) = l;
}

// 8 values as one 16-byte core-matrix row of the hi and of the lo tile
__device__ __forceinline__ void put8_split(unsigned char *hi, unsigned char *lo, uint32_t off, const float (&v)[8]) {
    uint4 h, l;
    split2_bf16(v[0], v[1], h.x, l.x);
    split2_bf16(v[2], v[3], h.y, l.y);
    split2_bf16(v[4], v[5], h.z, l.z);
    split2_bf16(v[6], v[7], h.w, l.w);
    *reinterpret_cast<uint4 *>(hi + off) = h;
    *reinterpret_cast<uint4 *>(lo + off) = l;
}

// Sum over the warp's lanes of v[lane]: the 32 values of every lane are
// reduce-scattered, lane l keeps the total of entry l.
__device__ __forceinline__ float warp_rs32(float (&v)[32], int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int t = 0; t < s; ++t) {
            const float send = up ? v[t] : v[t + s];
            const float keep = up ? v[t + s] : v[t];
            v[t] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

__global__ void __launch_bounds__(lt::kT, 1) k_lift_tc(
    ViewTable vt, int n_cells, int patch, const float *__restrict__ feat_all, const float *__restrict__ w1,
    const float *__restrict__ b1, const float *__restrict__ Mg, const float *__restrict__ E,
    const float *__restrict__ s, const float *__restrict__ u, const float *__restrict__ beta,
    const float *__restrict__ gram, const float *__restrict__ weight_all, float g0, float *__restrict__ loss,
    float *__restrict__ D, float *__restrict__ alpha, float *__restrict__ sb, float *__restrict__ hb_out,
    float *__restrict__ Gb, float *__restrict__ d_w1, float *__restrict__ d_b1, float *__restrict__ d_feat_all,
    int *__restrict__ err) {
    using namespace lt;
    constexpr int NF = 16;
    extern __shared__ __align__(1024) unsigned char smem_lt[];
    unsigned char *op = smem_lt + ((1024u - (umma::smem_addr(smem_lt) & 1023u)) & 1023u);
    LiftTcSmem &S = *reinterpret_cast<LiftTcSmem *>(op + kOpBytes);
    const uint32_t sop = umma::smem_addr(op);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kLiftHidden * NF; i += kT) {
        const int j = i / NF, c = i - j * NF;
        S.W1r[j][c] = w1[i];
    }
    for (int i = tid; i < kLiftHidden * (NF / 4); i += kT) {  // W1 row j, channels 4 q + [0, 4)
        const int j = i / (NF / 4), q = i % (NF / 4);
        const float4 v = make_float4(w1[j * NF + 4 * q], w1[j * NF + 4 * q + 1], w1[j * NF + 4 * q + 2],
                                     w1[j * NF + 4 * q + 3]);
        put4_tf32(S.W1A[0], S.W1A[1], umma::kmajor_offset(j, 4 * q, 4 * NF, 4), v);
    }
    if (tid < kLiftHidden) {
        S.b1[tid] = b1[tid];
        S.u[tid] = u[tid];
    }
    if (tid == 0) {
        int base = 0;
        for (int v = 0; v < vt.n; ++v) {
            const int wp = (vt.v[v].W + patch - 1) / patch, hp = (vt.v[v].H + patch - 1) / patch;
            S.vwp[v] = wp;
            S.vhp[v] = hp;
            S.vbase[v] = base;
            base += wp * hp;
        }
        umma::mbar_init(&S.mh_bar, 1);
        umma::mbar_init(&S.g_bar, 1);
        S.abort_flag = 0;
    }
    if (warp == 0) umma::tmem_alloc(&S.tmem_base, kTmemCols);
    umma::fence_before();
    umma::fence_async_smem();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = S.tmem_base;
    const int jt = 32 * (warp & 3) + lane, ph = 32 * (warp >> 2);
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    // M (symmetric) as BF16 hi/lo pairs into TMEM: lane jt = row jt, the
    // thread's warp half writes k in [64 (w / 4), + 64)
#pragma unroll 1
    for (int k0 = 2 * ph; k0 < 2 * ph + 64; k0 += 32) {
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 m = *reinterpret_cast<const float4 *>(Mg + (size_t)jt * kLiftHidden + k0 + 4 * q);
            split2_bf16(m.x, m.y, hi[2 * q], lo[2 * q]);
            split2_bf16(m.z, m.w, hi[2 * q + 1], lo[2 * q + 1]);
        }
        umma::tmem_st16(lane_addr + cMhi + k0 / 2, hi);
        umma::tmem_st16(lane_addr + cMlo + k0 / 2, lo);
    }
    umma::tmem_st_wait();
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const float bt = *beta;
    const float inv2p = 1.f / (float)(2 * patch);
    float hb = 0.f, db1 = 0.f;
    float t_loss = 0.f, t_sb = 0.f;
    uint32_t mh_phase = 0, g_phase = 0;
    bool g_pending = false, g_started = false, mh_pending = false, ok = true;
    const uint32_t id_mh = umma::idesc(umma::kBF16, 128, kP), id_g = umma::idesc(umma::kBF16, 128, 128),
                   id_dw = umma::idesc(umma::kBF16, 128, NF), id_z = umma::idesc(umma::kTF32, 128, kP);
    float *red = &S.red[0][0][0];  // [4][kP][2]
    // the chunk whose inputs are in flight to buffer buf (cell -1: none)
    int pre_cell = -1, pre_q0 = 0, buf = 0;
    if ((int)blockIdx.x < n_cells) {
        lift_chunk_issue(S, 0, vt, patch, blockIdx.x, 0, feat_all, d_feat_all, weight_all, E, s, gram, tid);
        pre_cell = blockIdx.x;
    }
    cp_async_commit();
    for (int cell = blockIdx.x; cell < n_cells && ok; cell += gridDim.x) {
        const CellGeo cg = cell_geo(S, vt, patch, cell);
        const int W = cg.W, nx = cg.nx, npx = cg.npx, xs = cg.xs, ys = cg.ys, x0 = cg.x0, y0 = cg.y0;
        const size_t HW = cg.HW, P = cg.P;
        float *d_feat = d_feat_all ? d_feat_all + (size_t)NF * P : nullptr;
        const float *weight = weight_all ? weight_all + P : nullptr;
        const int corner[4] = {cell_corner(cg, 0), cell_corner(cg, 1), cell_corner(cg, 2), cell_corner(cg, 3)};
        __syncthreads();  // the previous cell's shared data is no longer read
        for (int i = tid; i < 4 * kLiftHidden; i += kT) (&S.Dpart[0][0])[i] = 0.f;
        float al[4] = {0.f, 0.f, 0.f, 0.f};  // sum a w_k over the cell (threads < kP)
        for (int q0 = 0; q0 < npx; q0 += kP) {
            __syncthreads();
            // chunk pixels and their bilinear weights
            if (tid < kP) {
                const int q = q0 + tid;
                int pidx = -1;
                float w[4] = {0.f, 0.f, 0.f, 0.f};
                if (q < npx) {
                    const int y = ys + q / nx, x = xs + q % nx;
                    pidx = y * W + x;
                    const float ax = fminf(fmaxf((float)(2 * x + 1 - (2 * x0 + 1) * patch) * inv2p, 0.f), 1.f);
                    const float ay = fminf(fmaxf((float)(2 * y + 1 - (2 * y0 + 1) * patch) * inv2p, 0.f), 1.f);
                    w[0] = (1.f - ax) * (1.f - ay);
                    w[1] = ax * (1.f - ay);
                    w[2] = (1.f - ax) * ay;
                    w[3] = ax * ay;
                }
                S.pix[tid] = pidx;
#pragma unroll
                for (int k = 0; k < 4; ++k) S.w4[tid][k] = w[k];
            }
            // this chunk's global inputs were issued a chunk ahead (else now);
            // the next chunk's go to the other buffer, whose last reader (the
            // previous chunk) every thread has passed
            if (pre_cell != cell || pre_q0 != q0) {
                cp_async_wait<0>();
                lift_chunk_issue(S, buf, vt, patch, cell, q0, feat_all, d_feat_all, weight_all, E, s, gram, tid);
                cp_async_commit();
            }
            cp_async_wait<0>();
            // the previous chunk's Gram MMAs still read the H and b H tiles
            if (g_pending) {
                const bool w_ok = umma::mbar_wait(&S.g_bar, g_phase, kWait);
                g_phase ^= 1u;
                g_pending = false;
                if (!w_ok) S.abort_flag = 1;
            }
            __syncthreads();
            if (S.abort_flag) {
                ok = false;
                break;
            }
            umma::fence_after();
            // F~ as the TF32 hi / lo B tile of Z (pixel rows, channels along K)
            if (tid >= 128) {
                const int p = (tid - 128) & (kP - 1);
#pragma unroll
                for (int q = (tid - 128) >> 6; q < NF / 4; q += 2) {
                    const float4 v = make_float4(S.Fc[buf][4 * q][p], S.Fc[buf][4 * q + 1][p], S.Fc[buf][4 * q + 2][p],
                                                 S.Fc[buf][4 * q + 3][p]);
                    put4_tf32(S.FcN[0], S.FcN[1], umma::kmajor_offset(p, 4 * q, 4 * NF, 4), v);
                }
            }
            umma::fence_async_smem();
            __syncthreads();
            // Z = W1 F~ on the tensor cores in 3xTF32 (hi hi + hi lo + lo hi, two K
            // steps of 8, FP32 accumulation in the M H columns, free until M H): its
            // sign decides ReLU', so the operands keep about 22 bits (a BF16 hi / lo
            // split, about 16, flipped enough near-zero units to fail the dF~ bar)
            if (tid == 0) {
                umma::fence_after();
                const uint32_t whi = umma::smem_addr(S.W1A[0]), wlo = umma::smem_addr(S.W1A[1]);
                const uint32_t fhi = umma::smem_addr(S.FcN[0]), flo = umma::smem_addr(S.FcN[1]);
                for (int ks = 0; ks < NF / 8; ++ks) {
                    const uint32_t o = 256u * ks;
                    umma::mma<umma::kTF32>(tmem + cMH, umma::desc(whi + o, 4 * NF), umma::desc(fhi + o, 4 * NF), id_z,
                                           ks > 0 ? 1u : 0u);
                    umma::mma<umma::kTF32>(tmem + cMH, umma::desc(whi + o, 4 * NF), umma::desc(flo + o, 4 * NF), id_z,
                                           1u);
                    umma::mma<umma::kTF32>(tmem + cMH, umma::desc(wlo + o, 4 * NF), umma::desc(fhi + o, 4 * NF), id_z,
                                           1u);
                }
                umma::commit(&S.mh_bar);
            }
            mh_pending = true;
            // while the Z MMAs run: the next chunk's global inputs to the other
            // buffer (its last reader, the previous chunk, every thread has
            // passed) and F~ as the dW1 B tile
            {
                int ncell = cell, nq0 = q0 + kP;
                if (nq0 >= npx) {
                    ncell = cell + gridDim.x;
                    nq0 = 0;
                }
                pre_cell = -1;
                if (ncell < n_cells) {
                    lift_chunk_issue(S, buf ^ 1, vt, patch, ncell, nq0, feat_all, d_feat_all, weight_all, E, s, gram,
                                     tid);
                    pre_cell = ncell;
                    pre_q0 = nq0;
                }
                cp_async_commit();
            }
            // F~ as the BF16 hi / lo B tile of dW1 (channel rows, pixels along K);
            // the previous chunk's dW1 MMAs, which read it, completed with the Gram's
            if (d_w1 && tid < 128) {
                const int c = tid >> 3, p8 = 8 * (tid & 7);
                const float4 f0 = *reinterpret_cast<const float4 *>(&S.Fc[buf][c][p8]);
                const float4 f1 = *reinterpret_cast<const float4 *>(&S.Fc[buf][c][p8 + 4]);
                const float v[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
                put8_split(reinterpret_cast<unsigned char *>(S.FcT[0]), reinterpret_cast<unsigned char *>(S.FcT[1]),
                           umma::kmajor_offset(c, p8, 2 * kP, 2), v);
            }
            {
                const bool w_ok = umma::mbar_wait(&S.mh_bar, mh_phase, kWait);
                if (w_ok) {
                    mh_phase ^= 1u;
                    mh_pending = false;
                }
                if (__syncthreads_or(!w_ok)) {
                    if (tid == 0) S.abort_flag = 1;
                    ok = false;
                    break;
                }
            }
            umma::fence_after();
            // H = relu(Z + b1) of (jt, pixel half): registers, the Gram A tile
            // (row jt) and M H's B tile
            float hv[32];
            {
                const float bj = S.b1[jt];
                float t16[16];
                umma::tmem_ld16(lane_addr + cMH + ph, t16);
#pragma unroll
                for (int t = 0; t < 16; ++t) hv[t] = fmaxf(t16[t] + bj, 0.f);
                umma::tmem_ld16(lane_addr + cMH + ph + 16, t16);
#pragma unroll
                for (int t = 0; t < 16; ++t) hv[16 + t] = fmaxf(t16[t] + bj, 0.f);
            }
            {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) split2_bf16(hv[2 * t], hv[2 * t + 1], hi[t], lo[t]);
                umma::tmem_st16(lane_addr + cHAhi + ph / 2, hi);
                umma::tmem_st16(lane_addr + cHAlo + ph / 2, lo);
                umma::tmem_st_wait();
            }
            // H as M H's B tile, pixel rows of 8 straight from the registers
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float v[8] = {hv[8 * q],     hv[8 * q + 1], hv[8 * q + 2], hv[8 * q + 3],
                                    hv[8 * q + 4], hv[8 * q + 5], hv[8 * q + 6], hv[8 * q + 7]};
                put8_split(op + oHBhi, op + oHBlo, hb_mn_offset(jt, ph + 8 * q), v);
            }
            umma::fence_before();
            umma::fence_async_smem();
            __syncthreads();
            // M H on the tensor cores
            if (tid == 0) {
                umma::fence_after();
                for (int pass = 0; pass < 3; ++pass) {
                    const uint32_t a = tmem + (pass == 2 ? cMlo : cMhi), b = sop + (pass == 1 ? oHBlo : oHBhi);
                    for (int ks = 0; ks < kLiftHidden / 16; ++ks)
                        umma::mma_f16_ts(tmem + cMH, a + 8u * ks, desc_strides(b + 2048u * ks, 1024, 128),
                                         id_mh | (1u << 16), (pass > 0 || ks > 0) ? 1u : 0u);
                }
                umma::commit(&S.mh_bar);
            }
            mh_pending = true;
            const float e0 = S.E[buf][0][jt], e1 = S.E[buf][1][jt], e2 = S.E[buf][2][jt], e3 = S.E[buf][3][jt],
                        uj = S.u[jt];
            auto e_at = [&](int t) {
                const float4 w = *reinterpret_cast<const float4 *>(&S.w4[ph + t][0]);
                return w.x * e0 + w.y * e1 + w.z * e2 + w.w * e3;
            };
            // per pixel over this warp's 32 hidden units: H.e (while the M H
            // MMAs run), then H.(M H + 2 u), the two sums the cosine needs
            // (|F^|^2 = H.M H + 2 u.H + |b2|^2)
            {
                float v[32];
#pragma unroll
                for (int t = 0; t < 32; ++t) v[t] = hv[t] * e_at(t);
                red[((warp & 3) * kP + ph + lane) * 2 + 0] = warp_rs32(v, lane);
            }
            {
                const bool w_ok = umma::mbar_wait(&S.mh_bar, mh_phase, kWait);
                if (w_ok) {
                    mh_phase ^= 1u;
                    mh_pending = false;
                }
                if (__syncthreads_or(!w_ok)) {
                    if (tid == 0) S.abort_flag = 1;
                    ok = false;
                    break;
                }
            }
            umma::fence_after();
            // thread (jt, pixel half ph): its M H row, the corner terms
            float mh[32];
            {
                float t16[16];
                umma::tmem_ld16(lane_addr + cMH + ph, t16);
#pragma unroll
                for (int t = 0; t < 16; ++t) mh[t] = t16[t];
                umma::tmem_ld16(lane_addr + cMH + ph + 16, t16);
#pragma unroll
                for (int t = 0; t < 16; ++t) mh[16 + t] = t16[t];
            }
            {
                float v[32];
#pragma unroll
                for (int t = 0; t < 32; ++t) v[t] = hv[t] * fmaf(2.f, uj, mh[t]);
                red[((warp & 3) * kP + ph + lane) * 2 + 1] = warp_rs32(v, lane);
            }
            __syncthreads();
            // per pixel: cosine, loss, a_p, b_p
            if (tid < kP) {
                const int p = tid;
                float de = 0.f, dmu = 0.f;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    de += red[(b * kP + p) * 2 + 0];
                    dmu += red[(b * kP + p) * 2 + 1];
                }
                const float *w = S.w4[p];
                const float *sS = S.sS[buf], *sG = S.sG[buf];
                const float dot = de + w[0] * sS[0] + w[1] * sS[1] + w[2] * sS[2] + w[3] * sS[3];
                const float nF2 = w[0] * w[0] * sG[0] + w[1] * w[1] * sG[4] + w[2] * w[2] * sG[7] +
                                  w[3] * w[3] * sG[9] +
                                  2.f * (w[0] * w[1] * sG[1] + w[0] * w[2] * sG[2] + w[0] * w[3] * sG[3] +
                                         w[1] * w[2] * sG[5] + w[1] * w[3] * sG[6] + w[2] * w[3] * sG[8]);
                const float nFh2 = dmu + bt;
                float a = 0.f, b = 0.f;
                const int pidx = S.pix[p];
                if (pidx >= 0) {
                    const bool okp = nF2 > 0.f && nFh2 > 0.f;
                    const float wpx = weight ? S.wpx[buf][p] : 1.f;
                    const float g = g0 * wpx;
                    const float inv = okp ? rsqrtf(nF2) * rsqrtf(nFh2) : 0.f;
                    const float cs = dot * inv;
                    t_loss += wpx * (1.f - cs);
                    a = -g * inv;
                    b = okp ? g * cs / nFh2 : 0.f;
                    t_sb += b;
                }
                S.ab[p][0] = a;
                S.ab[p][1] = b;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    S.aw[p][k] = a * w[k];
                    al[k] += a * w[k];
                }
            }
            __syncthreads();
            // dZ (to Hh), b H (to the Gram B tile), db1, hb and D of the corners
            // (thread jt over its pixel half)
            {
                float Dk[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int p = ph + t;
                    // dL/dH = a e_p + b (M H + u), a e_p = sum_k (a w_k) e_k
                    const float bp = S.ab[p][1];
                    const float4 awp = *reinterpret_cast<const float4 *>(&S.aw[p][0]);
                    const float dh =
                        fmaf(awp.x, e0, fmaf(awp.y, e1, fmaf(awp.z, e2, fmaf(awp.w, e3, bp * (mh[t] + uj)))));
                    const float dz = hv[t] > 0.f ? dh : 0.f;
                    Dk[0] = fmaf(awp.x, hv[t], Dk[0]);
                    Dk[1] = fmaf(awp.y, hv[t], Dk[1]);
                    Dk[2] = fmaf(awp.z, hv[t], Dk[2]);
                    Dk[3] = fmaf(awp.w, hv[t], Dk[3]);
                    db1 += dz;
                    hb = fmaf(bp, hv[t], hb);
                    mh[t] = dz;
                    hv[t] *= bp;
                }
#pragma unroll
                for (int t4 = 0; t4 < 8; ++t4)
                    *reinterpret_cast<float4 *>(&S.Hh[jt][ph + 4 * t4]) =
                        make_float4(mh[4 * t4], mh[4 * t4 + 1], mh[4 * t4 + 2], mh[4 * t4 + 3]);
#pragma unroll
                for (int c8 = 0; c8 < 4; ++c8) {
                    const float v[8] = {hv[8 * c8],     hv[8 * c8 + 1], hv[8 * c8 + 2], hv[8 * c8 + 3],
                                        hv[8 * c8 + 4], hv[8 * c8 + 5], hv[8 * c8 + 6], hv[8 * c8 + 7]};
                    put8_split(op + oBHhi, op + oBHlo, umma::kmajor_offset(jt, ph + 8 * c8, 2 * kP, 2), v);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) atomicAdd(&S.Dpart[k][jt], Dk[k]);
                if (d_w1) {  // dZ as the A operand of dW1 (row jt, pixel pairs)
                    uint32_t hi[16], lo[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) split2_bf16(mh[2 * q], mh[2 * q + 1], hi[q], lo[q]);
                    umma::tmem_st16(lane_addr + cDZhi + ph / 2, hi);
                    umma::tmem_st16(lane_addr + cDZlo + ph / 2, lo);
                    umma::tmem_st_wait();
                }
            }
            umma::fence_before();
            umma::fence_async_smem();
            __syncthreads();
            // Gram += H (b H)^T on the tensor cores, left running
            if (tid == kGramTid) {
                umma::fence_after();
                for (int pass = 0; pass < 3; ++pass) {
                    const uint32_t a = tmem + (pass == 2 ? cHAlo : cHAhi), b = sop + (pass == 1 ? oBHlo : oBHhi);
                    for (int ks = 0; ks < kP / 16; ++ks)
                        umma::mma_f16_ts(tmem + cG, a + 8u * ks, umma::desc(b + 256u * ks, 2 * kP), id_g,
                                         (g_started || pass > 0 || ks > 0) ? 1u : 0u);
                }
                // dW1 += dZ F~^T: A = dZ in TMEM, B = the F~ tile, accumulated over the CTA's chunks
                if (d_w1) {
                    const uint32_t fhi = umma::smem_addr(S.FcT[0]), flo = umma::smem_addr(S.FcT[1]);
                    for (int pass = 0; pass < 3; ++pass) {
                        const uint32_t a = tmem + (pass == 2 ? cDZlo : cDZhi), b = pass == 1 ? flo : fhi;
                        for (int ks = 0; ks < kP / 16; ++ks)
                            umma::mma_f16_ts(tmem + cDW, a + 8u * ks, umma::desc(b + 256u * ks, 2 * kP), id_dw,
                                             (g_started || pass > 0 || ks > 0) ? 1u : 0u);
                    }
                }
                umma::commit(&S.g_bar);
            }
            g_started = true;
            g_pending = true;
            if (d_feat) {
                // dF~ = W1^T dZ: each warp sums a range of hidden units for all
                // channels of lane l's pixels 2 l and 2 l + 1, channel pairs packed
                // (the warp that issued the Gram and dW1 MMAs takes 2 units, the
                // other seven 18); W1 rows come in warp-uniform loads, and the eight
                // warps' partial sums meet in the M H operand tile, free until the
                // next chunk
                constexpr int kIssueWarp = kGramTid / 32, kShort = 2, kLong = (kLiftHidden - kShort) / 7;
                static_assert(7 * kLong + kShort == kLiftHidden, "hidden units over the dF~ warps");
                const int j0 = warp < kIssueWarp ? kLong * warp : warp == kIssueWarp ? kLong * warp
                                                                                     : kLong * (warp - 1) + kShort;
                const int nj = warp == kIssueWarp ? kShort : kLong;
                f2 acc[NF / 2][2];  // [channel pair][pixel]
#pragma unroll
                for (int k = 0; k < NF / 2; ++k) acc[k][0] = acc[k][1] = 0ull;
#pragma unroll 2
                for (int jj = 0; jj < nj; ++jj) {
                    const int j = j0 + jj;
                    const float2 dz = *reinterpret_cast<const float2 *>(&S.Hh[j][2 * lane]);
                    const f2 d0 = f2_make(dz.x, dz.x), d1 = f2_make(dz.y, dz.y);
#pragma unroll
                    for (int k4 = 0; k4 < NF / 4; ++k4) {
                        const ulonglong2 w = *reinterpret_cast<const ulonglong2 *>(&S.W1r[j][4 * k4]);
                        acc[2 * k4][0] = f2_fma(w.x, d0, acc[2 * k4][0]);
                        acc[2 * k4][1] = f2_fma(w.x, d1, acc[2 * k4][1]);
                        acc[2 * k4 + 1][0] = f2_fma(w.y, d0, acc[2 * k4 + 1][0]);
                        acc[2 * k4 + 1][1] = f2_fma(w.y, d1, acc[2 * k4 + 1][1]);
                    }
                }
                float *part = reinterpret_cast<float *>(op + oHBhi);  // [8 warps][NF][kP]
#pragma unroll
                for (int k = 0; k < NF / 2; ++k) {
                    float a0, b0, a1, b1;  // (channel 2 k, 2 k + 1) at pixels 2 l and 2 l + 1
                    f2_split(acc[k][0], a0, b0);
                    f2_split(acc[k][1], a1, b1);
                    *reinterpret_cast<float2 *>(&part[(warp * NF + 2 * k) * kP + 2 * lane]) = make_float2(a0, a1);
                    *reinterpret_cast<float2 *>(&part[(warp * NF + 2 * k + 1) * kP + 2 * lane]) = make_float2(b0, b1);
                }
                __syncthreads();
                // thread t: channel t / 16, pixels 4 (t % 16) + [0, 4)
                const int c = tid >> 4, p0 = 4 * (tid & 15);
                const float4 d4 = *reinterpret_cast<const float4 *>(&S.dF0[buf][c][p0]);
                float sum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    const float4 v = *reinterpret_cast<const float4 *>(&part[(w * NF + c) * kP + p0]);
                    sum[0] += v.x;
                    sum[1] += v.y;
                    sum[2] += v.z;
                    sum[3] += v.w;
                }
                const float o[4] = {d4.x, d4.y, d4.z, d4.w};
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int pidx = S.pix[p0 + y];
                    if (pidx >= 0) d_feat[(size_t)c * HW + pidx] = o[y] + sum[y];
                }
            }
            buf ^= 1;
        }
        if (!ok) break;
        __syncthreads();
        // the cell's D rows and alpha
        for (int i = tid; i < 4 * kLiftHidden; i += kT) {
            const int k = i / kLiftHidden, j = i - k * kLiftHidden;
            if (npx > 0) atomicAdd(D + (size_t)corner[k] * kLiftHidden + j, S.Dpart[k][j]);
        }
        if (tid < kP && npx > 0)
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(alpha + corner[k], al[k]);
    }
    cp_async_wait<0>();  // no copy still writes shared memory
    // the last Gram MMAs (and an M H that a wait gave up on), then the CTA's sums
    if (mh_pending && !umma::mbar_wait(&S.mh_bar, mh_phase, kWait)) S.abort_flag = 1;
    if (g_pending) {
        const bool w_ok = umma::mbar_wait(&S.g_bar, g_phase, kWait);
        g_phase ^= 1u;
        if (!w_ok) S.abort_flag = 1;
    }
    __syncthreads();
    umma::fence_after();
    ok = ok && !S.abort_flag;
    if (ok && g_started) {
        // Gram (symmetric): thread jt, the half of the columns its warp's pixel half names
#pragma unroll 1
        for (int c0 = 0; c0 < kLiftHidden / 2; c0 += 16) {
            float d[16];
            umma::tmem_ld16(lane_addr + cG + 2 * ph + c0, d);
#pragma unroll
            for (int t = 0; t < 16; ++t) atomicAdd(Gb + (size_t)jt * kLiftHidden + 2 * ph + c0 + t, d[t]);
        }
    }
    if (!ok && tid == 0 && err) atomicExch(err, 1);
    if (ok) {
        atomicAdd(hb_out + jt, hb);
        if (d_b1) atomicAdd(d_b1 + jt, db1);
        if (d_w1 && g_started && warp < 4) {  // dW1 row jt from TMEM
            float d[16];
            umma::tmem_ld16(lane_addr + cDW, d);
#pragma unroll
            for (int c = 0; c < NF; ++c) atomicAdd(d_w1 + (size_t)jt * NF + c, d[c]);
        }
        float v2[2] = {t_loss, t_sb};
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v2[i] += __shfl_xor_sync(0xffffffffu, v2[i], o);
        if (lane == 0) {
            atomicAdd(loss, g0 * v2[0]);
            atomicAdd(sb, v2[1]);
        }
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, kTmemCols);
}

// y[i] += x[i] * (*c)
__global__ void k_axpy_dev(int n, const float *__restrict__ x, const float *__restrict__ c, float *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fmaf(x[i], *c, y[i]);
}

size_t round64(size_t n) { return (n + 63) & ~size_t(63); }

// scratch of one call, in floats (np: patches of all views)
struct LiftLayout {
    size_t E, s, M, u, beta, gram, D, alpha, hb, sb, Gb, total;
};
LiftLayout lift_layout(size_t np) {
    LiftLayout L{};
    size_t o = 0;
    auto take = [&](size_t n) {
        const size_t at = o;
        o += round64(n);
        return at;
    };
    L.E = take(kLiftHidden * np);
    L.s = take(np);
    L.M = take(kLiftHidden * kLiftHidden);
    L.u = take(kLiftHidden);
    L.beta = take(1);
    L.gram = take(10 * np);
    // D, alpha, hb, sb: one run, cleared per call
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

size_t lift_scratch_floats(size_t np_total) { return lift_layout(np_total).total; }

// All views at once: forward, loss and backward.  feat / d_feat: the image
// layout (view v's nf planes at nf * P_v); grid: the views' patch grids
// concatenated ([np_total][nh], view after view); weight: the per-pixel
// weights in the depth layout (null: 1); scratch: lift_scratch_floats(np_total).
// d_w1 [128][nf], d_b1 [128], d_w2 [nh][128], d_b2 [nh] and d_feat are
// accumulated (may be null: that gradient is skipped).
cudaError_t lift_all(int num_sms, cudaStream_t st, const ViewTable &vt, int nf, int nh, int patch, const float *feat,
                     const float *grid, const float *w1, const float *b1, const float *w2, const float *b2, float g,
                     const float *weight, float *loss, float *d_w1, float *d_b1, float *d_w2, float *d_b2,
                     float *d_feat, float *scratch, int *err, int *launches) {
    int np = 0;
    for (int v = 0; v < vt.n; ++v) np += ((vt.v[v].H + patch - 1) / patch) * ((vt.v[v].W + patch - 1) / patch);
    const int NH = kLiftHidden;
    const LiftLayout L = lift_layout((size_t)np);
    float *E = scratch + L.E, *sv = scratch + L.s, *M = scratch + L.M, *u = scratch + L.u, *beta = scratch + L.beta;
    float *gram = scratch + L.gram, *D = scratch + L.D, *alpha = scratch + L.alpha, *hb = scratch + L.hb;
    float *sb = scratch + L.sb, *Gb = scratch + L.Gb;
    const dim3 blk(256);
    cudaError_t e;
    // weight-sized: M = W2^T W2, u = W2^T b2, beta = |b2|^2; per patch of every
    // view: E = G W2 ([np][128]), s = G b2
    if ((e = gemm_f32(st, false, true, NH, NH, nh, 1.f, w2, NH, w2, NH, 0.f, M, NH, num_sms, launches)) != cudaSuccess) return e;
    if ((e = gemm_f32(st, false, false, NH, 1, nh, 1.f, w2, NH, b2, nh, 0.f, u, NH, num_sms, launches)) != cudaSuccess) return e;
    if ((e = gemm_f32(st, true, false, 1, 1, nh, 1.f, b2, nh, b2, nh, 0.f, beta, 1, num_sms, launches)) != cudaSuccess) return e;
    if ((e = gemm_f32(st, false, false, NH, np, nh, 1.f, w2, NH, grid, nh, 0.f, E, NH, num_sms, launches)) != cudaSuccess) return e;
    if ((e = gemm_f32(st, true, false, np, 1, nh, 1.f, grid, nh, b2, nh, 0.f, sv, np, num_sms, launches)) != cudaSuccess) return e;
    k_cell_gram<<<(unsigned)((np + 7) / 8), blk, 0, st>>>(vt, patch, np, grid, nh, gram);
    ++*launches;
    // the fused kernel adds into D, alpha, hb, sb and Gb
    if ((e = cudaMemsetAsync(D, 0, (L.sb + 1 - L.D) * sizeof(float), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Gb, 0, (size_t)NH * NH * sizeof(float), st)) != cudaSuccess) return e;
    const int grid_ctas = std::max(1, std::min(np, num_sms));
    if (nf == 16) {
        // M H and the Gram on the tensor cores
        const size_t smem = lift_tc_smem_bytes();
        // one CTA per SM: it holds all 512 TMEM columns
        if (smem > 227 * 1024 || 2 * (smem + 1024) <= 228 * 1024) return cudaErrorInvalidConfiguration;
        cudaFuncSetAttribute(k_lift_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_lift_tc<<<grid_ctas, lt::kT, smem, st>>>(vt, np, patch, feat, w1, b1, M, E, sv, u, beta, gram, weight, g,
                                                   loss, D, alpha, sb, hb, Gb, d_w1, d_b1, d_feat, err);
    } else if (nf == 32) {
        // the BF16 operand tiles and the FP32 arrays of N_l = 32 exceed shared memory: all FP32 on the CUDA cores
        const size_t smem = fused_smem_bytes(nf);
        cudaFuncSetAttribute(k_lift_fused<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_lift_fused<32><<<grid_ctas, kFT, smem, st>>>(vt, np, patch, feat, w1, b1, M, E, sv, u, beta, gram, weight,
                                                       g, loss, D, alpha, sb, hb, Gb, d_w1, d_b1, d_feat);
    } else {
        return cudaErrorInvalidValue;
    }
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (d_w2) {
        // dW2 ([nh][128] row-major = column-major 128 x nh) += D G, Gb W2, hb b2^T
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
    return cudaGetLastError();
}

}  // namespace ups
