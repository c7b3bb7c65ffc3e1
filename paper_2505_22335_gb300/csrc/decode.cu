// Per-anchor MLP decode of K neural Gaussians (Eq. 8-9) and its backward,
// FP32 on the CUDA cores.
//
// Row = (anchor, view).  MLP input x = [f_v, delta_vc, d_vc, sin(pi t),
// cos(pi t)]; four MLPs (opacity, covariance, colour: ReLU hidden; feature
// F_d: SoftPlus hidden) of width `hidden` = 32.  Weights live in shared memory
// and are read as float4 broadcasts (every lane of a warp reads the same
// weight), so the inner loops are FMA-bound.
//
// Backward (FP32 data path): one thread per row recomputes each MLP group's
// hidden layer, forms dL/dY of the group's outputs and propagates it to the
// hidden layer and the MLP input (k_decode_bwd_rows); the hidden activations
// and pre-activation gradients go to a feature-major scratch from which the
// weight gradients are reduced by a separate kernel (decode_bwd_tc.cu).
#include <algorithm>

#include "decode_bwd.cuh"

namespace ups {

namespace {

constexpr int kH = 32;       // hidden width per MLP
constexpr int kFin = 32;     // anchor feature width
constexpr int kDin = kFin + 6;
constexpr int kDinP = 40;    // padded input width (float4 rows)
constexpr int kDX = kFin + 4;  // MLP inputs with a gradient: f_v, delta_vc, d_vc
constexpr size_t kMaxSmem = 227 * 1024;  // opt-in shared memory per block

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + __expf(-x)); }
__device__ __forceinline__ float softplus(float x) { return x > 20.f ? x : log1pf(__expf(x)); }
__device__ __forceinline__ float opacity_act(float y, int op_tanh) { return op_tanh ? tanhf(y) : sigm(y); }

struct DecodeArgs {
    int A, K, NF, n_out;
    const float *pos, *afeat, *offs, *ascale;
    const float *w1, *b1, *w2, *b2;
    int op_tanh;  // opacity = tanh(y) (Scaffold-GS form) instead of sigmoid(y)
};

// x (padded to 40) for anchor `an` seen from view `cam`; returns delta and d.
__device__ __forceinline__ void mlp_input(const DecodeArgs &a, const DevView &cam, int an,
                                          float x[kDinP], float delta[3], float &dist) {
    const float4 *f4 = reinterpret_cast<const float4 *>(a.afeat + (size_t)an * kFin);
#pragma unroll
    for (int i = 0; i < kFin / 4; ++i) {
        float4 f = f4[i];
        x[4 * i] = f.x;
        x[4 * i + 1] = f.y;
        x[4 * i + 2] = f.z;
        x[4 * i + 3] = f.w;
    }
    // camera centre o_c = -R^T t
    float oc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        oc[i] = -(cam.R[i] * cam.t[0] + cam.R[3 + i] * cam.t[1] + cam.R[6 + i] * cam.t[2]);
    float r[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] = a.pos[3 * an + i] - oc[i];
    dist = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    float id = 1.f / dist;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        delta[i] = r[i] * id;
        x[kFin + i] = delta[i];
    }
    x[kFin + 3] = dist;
    float s, c;
    sincospif(cam.t_norm, &s, &c);
    x[kFin + 4] = s;
    x[kFin + 5] = c;
    x[38] = 0.f;
    x[39] = 0.f;
}

// hidden block g: z = W1_g x + b1_g (32 values, held as 16 packed pairs
// (z_2p, z_2p+1) for fma.rn.f32x2), input-outer so the accumulators stay in
// registers.  W1 is transposed in shared memory ([38][128]: input-major); the
// anchor-feature part of x is read through L1 (rows of the same anchor share
// it), the camera-dependent tail x[32..37] comes in registers.  Each element
// is rounded exactly as a scalar fmaf chain over the inputs in order.
constexpr int kH2 = kH / 2;
__device__ __forceinline__ void hidden_T(const float *sW1T, const float *sb1, int g, const float *afeat_row,
                                         const float xt[6], f2 h[kH2]) {
    const f2 *b2 = reinterpret_cast<const f2 *>(sb1 + g * kH);
#pragma unroll
    for (int p = 0; p < kH2; ++p) h[p] = b2[p];
    const float4 *f4 = reinterpret_cast<const float4 *>(afeat_row);
    // the next four inputs are loaded while the current four are applied (one
    // load in flight per step instead of a stall on each)
    float4 nxt = __ldg(f4);
#pragma unroll 1
    for (int i4 = 0; i4 < kFin / 4; ++i4) {
        const float4 xv = nxt;
        if (i4 + 1 < kFin / 4) nxt = __ldg(f4 + i4 + 1);
        const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const ulonglong2 *w = reinterpret_cast<const ulonglong2 *>(sW1T + (4 * i4 + u) * 128 + g * kH);
            const f2 xx = f2_make(xs[u], xs[u]);
#pragma unroll
            for (int q = 0; q < kH / 4; ++q) {
                const ulonglong2 ww = w[q];
                h[2 * q] = f2_fma(ww.x, xx, h[2 * q]);
                h[2 * q + 1] = f2_fma(ww.y, xx, h[2 * q + 1]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 6; ++u) {
        const ulonglong2 *w = reinterpret_cast<const ulonglong2 *>(sW1T + (kFin + u) * 128 + g * kH);
        const f2 xx = f2_make(xt[u], xt[u]);
#pragma unroll
        for (int q = 0; q < kH / 4; ++q) {
            const ulonglong2 ww = w[q];
            h[2 * q] = f2_fma(ww.x, xx, h[2 * q]);
            h[2 * q + 1] = f2_fma(ww.y, xx, h[2 * q + 1]);
        }
    }
}

// element-wise activation of the packed hidden values: ReLU (act 0) or
// SoftPlus (act 1)
template <int ACT>
__device__ __forceinline__ void activate(f2 h[kH2]) {
#pragma unroll
    for (int p = 0; p < kH2; ++p) {
        float lo, hi;
        f2_split(h[p], lo, hi);
        h[p] = ACT == 0 ? f2_make(fmaxf(lo, 0.f), fmaxf(hi, 0.f)) : f2_make(softplus(lo), softplus(hi));
    }
}

// y_r = W2[r] . h + b2[r] with four partial sums (short dependency chains):
// the pairs (s0, s1) and (s2, s3) of the scalar form, summed (s0+s1)+(s2+s3)
__device__ __forceinline__ float out_row(const float *sW2, const float *sb2, int r, const f2 h[kH2]) {
    const ulonglong2 *w = reinterpret_cast<const ulonglong2 *>(sW2 + r * kH);
    f2 a01 = f2_make(sb2[r], 0.f), a23 = 0ull;
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
        const ulonglong2 ww = w[q];
        a01 = f2_fma(ww.x, h[2 * q], a01);
        a23 = f2_fma(ww.y, h[2 * q + 1], a23);
    }
    float s0, s1, s2, s3;
    f2_split(a01, s0, s1);
    f2_split(a23, s2, s3);
    return (s0 + s1) + (s2 + s3);
}

// shared layout of the decode kernels: W1 transposed [38][128], b1 [128],
// W2 [n_out][32], b2 [n_out] (padded to 4)
__device__ __forceinline__ void load_weights_T(const DecodeArgs &a, float *sW1T, float *sb1, float *sW2,
                                               float *sb2) {
    for (int i = threadIdx.x; i < kDin * 4 * kH; i += blockDim.x) {
        const int ii = i / (4 * kH), h = i - ii * (4 * kH);
        sW1T[i] = a.w1[h * kDin + ii];
    }
    for (int i = threadIdx.x; i < 4 * kH; i += blockDim.x) sb1[i] = a.b1[i];
    for (int i = threadIdx.x; i < a.n_out * kH; i += blockDim.x) sW2[i] = a.w2[i];
    for (int i = threadIdx.x; i < a.n_out; i += blockDim.x) sb2[i] = a.b2[i];
}

// forward decode: rows (threads) per CTA and resident CTAs per SM (its grid);
// 2 x 384 (24 warps at 80 registers) measured 0.90 ms against 0.95 for 4 x 128
// and 0.93 for 3 x 256 on the bench workload
#ifndef UPS_DECF_THREADS
#define UPS_DECF_THREADS 384
#endif
#ifndef UPS_DECF_CTAS
#define UPS_DECF_CTAS 2
#endif
constexpr int kFwdThreads = UPS_DECF_THREADS, kFwdCtas = UPS_DECF_CTAS;

template <int NF>
__global__ void __launch_bounds__(kFwdThreads, kFwdCtas) k_decode_fwd(ViewTable vt, DecodeArgs a,
                                                    float4 *__restrict__ mean_op,
                                                    float4 *__restrict__ scale_out,
                                                    float4 *__restrict__ quat_out,
                                                    float4 *__restrict__ color_out,
                                                    float *__restrict__ feat_out) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *sW1T = sm, *sb1 = sW1T + kDin * 4 * kH, *sW2 = sb1 + 4 * kH, *sb2 = sW2 + a.n_out * kH;
    load_weights_T(a, sW1T, sb1, sW2, sb2);
    __syncthreads();
    const int K = a.K;
    const int rows = a.A * vt.n;
    const size_t NG = (size_t)a.A * K;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += gridDim.x * blockDim.x) {
        const int v = row / a.A, an = row - v * a.A;
        const DevView &cam = vt.v[v];
        float xt[6];
        {
            float x[kDinP], delta[3], dist;
            mlp_input(a, cam, an, x, delta, dist);
#pragma unroll
            for (int u = 0; u < 6; ++u) xt[u] = x[kFin + u];
        }
        const float *af = a.afeat + (size_t)an * kFin;
        f2 z[kH2];
        const size_t gbase = (size_t)v * NG + (size_t)an * K;
        // opacity, and the mean
        hidden_T(sW1T, sb1, 0, af, xt, z);
        activate<0>(z);
        const float px = a.pos[3 * an], py = a.pos[3 * an + 1], pz = a.pos[3 * an + 2];
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            const float *o3 = a.offs + ((size_t)an * K + k) * 3;
            mean_op[gbase + k] = make_float4(px + o3[0], py + o3[1], pz + o3[2],
                                             opacity_act(out_row(sW2, sb2, k, z), a.op_tanh));
        }
        // covariance: 3 scale + 4 quaternion per Gaussian
        hidden_T(sW1T, sb1, 1, af, xt, z);
        activate<0>(z);
        const float lx = a.ascale[3 * an], ly = a.ascale[3 * an + 1], lz = a.ascale[3 * an + 2];
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            const int r = K + 7 * k;
            const float s0 = lx * sigm(out_row(sW2, sb2, r, z));
            const float s1 = ly * sigm(out_row(sW2, sb2, r + 1, z));
            const float s2 = lz * sigm(out_row(sW2, sb2, r + 2, z));
            const float q0 = out_row(sW2, sb2, r + 3, z), q1 = out_row(sW2, sb2, r + 4, z);
            const float q2 = out_row(sW2, sb2, r + 5, z), q3 = out_row(sW2, sb2, r + 6, z);
            scale_out[gbase + k] = make_float4(s0, s1, s2, 0.f);
            quat_out[gbase + k] = make_float4(q0, q1, q2, q3);
        }
        // colour
        hidden_T(sW1T, sb1, 2, af, xt, z);
        activate<0>(z);
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            const int r = 8 * K + 3 * k;
            color_out[gbase + k] = make_float4(sigm(out_row(sW2, sb2, r, z)), sigm(out_row(sW2, sb2, r + 1, z)),
                                               sigm(out_row(sW2, sb2, r + 2, z)), 0.f);
        }
        if (NF > 0) {
            hidden_T(sW1T, sb1, 3, af, xt, z);
            activate<1>(z);
#pragma unroll 1
            for (int k = 0; k < K; ++k) {
                float4 *dst = reinterpret_cast<float4 *>(feat_out + (gbase + k) * NF);
                const int r = 11 * K + NF * k;
#pragma unroll
                for (int c = 0; c < NF / 4; ++c)
                    dst[c] = make_float4(out_row(sW2, sb2, r + 4 * c, z), out_row(sW2, sb2, r + 4 * c + 1, z),
                                         out_row(sW2, sb2, r + 4 * c + 2, z), out_row(sW2, sb2, r + 4 * c + 3, z));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// backward, per row (FP32)
// ---------------------------------------------------------------------------

// One MLP group of one row: Z = W1_g x + b1 (recomputed), H = act(Z); for each
// output o of the group the pre-activation Y_o (only where the output
// activation has a derivative: opacity, scale, colour), DY_o = dL/dY_o, and
// DH += DY_o W2[o]; DZ = DH * act'(Z); dx += DZ W1_g.  H, DY, DZ go to the
// feature-major scratch for the weight-gradient kernel.
template <int G, int NF>
__device__ __forceinline__ void bwd_group(const dbwd::Args &a, const DecodeArgs &da, const float *sW1T,
                                          const float *sb1, const float *sW2, const float *sb2,
                                          const float xt[6], int an, bool valid, size_t gbase, int lr,
                                          float *sDX, float dls[3]) {
    constexpr int M = G == 0 ? 1 : G == 1 ? 7 : G == 2 ? 3 : NF;
    const int K = a.K;
    const bool want_mlp = a.s.X != nullptr && valid;
    const int ld = a.s.ld;
    f2 h[kH2];
    hidden_T(sW1T, sb1, G, a.afeat + (size_t)an * kFin, xt, h);
    unsigned relu_on = 0;  // ReLU derivative as a bit mask
#pragma unroll
    for (int p = 0; p < kH2; ++p) {
        float lo, hi;
        f2_split(h[p], lo, hi);
        if (G < 3) {
            relu_on |= (lo > 0.f ? 1u : 0u) << (2 * p);
            relu_on |= (hi > 0.f ? 1u : 0u) << (2 * p + 1);
            h[p] = f2_make(fmaxf(lo, 0.f), fmaxf(hi, 0.f));
        } else {
            h[p] = f2_make(softplus(lo), softplus(hi));
        }
    }
    if (want_mlp)
#pragma unroll
        for (int p = 0; p < kH2; ++p) {
            float lo, hi;
            f2_split(h[p], lo, hi);
            a.s.H[(size_t)(G * kH + 2 * p) * ld + lr] = lo;
            a.s.H[(size_t)(G * kH + 2 * p + 1) * ld + lr] = hi;
        }
    f2 dh[kH2];
#pragma unroll
    for (int p = 0; p < kH2; ++p) dh[p] = 0ull;
    const int r0 = dbwd::grp_r0(G, K);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    // dL/dG of Gaussian k for this group, loaded one Gaussian ahead so the
    // loads of k + 1 are in flight while k is processed
    constexpr int NQ = G == 3 ? (NF / 4 > 0 ? NF / 4 : 1) : 2;
    constexpr bool kAhead = UPS_DECB_AHEAD && NQ <= 4;
    auto load = [&](int k, float4 (&q)[NQ]) {
        const size_t gi = gbase + k;
#pragma unroll
        for (int i = 0; i < NQ; ++i) q[i] = z4;
        if (!valid || k >= K) return;
        if (G == 0) q[0] = a.d_mean_op[gi];
        if (G == 1) {
            q[0] = a.d_scale[gi];
            q[1] = a.d_quat[gi];
        }
        if (G == 2) q[0] = a.d_color[gi];
        if (G == 3)
#pragma unroll
            for (int i = 0; i < NF / 4; ++i) q[i] = reinterpret_cast<const float4 *>(a.d_feat + gi * NF)[i];
    };
    float4 nxt[NQ];
    if (kAhead) load(0, nxt);
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        float4 cur[NQ];
        if (kAhead) {
#pragma unroll
            for (int i = 0; i < NQ; ++i) cur[i] = nxt[i];
            load(k + 1, nxt);
        } else {
            load(k, cur);
        }
        const float4 g4a = cur[0], g4b = cur[NQ > 1 ? 1 : 0];
#pragma unroll
        for (int c = 0; c < M; ++c) {
            const int o = r0 + M * k + c;
            const bool nl = G == 0 || G == 2 || (G == 1 && c < 3);
            float gin;
            if (G == 0) {
                gin = g4a.w;
            } else if (G == 1) {
                gin = c == 0 ? g4a.x : c == 1 ? g4a.y : c == 2 ? g4a.z : c == 3 ? g4b.x : c == 4 ? g4b.y
                                                                          : c == 5 ? g4b.z : g4b.w;
            } else if (G == 2) {
                gin = c == 0 ? g4a.x : c == 1 ? g4a.y : g4a.z;
            } else {
                const float4 f4 = cur[(c >> 2) < NQ ? (c >> 2) : 0];
                gin = (c & 3) == 0 ? f4.x : (c & 3) == 1 ? f4.y : (c & 3) == 2 ? f4.z : f4.w;
            }
            float dy = gin;
            if (G == 0 && da.op_tanh) {
                const float t = tanhf(out_row(sW2, sb2, o, h));
                dy = gin * (1.f - t * t);
            } else if (nl) {
                const float s = sigm(out_row(sW2, sb2, o, h));
                if (G == 1) {
                    dy = gin * a.ascale[3 * an + c] * s * (1.f - s);
                    dls[c] += gin * s;
                } else {
                    dy = gin * s * (1.f - s);
                }
            }
            if (want_mlp) a.s.DY[(size_t)o * ld + lr] = dy;
            const ulonglong2 *w = reinterpret_cast<const ulonglong2 *>(sW2 + o * kH);
            const f2 dy2 = f2_make(dy, dy);
#pragma unroll
            for (int q = 0; q < kH / 4; ++q) {
                const ulonglong2 ww = w[q];
                dh[2 * q] = f2_fma(dy2, ww.x, dh[2 * q]);
                dh[2 * q + 1] = f2_fma(dy2, ww.y, dh[2 * q + 1]);
            }
        }
    }
    // DZ = DH * act'(Z): ReLU -> mask; SoftPlus -> sigmoid(Z) = 1 - exp(-H)
#pragma unroll
    for (int p = 0; p < kH2; ++p) {
        float d0, d1, h0, h1;
        f2_split(dh[p], d0, d1);
        f2_split(h[p], h0, h1);
        d0 *= G < 3 ? (float)((relu_on >> (2 * p)) & 1u) : -expm1f(-h0);
        d1 *= G < 3 ? (float)((relu_on >> (2 * p + 1)) & 1u) : -expm1f(-h1);
        dh[p] = f2_make(d0, d1);
        if (want_mlp) {
            a.s.DZ[(size_t)(G * kH + 2 * p) * ld + lr] = d0;
            a.s.DZ[(size_t)(G * kH + 2 * p + 1) * ld + lr] = d1;
        }
    }
    // dx += DZ W1_g for the inputs that have a gradient (f_v, delta_vc, d_vc),
    // accumulated in shared memory (column tid of sDX); partial sums as in
    // out_row
#pragma unroll 1
    for (int i = 0; i < kDX; ++i) {
        const ulonglong2 *w = reinterpret_cast<const ulonglong2 *>(sW1T + i * 128 + G * kH);
        f2 a01 = 0ull, a23 = 0ull;
#pragma unroll
        for (int q = 0; q < kH / 4; ++q) {
            const ulonglong2 ww = w[q];
            a01 = f2_fma(dh[2 * q], ww.x, a01);
            a23 = f2_fma(dh[2 * q + 1], ww.y, a23);
        }
        float s0, s1, s2, s3;
        f2_split(a01, s0, s1);
        f2_split(a23, s2, s3);
        sDX[i * dbwd::kRowsFp32] += (s0 + s1) + (s2 + s3);
    }
}

// One thread per row (anchor-major), 128 rows per step of a grid-stride loop;
// weights in shared memory read as broadcasts.
template <int NF>
__global__ void __launch_bounds__(dbwd::kRowsFp32, dbwd::kRowsCtasPerSm) k_decode_bwd_rows(ViewTable vt,
                                                                                               dbwd::Args a) {
    extern __shared__ float4 smem4[];
    __shared__ float aPose[3 * UPS_MAX_VIEWS];
    float *sm = reinterpret_cast<float *>(smem4);
    const int n_out = dbwd::n_out(a.K, NF);
    const DecodeArgs da{a.A, a.K, NF, n_out, a.pos, a.afeat, a.offs, a.ascale, a.w1, a.b1, a.w2, a.b2, a.op_tanh};
    // W1 transposed [38][128] (inputs x hidden), b1, W2 [n_out][32], b2, and
    // the per-row input gradients dx [36][128 rows]
    float *sW1T = sm, *sb1 = sW1T + kDin * 4 * kH, *sW2 = sb1 + 4 * kH, *sb2 = sW2 + n_out * kH;
    float *sDXall = sb2 + ((n_out + 3) & ~3);
    load_weights_T(da, sW1T, sb1, sW2, sb2);
    const int V = vt.n;
    for (int i = threadIdx.x; i < 3 * V; i += blockDim.x) aPose[i] = 0.f;
    __syncthreads();
    const size_t NG = (size_t)a.A * a.K;
    float *sDX = sDXall + threadIdx.x;
    for (int base = a.row_begin + blockIdx.x * dbwd::kRowsFp32; base < a.row_end;
         base += gridDim.x * dbwd::kRowsFp32) {
        const int row = base + threadIdx.x;
        const bool valid = row < a.row_end;
        const int an = valid ? row / V : 0, v = valid ? row - an * V : 0;
        const int lr = row - a.row_begin;
        const DevView &cam = vt.v[v];
        const size_t gbase = (size_t)v * NG + (size_t)an * a.K;
        float x[kDinP], delta[3], dist;
        mlp_input(da, cam, an, x, delta, dist);
        if (a.s.X && valid) {
            x[38] = 1.f;
#pragma unroll
            for (int i = 0; i < kDinP; ++i) a.s.X[(size_t)i * a.s.ld + lr] = x[i];
        }
        const float xt[6] = {x[kFin], x[kFin + 1], x[kFin + 2], x[kFin + 3], x[kFin + 4], x[kFin + 5]};
#pragma unroll
        for (int i = 0; i < kDX; ++i) sDX[i * dbwd::kRowsFp32] = 0.f;
        float dls[3] = {0.f, 0.f, 0.f};
        bwd_group<0, NF>(a, da, sW1T, sb1, sW2, sb2, xt, an, valid, gbase, lr, sDX, dls);
        bwd_group<1, NF>(a, da, sW1T, sb1, sW2, sb2, xt, an, valid, gbase, lr, sDX, dls);
        bwd_group<2, NF>(a, da, sW1T, sb1, sW2, sb2, xt, an, valid, gbase, lr, sDX, dls);
        if (NF > 0) bwd_group<3, NF>(a, da, sW1T, sb1, sW2, sb2, xt, an, valid, gbase, lr, sDX, dls);
        float dx[kDX];
#pragma unroll
        for (int i = 0; i < kDX; ++i) dx[i] = sDX[i * dbwd::kRowsFp32];
        dbwd::row_epilogue(a, valid ? an : -1, v, gbase, dx, delta, dist, dls, aPose);
    }
    __syncthreads();
    dbwd::flush_pose(a, vt, aPose);
}

// shared memory of the backward rows kernel
size_t bwd_rows_smem(int n_out) {
    return sizeof(float) * (kDin * 4 * kH + 4 * kH + n_out * kH + ((n_out + 3) & ~3) + kDX * dbwd::kRowsFp32);
}

size_t fwd_smem(int n_out) { return sizeof(float) * (kDin * 4 * kH + 4 * kH + n_out * kH + n_out); }

}  // namespace

size_t decode_bwd_rows_fp32_smem(int K, int NF) { return bwd_rows_smem(dbwd::n_out(K, NF)); }

cudaError_t launch_decode_bwd_rows_fp32(const ViewTable &vt, const dbwd::Args &a, int num_sms, cudaStream_t st) {
    const size_t smem = bwd_rows_smem(dbwd::n_out(a.K, a.NF));
    if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
    const int rows = a.row_end - a.row_begin;
    const int blocks = std::max(
        1, std::min((rows + dbwd::kRowsFp32 - 1) / dbwd::kRowsFp32, num_sms * dbwd::kRowsCtasPerSm));
#define UPS_DECB(NFV)                                                                              \
    do {                                                                                           \
        cudaFuncSetAttribute(k_decode_bwd_rows<NFV>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                             (int)smem);                                                           \
        k_decode_bwd_rows<NFV><<<blocks, dbwd::kRowsFp32, smem, st>>>(vt, a);                  \
    } while (0)
    switch (a.NF) {
        case 0: UPS_DECB(0); break;
        case 16: UPS_DECB(16); break;
        case 32: UPS_DECB(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef UPS_DECB
    return cudaGetLastError();
}

cudaError_t launch_decode_fwd(const ViewTable &vt, int A, int K, int NF, const ups_anchors &anc,
                              const ups_mlp &mlp, const ups_gaussians &out, int op_tanh, int num_sms,
                              cudaStream_t st) {
    DecodeArgs a{A, K, NF, K * (11 + NF), anc.pos, anc.feat, anc.offsets, anc.scaling,
                 mlp.w1, mlp.b1, mlp.w2, mlp.b2, op_tanh};
    size_t smem = fwd_smem(a.n_out);
    if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
    int rows = A * vt.n;
    int blocks = std::max(1, std::min((rows + kFwdThreads - 1) / kFwdThreads, num_sms * kFwdCtas));
#define UPS_DEC(NFV)                                                                        \
    do {                                                                                    \
        cudaFuncSetAttribute(k_decode_fwd<NFV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                    \
        k_decode_fwd<NFV><<<blocks, kFwdThreads, smem, st>>>(                               \
            vt, a, reinterpret_cast<float4 *>(out.mean_opacity),                            \
            reinterpret_cast<float4 *>(out.scale), reinterpret_cast<float4 *>(out.quat),    \
            reinterpret_cast<float4 *>(out.color), out.feat);                               \
    } while (0)
    switch (NF) {
        case 0: UPS_DEC(0); break;
        case 16: UPS_DEC(16); break;
        case 32: UPS_DEC(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef UPS_DEC
    return cudaGetLastError();
}

}  // namespace ups
