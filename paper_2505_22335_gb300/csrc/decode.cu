// Per-anchor MLP decode of K neural Gaussians (Eq. 8-9) and its backward,
// FP32 on the CUDA cores.
//
// Row = (anchor, view).  MLP input x = [f_v, delta_vc, d_vc, sin(pi t),
// cos(pi t)]; four MLPs (opacity, covariance, colour: ReLU hidden; feature
// F_d: SoftPlus hidden) of width `hidden` = 32.  Weights live in shared memory
// and are read as float4 broadcasts (every lane of a warp reads the same
// weight), so the inner loops are FMA-bound.
//
// Backward: tiles of rows are processed as small GEMMs in shared memory (see
// k_decode_bwd); weight gradients accumulate per block and are flushed once.
#include <algorithm>

#include "common.cuh"

namespace ups {

namespace {

constexpr int kH = 32;       // hidden width per MLP
constexpr int kFin = 32;     // anchor feature width
constexpr int kDin = kFin + 6;
constexpr int kDinP = 40;    // padded input width (float4 rows)
constexpr int kMaxK = 16;
constexpr size_t kMaxSmem = 227 * 1024;  // opt-in shared memory per block

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + __expf(-x)); }
__device__ __forceinline__ float softplus(float x) { return x > 20.f ? x : log1pf(__expf(x)); }

struct DecodeArgs {
    int A, K, NF, n_out;
    const float *pos, *afeat, *offs, *ascale;
    const float *w1, *b1, *w2, *b2;
};

// shared layout: W1 [128][40] (padded), b1 [128], W2 [n_out][32], b2 [n_out]
__device__ __forceinline__ void load_weights(const DecodeArgs &a, float *sW1, float *sb1, float *sW2,
                                             float *sb2) {
    for (int i = threadIdx.x; i < 4 * kH * kDinP; i += blockDim.x) {
        int r = i / kDinP, c = i - r * kDinP;
        sW1[i] = c < kDin ? a.w1[r * kDin + c] : 0.f;
    }
    for (int i = threadIdx.x; i < 4 * kH; i += blockDim.x) sb1[i] = a.b1[i];
    for (int i = threadIdx.x; i < a.n_out * kH; i += blockDim.x) sW2[i] = a.w2[i];
    for (int i = threadIdx.x; i < a.n_out; i += blockDim.x) sb2[i] = a.b2[i];
}

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

// hidden block g: z = W1_g x + b1_g (32 values)
__device__ __forceinline__ void hidden_pre(const float *sW1, const float *sb1, int g,
                                           const float x[kDinP], float z[kH]) {
#pragma unroll 4
    for (int j = 0; j < kH; ++j) {
        const float4 *w = reinterpret_cast<const float4 *>(sW1 + (g * kH + j) * kDinP);
        float acc = sb1[g * kH + j];
#pragma unroll
        for (int q = 0; q < kDinP / 4; ++q) {
            float4 ww = w[q];
            acc = fmaf(ww.x, x[4 * q], acc);
            acc = fmaf(ww.y, x[4 * q + 1], acc);
            acc = fmaf(ww.z, x[4 * q + 2], acc);
            acc = fmaf(ww.w, x[4 * q + 3], acc);
        }
        z[j] = acc;
    }
}

__device__ __forceinline__ float out_row(const float *sW2, const float *sb2, int r, const float h[kH]) {
    const float4 *w = reinterpret_cast<const float4 *>(sW2 + r * kH);
    float acc = sb2[r];
#pragma unroll
    for (int q = 0; q < kH / 4; ++q) {
        float4 ww = w[q];
        acc = fmaf(ww.x, h[4 * q], acc);
        acc = fmaf(ww.y, h[4 * q + 1], acc);
        acc = fmaf(ww.z, h[4 * q + 2], acc);
        acc = fmaf(ww.w, h[4 * q + 3], acc);
    }
    return acc;
}

template <int NF>
__global__ void __launch_bounds__(128) k_decode_fwd(ViewTable vt, DecodeArgs a,
                                                    float4 *__restrict__ mean_op,
                                                    float4 *__restrict__ scale_out,
                                                    float4 *__restrict__ quat_out,
                                                    float4 *__restrict__ color_out,
                                                    float *__restrict__ feat_out) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    float *sW1 = sm, *sb1 = sW1 + 4 * kH * kDinP, *sW2 = sb1 + 4 * kH, *sb2 = sW2 + a.n_out * kH;
    load_weights(a, sW1, sb1, sW2, sb2);
    __syncthreads();
    const int K = a.K;
    const int rows = a.A * vt.n;
    const size_t NG = (size_t)a.A * K;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += gridDim.x * blockDim.x) {
        const int v = row / a.A, an = row - v * a.A;
        const DevView &cam = vt.v[v];
        float x[kDinP], delta[3], dist;
        mlp_input(a, cam, an, x, delta, dist);
        float z[kH];
        float op[kMaxK];
        // opacity
        hidden_pre(sW1, sb1, 0, x, z);
#pragma unroll
        for (int j = 0; j < kH; ++j) z[j] = fmaxf(z[j], 0.f);
#pragma unroll 1
        for (int k = 0; k < K; ++k) op[k] = sigm(out_row(sW2, sb2, k, z));
        const float px = a.pos[3 * an], py = a.pos[3 * an + 1], pz = a.pos[3 * an + 2];
        const size_t gbase = (size_t)v * NG + (size_t)an * K;
        // covariance: 3 scale + 4 quaternion per Gaussian, and the mean
        hidden_pre(sW1, sb1, 1, x, z);
#pragma unroll
        for (int j = 0; j < kH; ++j) z[j] = fmaxf(z[j], 0.f);
        const float lx = a.ascale[3 * an], ly = a.ascale[3 * an + 1], lz = a.ascale[3 * an + 2];
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            {
                int r = K + 7 * k;
                float s0 = lx * sigm(out_row(sW2, sb2, r, z));
                float s1 = ly * sigm(out_row(sW2, sb2, r + 1, z));
                float s2 = lz * sigm(out_row(sW2, sb2, r + 2, z));
                float q0 = out_row(sW2, sb2, r + 3, z), q1 = out_row(sW2, sb2, r + 4, z);
                float q2 = out_row(sW2, sb2, r + 5, z), q3 = out_row(sW2, sb2, r + 6, z);
                const float *o3 = a.offs + ((size_t)an * K + k) * 3;
                mean_op[gbase + k] = make_float4(px + o3[0], py + o3[1], pz + o3[2], op[k]);
                scale_out[gbase + k] = make_float4(s0, s1, s2, 0.f);
                quat_out[gbase + k] = make_float4(q0, q1, q2, q3);
            }
        }
        // colour
        hidden_pre(sW1, sb1, 2, x, z);
#pragma unroll
        for (int j = 0; j < kH; ++j) z[j] = fmaxf(z[j], 0.f);
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            {
                int r = 8 * K + 3 * k;
                color_out[gbase + k] = make_float4(sigm(out_row(sW2, sb2, r, z)),
                                                   sigm(out_row(sW2, sb2, r + 1, z)),
                                                   sigm(out_row(sW2, sb2, r + 2, z)), 0.f);
            }
        }
        if (NF > 0) {
            hidden_pre(sW1, sb1, 3, x, z);
#pragma unroll
            for (int j = 0; j < kH; ++j) z[j] = softplus(z[j]);
            for (int k = 0; k < K; ++k) {
                float4 *dst = reinterpret_cast<float4 *>(feat_out + (gbase + k) * NF);
                int r = 11 * K + NF * k;
#pragma unroll
                for (int c = 0; c < NF / 4; ++c)
                    dst[c] = make_float4(out_row(sW2, sb2, r + 4 * c, z), out_row(sW2, sb2, r + 4 * c + 1, z),
                                         out_row(sW2, sb2, r + 4 * c + 2, z), out_row(sW2, sb2, r + 4 * c + 3, z));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

struct DecodeGrads {
    const float4 *d_mean_op, *d_scale, *d_quat, *d_color;
    const float *d_feat;
    float *g_w1, *g_b1, *g_w2, *g_b2;            // MLP (accumulated)
    float *g_pos, *g_afeat, *g_offs, *g_ascale;  // anchors (accumulated)
    float *g_pose;                               // [V][6] (accumulated)
    unsigned mask;
};

// Tiled backward: R rows (anchor-major: row = anchor * V + view) per tile,
// 8 threads per row.  Per MLP group g, all in shared memory:
//   Z = X W1_g^T + b1 (H = act(Z), AP = act'(Z));  Y = H W2_g^T + b2 and
//   DY = dL/dY through the output activation;  DZ = (DY W2_g) * AP;
//   DX += DZ W1_g;  dW2_g += DY^T H, db2 += 1^T DY;  dW1_g += DZ^T X, db1 += 1^T DZ.
// The weight-gradient products use 4x4 register micro-tiles over the R rows and
// accumulate in per-block shared memory, flushed once per block.
constexpr int kW1S = 132;  // W1^T row stride (conflict-free column walks)
constexpr int kXS = 44;    // X / DX row stride (col 38 of X is 1: the db1 column)
constexpr int kHS = 36;    // H / AP / DZ row stride
constexpr int kW2S = 36;   // W2 row stride (col 32 of the accumulator: db2)
constexpr int kAccW1S = 44;

__host__ __device__ constexpr int pad4(int x) { return (x + 3) & ~3; }

template <int NF> struct BwdTile {
    static constexpr int R = NF == 32 ? 16 : 32;  // rows per tile
    static constexpr int TPR = 16;                // threads per row
    static constexpr int T = TPR * R;             // threads
};

struct BwdLayout {
    int n_out, DYS, acc_rows;
    int oW1T, ob1, oW2, ob2, oX, oH, oAP, oDZ, oDY, oDX, oDLS, oDR, oAccW1, oAccW2, oPose, oInfo;
    int oSG, SGS, oSM, total;
};

__host__ __device__ inline BwdLayout bwd_layout(int K, int NF, int R, int V) {
    BwdLayout L;
    L.n_out = K * (11 + NF);
    int maxg = max(max(K, 7 * K), max(3 * K, K * NF));
    L.DYS = pad4(maxg) + 4;
    L.acc_rows = pad4(K) + pad4(7 * K) + pad4(3 * K) + pad4(K * NF);
    int o = 0;
    auto take = [&](int n) { int r = o; o += pad4(n); return r; };
    L.oW1T = take(40 * kW1S);
    L.ob1 = take(128);
    L.oW2 = take(L.n_out * kW2S);
    L.ob2 = take(L.n_out);
    L.oX = take(R * kXS);
    L.oH = take(R * kHS);
    L.oAP = take(R * kHS);
    L.oDZ = take(R * kHS);
    L.oDY = take(R * L.DYS);
    L.oDX = take(R * kXS);
    L.oDLS = take(R * 4);
    L.oDR = take(R * 4);
    L.oAccW1 = take(128 * kAccW1S);
    L.oAccW2 = take(L.acc_rows * kW2S);
    L.oPose = take(3 * V);
    L.oInfo = take(R * 8);  // per row: anchor, view, valid, dist, delta[3]
    L.SGS = pad4(K * max(7, NF));  // staged dL/dG of one group, per row
    L.oSG = take(R * L.SGS);
    L.oSM = take(R * K * 4);       // staged dL/d(mean, opacity), per row and Gaussian
    L.total = o;
    return L;
}

template <int NF>
__global__ void __launch_bounds__(BwdTile<NF>::T) k_decode_bwd(ViewTable vt, DecodeArgs a, DecodeGrads gr) {
    constexpr int R = BwdTile<NF>::R, NT = BwdTile<NF>::T;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int K = a.K, V = vt.n;
    const BwdLayout L = bwd_layout(K, NF, R, V);
    float *W1T = sm + L.oW1T, *sb1 = sm + L.ob1, *W2s = sm + L.oW2, *sb2 = sm + L.ob2;
    float *X = sm + L.oX, *H = sm + L.oH, *AP = sm + L.oAP, *DZ = sm + L.oDZ, *DY = sm + L.oDY;
    float *DX = sm + L.oDX, *DLS = sm + L.oDLS, *DR = sm + L.oDR;
    float *AccW1 = sm + L.oAccW1, *AccW2 = sm + L.oAccW2, *aPose = sm + L.oPose;
    float *Info = sm + L.oInfo;
    float *SG = sm + L.oSG, *SM = sm + L.oSM;
    constexpr int TPR = BwdTile<NF>::TPR;
    const int tid = threadIdx.x;
    const bool want_mlp = gr.mask & UPS_GRAD_MLP;
    const bool want_anc = gr.mask & UPS_GRAD_ANCHOR;
    const bool want_pose = gr.mask & UPS_GRAD_POSE;
    // weights (W1 transposed) and zeroed accumulators
    for (int i = tid; i < 40 * kW1S; i += NT) {
        int ii = i / kW1S, h = i - ii * kW1S;
        W1T[i] = (ii < kDin && h < 128) ? a.w1[h * kDin + ii] : 0.f;
    }
    for (int i = tid; i < 128; i += NT) sb1[i] = a.b1[i];
    for (int i = tid; i < L.n_out * kW2S; i += NT) {
        int o = i / kW2S, j = i - o * kW2S;
        W2s[i] = j < kH ? a.w2[o * kH + j] : 0.f;
    }
    for (int i = tid; i < L.n_out; i += NT) sb2[i] = a.b2[i];
    for (int i = tid; i < 128 * kAccW1S; i += NT) AccW1[i] = 0.f;
    for (int i = tid; i < L.acc_rows * kW2S; i += NT) AccW2[i] = 0.f;
    for (int i = tid; i < 3 * V; i += NT) aPose[i] = 0.f;
    __syncthreads();
    const int rows = a.A * V;
    const int ntiles = (rows + R - 1) / R;
    const size_t NG = (size_t)a.A * K;
    const int r = tid / TPR, q = tid % TPR;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row0 = tile * R;
        // ---- inputs of each row
        if (tid < R) {
            const int row = row0 + tid;
            const bool valid = row < rows;
            const int an = valid ? row / V : 0, v = valid ? row - an * V : 0;
            float x[kDinP], delta[3], dist;
            mlp_input(a, vt.v[v], an, x, delta, dist);
            float *xr = X + tid * kXS;
#pragma unroll
            for (int i = 0; i < kDin; ++i) xr[i] = valid ? x[i] : 0.f;
            xr[38] = valid ? 1.f : 0.f;
#pragma unroll
            for (int i = 39; i < kXS; ++i) xr[i] = 0.f;
#pragma unroll
            for (int i = 0; i < kXS; ++i) DX[tid * kXS + i] = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) DLS[tid * 4 + i] = 0.f;
            float *inf = Info + tid * 8;
            inf[0] = __int_as_float(an);
            inf[1] = __int_as_float(v);
            inf[2] = valid ? 1.f : 0.f;
            inf[3] = dist;
            inf[4] = delta[0];
            inf[5] = delta[1];
            inf[6] = delta[2];
        }
        __syncthreads();
        const int an_r = __float_as_int(Info[r * 8]);
        const bool valid_r = Info[r * 8 + 2] != 0.f;
        int gacc = 0;
        for (int g = 0; g < 4; ++g) {
            const int m = g == 0 ? 1 : g == 1 ? 7 : g == 2 ? 3 : NF;
            if (m == 0) break;
            const int ng = K * m, npad = pad4(ng);
            const int r0 = g == 0 ? 0 : g == 1 ? K : g == 2 ? 8 * K : 11 * K;
            // ---- stage this group's dL/dG of the tile's rows (coalesced, all threads)
            if (g == 3) {
                const int per_row = K * NF / 4;
                for (int it = tid; it < R * per_row; it += NT) {
                    const int rr = it / per_row, e = it - rr * per_row;
                    float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (Info[rr * 8 + 2] != 0.f) {
                        const size_t gb = (size_t)__float_as_int(Info[rr * 8 + 1]) * NG +
                                          (size_t)__float_as_int(Info[rr * 8]) * K;
                        val = reinterpret_cast<const float4 *>(gr.d_feat + gb * NF)[e];
                    }
                    *reinterpret_cast<float4 *>(SG + rr * L.SGS + 4 * e) = val;
                }
            } else {
                for (int it = tid; it < R * K; it += NT) {
                    const int rr = it / K, k = it - rr * K;
                    const bool ok = Info[rr * 8 + 2] != 0.f;
                    const size_t gi = ok ? (size_t)__float_as_int(Info[rr * 8 + 1]) * NG +
                                               (size_t)__float_as_int(Info[rr * 8]) * K + k
                                         : 0;
                    float *dst = SG + rr * L.SGS;
                    if (g == 0) {
                        const float4 dm = ok ? gr.d_mean_op[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
                        *reinterpret_cast<float4 *>(SM + (rr * K + k) * 4) = dm;
                        dst[k] = dm.w;
                    } else if (g == 1) {
                        const float4 ds = ok ? gr.d_scale[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float4 dq = ok ? gr.d_quat[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
                        dst[7 * k] = ds.x;
                        dst[7 * k + 1] = ds.y;
                        dst[7 * k + 2] = ds.z;
                        dst[7 * k + 3] = dq.x;
                        dst[7 * k + 4] = dq.y;
                        dst[7 * k + 5] = dq.z;
                        dst[7 * k + 6] = dq.w;
                    } else {
                        const float4 dc = ok ? gr.d_color[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
                        dst[3 * k] = dc.x;
                        dst[3 * k + 1] = dc.y;
                        dst[3 * k + 2] = dc.z;
                    }
                }
            }
            // ---- Z, H, act'  (two hidden units per thread)
            {
                float z[2];
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) z[jj] = sb1[g * kH + 2 * q + jj];
                const float *xr = X + r * kXS;
#pragma unroll 8
                for (int i = 0; i < 40; ++i) {
                    const float xi = xr[i];
                    const float2 w = *reinterpret_cast<const float2 *>(W1T + i * kW1S + g * kH + 2 * q);
                    z[0] = fmaf(xi, w.x, z[0]);
                    z[1] = fmaf(xi, w.y, z[1]);
                }
                float hv[2], ap[2];
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    if (g < 3) {
                        hv[jj] = fmaxf(z[jj], 0.f);
                        ap[jj] = z[jj] > 0.f ? 1.f : 0.f;
                    } else {
                        hv[jj] = softplus(z[jj]);
                        ap[jj] = sigm(z[jj]);
                    }
                }
                *reinterpret_cast<float2 *>(H + r * kHS + 2 * q) = make_float2(hv[0], hv[1]);
                *reinterpret_cast<float2 *>(AP + r * kHS + 2 * q) = make_float2(ap[0], ap[1]);
            }
            __syncthreads();
            // ---- Y and dL/dY
            {
                float h[kH];
#pragma unroll
                for (int qq = 0; qq < kH / 4; ++qq) {
                    float4 t4 = *reinterpret_cast<const float4 *>(H + r * kHS + 4 * qq);
                    h[4 * qq] = t4.x;
                    h[4 * qq + 1] = t4.y;
                    h[4 * qq + 2] = t4.z;
                    h[4 * qq + 3] = t4.w;
                }
                for (int o = q; o < npad; o += TPR) {
                    float dy = 0.f;
                    if (o < ng && valid_r) {
                        const int row_o = r0 + o;
                        const int k = o / m, c = o - k * m;
                        // the pre-activation is needed only where an output
                        // activation has a derivative (not for the linear
                        // quaternion and feature outputs)
                        const bool need_y = g == 0 || g == 2 || (g == 1 && c < 3);
                        float y = 0.f;
                        if (need_y) {
                            const float4 *w = reinterpret_cast<const float4 *>(W2s + row_o * kW2S);
                            y = sb2[row_o];
#pragma unroll
                            for (int qq = 0; qq < kH / 4; ++qq) {
                                float4 ww = w[qq];
                                y = fmaf(ww.x, h[4 * qq], y);
                                y = fmaf(ww.y, h[4 * qq + 1], y);
                                y = fmaf(ww.z, h[4 * qq + 2], y);
                                y = fmaf(ww.w, h[4 * qq + 3], y);
                            }
                        }
                        const float gin = SG[r * L.SGS + o];
                        if (g == 0) {
                            float s = sigm(y);
                            dy = gin * s * (1.f - s);
                        } else if (g == 1) {
                            if (c < 3) {
                                float s = sigm(y);
                                float l = a.ascale[3 * an_r + c];
                                dy = gin * l * s * (1.f - s);
                                atomicAdd(DLS + r * 4 + c, gin * s);
                            } else {
                                dy = gin;
                            }
                        } else if (g == 2) {
                            float cc = sigm(y);
                            dy = gin * cc * (1.f - cc);
                        } else {
                            dy = gin;
                        }
                    }
                    DY[r * L.DYS + o] = dy;
                }
            }
            __syncthreads();
            // ---- DZ = (DY W2_g) * act'(Z)
            {
                float dh[2] = {0.f, 0.f};
                const float *dyr = DY + r * L.DYS;
#pragma unroll 4
                for (int o = 0; o < ng; ++o) {
                    const float d = dyr[o];
                    const float2 w = *reinterpret_cast<const float2 *>(W2s + (r0 + o) * kW2S + 2 * q);
                    dh[0] = fmaf(d, w.x, dh[0]);
                    dh[1] = fmaf(d, w.y, dh[1]);
                }
                const float2 ap = *reinterpret_cast<const float2 *>(AP + r * kHS + 2 * q);
                *reinterpret_cast<float2 *>(DZ + r * kHS + 2 * q) = make_float2(dh[0] * ap.x, dh[1] * ap.y);
            }
            __syncthreads();
            // ---- DX += DZ W1_g  (thread owns inputs q, q+16, q+32)
            {
                const float *dzr = DZ + r * kHS;
#pragma unroll
                for (int mm = 0; mm < 3; ++mm) {
                    const int i = q + TPR * mm;
                    if (i >= 40) break;
                    float acc = 0.f;
#pragma unroll 8
                    for (int j = 0; j < kH; ++j) acc = fmaf(dzr[j], W1T[i * kW1S + g * kH + j], acc);
                    DX[r * kXS + i] += acc;
                }
            }
            // ---- weight gradients (micro-tiles over the R rows)
            if (want_mlp) {
                const int nA = (npad / 4) * 8;  // dW2_g: (o-block, j-block)
                const int nB = 8 * 10;          // dW1_g: (j-block, i-block), i < 40 incl. the db1 column
                for (int mt = tid; mt < nA + nB; mt += NT) {
                    float acc[4][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int w = 0; w < 4; ++w) acc[u][w] = 0.f;
                    if (mt < nA) {
                        const int ob = mt >> 3, jb = mt & 7;
                        float sb[4] = {0.f, 0.f, 0.f, 0.f};
                        for (int rr = 0; rr < R; ++rr) {
                            const float4 av = *reinterpret_cast<const float4 *>(DY + rr * L.DYS + 4 * ob);
                            const float4 bv = *reinterpret_cast<const float4 *>(H + rr * kHS + 4 * jb);
                            const float aa[4] = {av.x, av.y, av.z, av.w}, bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                sb[u] += aa[u];
#pragma unroll
                                for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(aa[u], bb[w], acc[u][w]);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            float *dst = AccW2 + (gacc + 4 * ob + u) * kW2S;
#pragma unroll
                            for (int w = 0; w < 4; ++w) dst[4 * jb + w] += acc[u][w];
                            if (jb == 0) dst[32] += sb[u];
                        }
                    } else {
                        const int t2 = mt - nA, jb = t2 / 10, ib = t2 - jb * 10;
                        for (int rr = 0; rr < R; ++rr) {
                            const float4 av = *reinterpret_cast<const float4 *>(DZ + rr * kHS + 4 * jb);
                            const float4 bv = *reinterpret_cast<const float4 *>(X + rr * kXS + 4 * ib);
                            const float aa[4] = {av.x, av.y, av.z, av.w}, bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                            for (int u = 0; u < 4; ++u)
#pragma unroll
                                for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(aa[u], bb[w], acc[u][w]);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            float *dst = AccW1 + (g * kH + 4 * jb + u) * kAccW1S + 4 * ib;
#pragma unroll
                            for (int w = 0; w < 4; ++w) dst[w] += acc[u][w];
                        }
                    }
                }
            }
            gacc += npad;
            __syncthreads();
        }
        // ---- per row: delta_vc, d_vc -> r = x_v - o_c
        if (tid < R && Info[tid * 8 + 2] != 0.f) {
            const float *dx = DX + tid * kXS;
            const float dist = Info[tid * 8 + 3];
            const float de[3] = {Info[tid * 8 + 4], Info[tid * 8 + 5], Info[tid * 8 + 6]};
            const float ddl[3] = {dx[kFin], dx[kFin + 1], dx[kFin + 2]}, dd = dx[kFin + 3];
            const float dot = de[0] * ddl[0] + de[1] * ddl[1] + de[2] * ddl[2];
            const float idist = 1.f / dist;
            const int v = __float_as_int(Info[tid * 8 + 1]);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const float drr = (ddl[i] - de[i] * dot) * idist + dd * de[i];
                DR[tid * 4 + i] = drr;
                if (want_pose) atomicAdd(aPose + 3 * v + i, -drr);
            }
        } else if (tid < R) {
            DR[tid * 4] = DR[tid * 4 + 1] = DR[tid * 4 + 2] = 0.f;
        }
        __syncthreads();
        // ---- anchor gradients: sum the tile's rows of each anchor, one atomic per value
        if (want_anc) {
            const int a_first = __float_as_int(Info[0]);
            const int last_row = min(row0 + R, rows) - 1;
            const int a_last = last_row / V;
            const int nseg = a_last - a_first + 1;
            const int ncomp = kFin + 3 + 3 + 3 * K;
            for (int it = tid; it < nseg * ncomp; it += NT) {
                const int seg = it / ncomp, comp = it - seg * ncomp;
                const int an = a_first + seg;
                const int rb = max(an * V - row0, 0), re = min((an + 1) * V - row0, last_row - row0 + 1);
                float s = 0.f;
                if (comp < kFin) {
                    for (int rr = rb; rr < re; ++rr) s += DX[rr * kXS + comp];
                    atomicAdd(gr.g_afeat + (size_t)an * kFin + comp, s);
                } else if (comp < kFin + 3) {
                    const int c = comp - kFin;
                    for (int rr = rb; rr < re; ++rr) {
                        s += DR[rr * 4 + c];
                        for (int k = 0; k < K; ++k) s += SM[(rr * K + k) * 4 + c];
                    }
                    atomicAdd(gr.g_pos + 3 * an + c, s);
                } else if (comp < kFin + 6) {
                    const int c = comp - kFin - 3;
                    for (int rr = rb; rr < re; ++rr) s += DLS[rr * 4 + c];
                    atomicAdd(gr.g_ascale + 3 * an + c, s);
                } else {
                    const int kc = comp - kFin - 6, k = kc / 3, c = kc - 3 * k;
                    for (int rr = rb; rr < re; ++rr) s += SM[(rr * K + k) * 4 + c];
                    atomicAdd(gr.g_offs + ((size_t)an * K + k) * 3 + c, s);
                }
            }
        }
        __syncthreads();
    }
    // ---- flush block accumulators
    if (want_mlp) {
        for (int i = tid; i < 128 * 39; i += NT) {
            const int h = i / 39, c = i - h * 39;
            const float v = AccW1[h * kAccW1S + c];
            if (c < kDin)
                atomicAdd(gr.g_w1 + h * kDin + c, v);
            else
                atomicAdd(gr.g_b1 + h, v);
        }
        int gacc = 0;
        for (int g = 0; g < 4; ++g) {
            const int m = g == 0 ? 1 : g == 1 ? 7 : g == 2 ? 3 : NF;
            if (m == 0) break;
            const int ng = K * m;
            const int r0 = g == 0 ? 0 : g == 1 ? K : g == 2 ? 8 * K : 11 * K;
            for (int i = tid; i < ng * 33; i += NT) {
                const int o = i / 33, j = i - o * 33;
                const float v = AccW2[(gacc + o) * kW2S + j];
                if (j < kH)
                    atomicAdd(gr.g_w2 + (r0 + o) * kH + j, v);
                else
                    atomicAdd(gr.g_b2 + r0 + o, v);
            }
            gacc += pad4(ng);
        }
    }
    if (want_pose) {
        // o_c(xi) = t_wc - R_wc rho (first order): d rho = -W dL/do_c
        for (int v = tid; v < V; v += NT) {
            const DevView &cam = vt.v[v];
            const float *go = aPose + 3 * v;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float s = -(cam.R[3 * i] * go[0] + cam.R[3 * i + 1] * go[1] + cam.R[3 * i + 2] * go[2]);
                atomicAdd(gr.g_pose + 6 * v + i, s);
            }
        }
    }
}

size_t fwd_smem(int n_out) { return sizeof(float) * (4 * kH * kDinP + 4 * kH + n_out * kH + n_out); }

}  // namespace

// Shared memory the decode backward needs for K, n_feat and n_views.
size_t decode_bwd_smem_bytes(int K, int NF, int V) {
    const int R = NF == 32 ? BwdTile<32>::R : BwdTile<16>::R;
    return sizeof(float) * (size_t)bwd_layout(K, NF, R, V).total;
}

size_t decode_smem_limit() { return kMaxSmem; }

cudaError_t launch_decode_fwd(const ViewTable &vt, int A, int K, int NF, const ups_anchors &anc,
                              const ups_mlp &mlp, const ups_gaussians &out, int num_sms,
                              cudaStream_t st) {
    DecodeArgs a{A, K, NF, K * (11 + NF), anc.pos, anc.feat, anc.offsets, anc.scaling,
                 mlp.w1, mlp.b1, mlp.w2, mlp.b2};
    size_t smem = fwd_smem(a.n_out);
    if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
    int rows = A * vt.n;
    int blocks = std::max(1, std::min((rows + 127) / 128, num_sms * 4));
#define UPS_DEC(NFV)                                                                        \
    do {                                                                                    \
        cudaFuncSetAttribute(k_decode_fwd<NFV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                    \
        k_decode_fwd<NFV><<<blocks, 128, smem, st>>>(                                       \
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

cudaError_t launch_decode_bwd(const ViewTable &vt, int A, int K, int NF, const ups_anchors &anc,
                              const ups_mlp &mlp, const ups_gaussians &dG, unsigned mask,
                              const ups_mlp *d_mlp, const ups_anchors *d_anc, float *d_pose,
                              int num_sms, cudaStream_t st) {
    DecodeArgs a{A, K, NF, K * (11 + NF), anc.pos, anc.feat, anc.offsets, anc.scaling,
                 mlp.w1, mlp.b1, mlp.w2, mlp.b2};
    DecodeGrads g{};
    g.d_mean_op = reinterpret_cast<const float4 *>(dG.mean_opacity);
    g.d_scale = reinterpret_cast<const float4 *>(dG.scale);
    g.d_quat = reinterpret_cast<const float4 *>(dG.quat);
    g.d_color = reinterpret_cast<const float4 *>(dG.color);
    g.d_feat = dG.feat;
    if (d_mlp) {
        g.g_w1 = d_mlp->w1;
        g.g_b1 = d_mlp->b1;
        g.g_w2 = d_mlp->w2;
        g.g_b2 = d_mlp->b2;
    }
    if (d_anc) {
        g.g_pos = d_anc->pos;
        g.g_afeat = d_anc->feat;
        g.g_offs = d_anc->offsets;
        g.g_ascale = d_anc->scaling;
    }
    g.g_pose = d_pose;
    g.mask = mask;
    int rows = A * vt.n;
#define UPS_DECB(NFV)                                                                        \
    do {                                                                                     \
        constexpr int R = BwdTile<NFV>::R, NT = BwdTile<NFV>::T;                              \
        const size_t smem = sizeof(float) * (size_t)bwd_layout(K, NFV, R, vt.n).total;       \
        if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;                           \
        const int blocks = std::max(1, std::min((rows + R - 1) / R, num_sms));               \
        cudaFuncSetAttribute(k_decode_bwd<NFV>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             (int)smem);                                                     \
        k_decode_bwd<NFV><<<blocks, NT, smem, st>>>(vt, a, g);                               \
    } while (0)
    switch (NF) {
        case 0: UPS_DECB(0); break;
        case 16: UPS_DECB(16); break;
        case 32: UPS_DECB(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef UPS_DECB
    return cudaGetLastError();
}

}  // namespace ups
