// Per-anchor MLP decode of K neural Gaussians (Eq. 8-9) and its backward,
// FP32 on the CUDA cores.
//
// Row = (anchor, view).  MLP input x = [f_v, delta_vc, d_vc, sin(pi t),
// cos(pi t)]; four MLPs (opacity, covariance, colour: ReLU hidden; feature
// F_d: SoftPlus hidden) of width `hidden` = 32.  Weights live in shared memory
// and are read as float4 broadcasts (every lane of a warp reads the same
// weight), so the inner loops are FMA-bound.
//
// Backward: one thread per row recomputes the forward, back-propagates to the
// input, and produces its share of the weight gradients; the per-row outer
// products are summed over the 32 rows of a warp with a transposed butterfly
// (each lane ends up owning one hidden unit) and added to per-block shared
// accumulators, which are flushed to global memory once per block.
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

// Sum a 32-vector over the warp; on return lane L holds the sum of element L.
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32], int lane) {
#pragma unroll
    for (int o = 16, n = 32; o >= 1; o >>= 1, n >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (i < n / 2) {
                float send = up ? v[i] : v[i + n / 2];
                float keep = up ? v[i + n / 2] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
    return v[0];
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

struct DecodeGrads {
    const float4 *d_mean_op, *d_scale, *d_quat, *d_color;
    const float *d_feat;
    float *g_w1, *g_b1, *g_w2, *g_b2;            // MLP (accumulated)
    float *g_pos, *g_afeat, *g_offs, *g_ascale;  // anchors (accumulated)
    float *g_pose;                               // [V][6] (accumulated)
    unsigned mask;
};

constexpr int kAccW1Stride = 41;  // odd stride: conflict-free column writes
constexpr int kXStride = 41;

template <int NF>
__global__ void __launch_bounds__(128) k_decode_bwd(ViewTable vt, DecodeArgs a, DecodeGrads gr) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int n_out = a.n_out;
    float *sW1 = sm;
    float *sb1 = sW1 + 4 * kH * kDinP;
    float *sW2 = sb1 + 4 * kH;
    float *sb2 = sW2 + n_out * kH;
    float *aW1 = sb2 + n_out;                    // [128][41]
    float *ab1 = aW1 + 4 * kH * kAccW1Stride;    // [128]
    float *aW2 = ab1 + 4 * kH;                   // [n_out][32]
    float *ab2 = aW2 + n_out * kH;               // [n_out]
    float *aPose = ab2 + n_out;                  // [V][3] camera-centre gradient
    float *sX = aPose + 3 * vt.n;                // [128][41] per-thread MLP input
    load_weights(a, sW1, sb1, sW2, sb2);
    const bool want_mlp = gr.mask & UPS_GRAD_MLP;
    const bool want_anc = gr.mask & UPS_GRAD_ANCHOR;
    const bool want_pose = gr.mask & UPS_GRAD_POSE;
    for (int i = threadIdx.x; i < 4 * kH * kAccW1Stride + 4 * kH + n_out * kH + n_out + 3 * vt.n;
         i += blockDim.x)
        aW1[i] = 0.f;
    __syncthreads();
    const int K = a.K, V = vt.n;
    const int lane = threadIdx.x & 31;
    const int rows = a.A * V;
    const size_t NG = (size_t)a.A * K;
    const int nrow_iter = (rows + gridDim.x * blockDim.x - 1) / (gridDim.x * blockDim.x);
    for (int it = 0; it < nrow_iter; ++it) {
        const int row = (it * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
        const bool valid = row < rows;
        const int an = valid ? row / V : 0, v = valid ? row - an * V : 0;
        const DevView &cam = vt.v[v];
        float x[kDinP], delta[3], dist;
        mlp_input(a, cam, an, x, delta, dist);
        float dx[kDinP];
#pragma unroll
        for (int i = 0; i < kDinP; ++i) {
            dx[i] = 0.f;
            sX[threadIdx.x * kXStride + i] = x[i];
        }
        const size_t gbase = (size_t)v * NG + (size_t)an * K;
        float dls[3] = {0.f, 0.f, 0.f};
        for (int g = 0; g < 4; ++g) {
            if (g == 3 && NF == 0) break;
            float z[kH], h[kH], dh[kH];
            hidden_pre(sW1, sb1, g, x, z);
#pragma unroll
            for (int j = 0; j < kH; ++j) {
                h[j] = g < 3 ? fmaxf(z[j], 0.f) : softplus(z[j]);
                dh[j] = 0.f;
            }
            const int m = g == 0 ? 1 : g == 1 ? 7 : g == 2 ? 3 : NF;
            const int r0 = g == 0 ? 0 : g == 1 ? K : g == 2 ? 8 * K : 11 * K;
            for (int k = 0; k < K; ++k) {
                const size_t gi = gbase + k;
                for (int c = 0; c < m; ++c) {
                    const int r = r0 + m * k + c;
                    float dy = 0.f;
                    if (valid) {
                        float y = out_row(sW2, sb2, r, h);
                        if (g == 0) {
                            float o = sigm(y);
                            dy = gr.d_mean_op[gi].w * o * (1.f - o);
                        } else if (g == 1) {
                            if (c < 3) {
                                float s = sigm(y);
                                float l = a.ascale[3 * an + c];
                                float ds = reinterpret_cast<const float *>(gr.d_scale + gi)[c];
                                dy = ds * l * s * (1.f - s);
                                dls[c] += ds * s;
                            } else {
                                dy = reinterpret_cast<const float *>(gr.d_quat + gi)[c - 3];
                            }
                        } else if (g == 2) {
                            float cc = sigm(y);
                            dy = reinterpret_cast<const float *>(gr.d_color + gi)[c] * cc * (1.f - cc);
                        } else {
                            dy = gr.d_feat[gi * NF + c];
                        }
                    }
                    // dh += dy W2[r]
                    const float4 *w = reinterpret_cast<const float4 *>(sW2 + r * kH);
#pragma unroll
                    for (int q = 0; q < kH / 4; ++q) {
                        float4 ww = w[q];
                        dh[4 * q] = fmaf(dy, ww.x, dh[4 * q]);
                        dh[4 * q + 1] = fmaf(dy, ww.y, dh[4 * q + 1]);
                        dh[4 * q + 2] = fmaf(dy, ww.z, dh[4 * q + 2]);
                        dh[4 * q + 3] = fmaf(dy, ww.w, dh[4 * q + 3]);
                    }
                    if (want_mlp && __any_sync(0xffffffffu, dy != 0.f)) {
                        float p[32];
#pragma unroll
                        for (int j = 0; j < kH; ++j) p[j] = dy * h[j];
                        float s = warp_transpose_sum32(p, lane);
                        atomicAdd(aW2 + r * kH + lane, s);
                        float sb = warp_sum(dy);
                        if (lane == 0) atomicAdd(ab2 + r, sb);
                    }
                }
            }
            // through the hidden activation
            float dz[kH];
#pragma unroll
            for (int j = 0; j < kH; ++j)
                dz[j] = g < 3 ? (z[j] > 0.f ? dh[j] : 0.f) : dh[j] * sigm(z[j]);
            // dx += W1_g^T dz
#pragma unroll 4
            for (int j = 0; j < kH; ++j) {
                const float4 *w = reinterpret_cast<const float4 *>(sW1 + (g * kH + j) * kDinP);
#pragma unroll
                for (int q = 0; q < kDinP / 4; ++q) {
                    float4 ww = w[q];
                    dx[4 * q] = fmaf(dz[j], ww.x, dx[4 * q]);
                    dx[4 * q + 1] = fmaf(dz[j], ww.y, dx[4 * q + 1]);
                    dx[4 * q + 2] = fmaf(dz[j], ww.z, dx[4 * q + 2]);
                    dx[4 * q + 3] = fmaf(dz[j], ww.w, dx[4 * q + 3]);
                }
            }
            if (want_mlp) {
                // db1 and dW1_g[j][i] = sum over rows dz_j x_i
                float p[32];
#pragma unroll
                for (int j = 0; j < kH; ++j) p[j] = dz[j];
                float s = warp_transpose_sum32(p, lane);
                atomicAdd(ab1 + g * kH + lane, s);
#pragma unroll 1
                for (int i = 0; i < kDin; ++i) {
                    const float xi = sX[threadIdx.x * kXStride + i];
#pragma unroll
                    for (int j = 0; j < kH; ++j) p[j] = dz[j] * xi;
                    float t = warp_transpose_sum32(p, lane);
                    atomicAdd(aW1 + (g * kH + lane) * kAccW1Stride + i, t);
                }
            }
        }
        if (!valid) continue;
        // anchor and camera-centre gradients
        float dmu[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < K; ++k) {
            float4 dm = gr.d_mean_op[gbase + k];
            if (want_anc) {
                float *o3 = gr.g_offs + ((size_t)an * K + k) * 3;
                atomicAdd(o3, dm.x);
                atomicAdd(o3 + 1, dm.y);
                atomicAdd(o3 + 2, dm.z);
            }
            dmu[0] += dm.x;
            dmu[1] += dm.y;
            dmu[2] += dm.z;
        }
        // delta = r/|r|, d = |r|, r = x_v - o_c
        float ddl[3] = {dx[kFin], dx[kFin + 1], dx[kFin + 2]}, dd = dx[kFin + 3];
        float dot = delta[0] * ddl[0] + delta[1] * ddl[1] + delta[2] * ddl[2];
        float idist = 1.f / dist;
        float dr[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) dr[i] = (ddl[i] - delta[i] * dot) * idist + dd * delta[i];
        if (want_anc) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                atomicAdd(gr.g_pos + 3 * an + i, dmu[i] + dr[i]);
                atomicAdd(gr.g_ascale + 3 * an + i, dls[i]);
            }
            float *gf = gr.g_afeat + (size_t)an * kFin;
#pragma unroll
            for (int i = 0; i < kFin; ++i) atomicAdd(gf + i, dx[i]);
        }
        if (want_pose) {
            // dL/do_c = -dr
#pragma unroll
            for (int i = 0; i < 3; ++i) atomicAdd(aPose + 3 * v + i, -dr[i]);
        }
    }
    __syncthreads();
    // flush block accumulators
    if (want_mlp) {
        for (int i = threadIdx.x; i < 4 * kH * kDin; i += blockDim.x) {
            int r = i / kDin, c = i - r * kDin;
            atomicAdd(gr.g_w1 + i, aW1[r * kAccW1Stride + c]);
        }
        for (int i = threadIdx.x; i < 4 * kH; i += blockDim.x) atomicAdd(gr.g_b1 + i, ab1[i]);
        for (int i = threadIdx.x; i < n_out * kH; i += blockDim.x) atomicAdd(gr.g_w2 + i, aW2[i]);
        for (int i = threadIdx.x; i < n_out; i += blockDim.x) atomicAdd(gr.g_b2 + i, ab2[i]);
    }
    if (want_pose) {
        // o_c(xi) = t_wc - R_wc rho (first order): d rho = -W dL/do_c
        for (int v = threadIdx.x; v < V; v += blockDim.x) {
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
size_t bwd_smem(int n_out, int V) {
    return fwd_smem(n_out) +
           sizeof(float) * (4 * kH * kAccW1Stride + 4 * kH + n_out * kH + n_out + 3 * V +
                            128 * kXStride);
}

}  // namespace

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
    size_t smem = bwd_smem(a.n_out, vt.n);
    if (smem > kMaxSmem) return cudaErrorInvalidConfiguration;
    int rows = A * vt.n;
    int blocks = std::max(1, std::min((rows + 127) / 128, num_sms * 2));
#define UPS_DECB(NFV)                                                                        \
    do {                                                                                     \
        cudaFuncSetAttribute(k_decode_bwd<NFV>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             (int)smem);                                                     \
        k_decode_bwd<NFV><<<blocks, 128, smem, st>>>(vt, a, g);                              \
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
