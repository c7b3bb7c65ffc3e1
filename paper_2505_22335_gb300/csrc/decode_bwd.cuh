// Shared pieces of the decode backward (Eq. 8-9 differentiated): the argument
// block of the per-row kernels, the feature-major scratch they hand to the
// weight-gradient kernel, and the per-row epilogue (camera-centre chain rule,
// pose and per-anchor reductions).
//
// Rows are (anchor, view) pairs in anchor-major order, row = anchor * V + view,
// so the rows of one anchor are adjacent: a warp sums them with a segmented
// shuffle scan and one lane per anchor adds the sum to global memory.
#pragma once

#include "common.cuh"

namespace ups {
namespace dbwd {

constexpr int kH = 32;        // hidden width of each MLP
constexpr int kFin = 32;      // anchor feature width
constexpr int kDin = kFin + 6;
constexpr int kXW = 40;       // stored input width: x[0..37], x[38] = 1 (db1 column), x[39] = 0
constexpr int kRowsPerBlock = 128;  // tcgen05 per-row kernel: one thread (TMEM lane) per row
// FP32 per-row kernel shape: 2 CTAs of 256 rows per SM (16 warps at 128
// registers, some spilled) beat 3 CTAs of 128 (12 warps at 168 registers:
// 1.73 ms) at 1.54 ms on the bench workload; with 16 warps the dL/dG loads
// need no software prefetch (UPS_DECB_AHEAD 1: 1.57 ms).
#ifndef UPS_DECB_ROWS
#define UPS_DECB_ROWS 256
#endif
#ifndef UPS_DECB_CTAS
#define UPS_DECB_CTAS 2
#endif
#ifndef UPS_DECB_AHEAD
#define UPS_DECB_AHEAD 0  // dL/dG of Gaussian k + 1 loaded while k is processed
#endif
constexpr int kRowsFp32 = UPS_DECB_ROWS;       // FP32 per-row kernel: rows (threads) per CTA
constexpr int kRowsCtasPerSm = UPS_DECB_CTAS;  // FP32 per-row kernel: resident CTAs per SM (its grid)

__host__ __device__ inline int n_out(int K, int NF) { return K * (11 + NF); }
// group g: outputs per Gaussian and first output row (opacity, covariance,
// colour, feature)
__host__ __device__ inline int grp_m(int g, int NF) { return g == 0 ? 1 : g == 1 ? 7 : g == 2 ? 3 : NF; }
__host__ __device__ inline int grp_r0(int g, int K) { return g == 0 ? 0 : g == 1 ? K : g == 2 ? 8 * K : 11 * K; }

// Scratch of one chunk of rows, feature-major (feature f of local row r at
// [f * ld + r]): X [40], H [128] (post-activation hidden of the four MLPs),
// DY [n_out] (dL/d pre-activation outputs), DZ [128] (dL/d pre-activation
// hidden).  ld is a multiple of 32.
struct Scratch {
    float *X = nullptr, *H = nullptr, *DY = nullptr, *DZ = nullptr;
    int ld = 0;
};
__host__ __device__ inline size_t scratch_floats(int ld, int n_out) {
    return (size_t)ld * (kXW + 128 + n_out + 128);
}
inline Scratch scratch_at(float *base, int ld, int n_out) {
    Scratch s;
    s.X = base;
    s.H = s.X + (size_t)ld * kXW;
    s.DY = s.H + (size_t)ld * 128;
    s.DZ = s.DY + (size_t)ld * n_out;
    s.ld = ld;
    return s;
}

struct Args {
    int A, K, NF;
    int row_begin, row_end;  // rows of this launch (anchor-major)
    const float *pos, *afeat, *offs, *ascale;
    const float *w1, *b1, *w2, *b2;
    const float4 *d_mean_op, *d_scale, *d_quat, *d_color;
    const float *d_feat;
    Scratch s;  // s.X == nullptr: no MLP gradients wanted
    float *g_pos, *g_afeat, *g_offs, *g_ascale, *g_pose;
    unsigned mask;
    int *err;
    int op_tanh;  // opacity = tanh(y) instead of sigmoid(y)
};

// MLP input of anchor `an` seen from `cam`: x = [f_v, delta_vc, d_vc,
// sin(pi t), cos(pi t), 1, 0]; returns delta_vc and d_vc.
__device__ __forceinline__ void mlp_input(const Args &a, const DevView &cam, int an, float x[kXW],
                                          float delta[3], float &dist) {
    const float4 *f4 = reinterpret_cast<const float4 *>(a.afeat + (size_t)an * kFin);
#pragma unroll
    for (int i = 0; i < kFin / 4; ++i) {
        const float4 f = f4[i];
        x[4 * i] = f.x;
        x[4 * i + 1] = f.y;
        x[4 * i + 2] = f.z;
        x[4 * i + 3] = f.w;
    }
    float r[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        // camera centre o_c = -R^T t
        const float oc = -(cam.R[i] * cam.t[0] + cam.R[3 + i] * cam.t[1] + cam.R[6 + i] * cam.t[2]);
        r[i] = a.pos[3 * an + i] - oc;
    }
    dist = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const float id = 1.f / dist;
#pragma unroll
    for (int i = 0; i < 3; ++i) delta[i] = x[kFin + i] = r[i] * id;
    x[kFin + 3] = dist;
    float s, c;
    sincospif(cam.t_norm, &s, &c);
    x[kFin + 4] = s;
    x[kFin + 5] = c;
    x[38] = 1.f;
    x[39] = 0.f;
}

// Segmented inclusive warp scan: lanes hold rows sorted by anchor; bit b of
// `ok` says lane - 2^b holds the same anchor.  The run's last lane ends with
// the run's sum.
__device__ __forceinline__ float seg_scan(float v, unsigned ok) {
#pragma unroll
    for (int b = 0; b < 5; ++b) {
        const float t = __shfl_up_sync(0xffffffffu, v, 1 << b);
        if ((ok >> b) & 1u) v += t;
    }
    return v;
}

struct SegInfo {
    unsigned ok;  // seg_scan mask
    bool tail;    // last lane of its anchor's run within the warp (and a valid row)
};

__device__ __forceinline__ SegInfo seg_info(int an) {  // an < 0: invalid row
    const int lane = threadIdx.x & 31;
    SegInfo s{0u, false};
#pragma unroll
    for (int b = 0; b < 5; ++b) {
        const int up = __shfl_up_sync(0xffffffffu, an, 1 << b);
        if (lane >= (1 << b) && up == an) s.ok |= 1u << b;
    }
    const int dn = __shfl_down_sync(0xffffffffu, an, 1);
    s.tail = an >= 0 && (lane == 31 || dn != an);
    return s;
}

// The end of a row's backward, all threads of the warp together (invalid
// rows pass an = -1 and zeros):
//   dx[0..31] = dL/df_v, dx[32..34] = dL/d delta_vc, dx[35] = dL/d d_vc;
//   dls = dL/d(anchor scaling) of this row; the dL/d(mean) of the row's K
//   Gaussians are read from d_mean_op.
// delta_vc = r / |r|, d_vc = |r| with r = x_v - o_c:  dL/dr = (I - delta
// delta^T) dL/d delta / d + dL/dd delta; x_v gets +dL/dr and the camera centre
// -dL/dr (accumulated per view in aPose, shared memory).  Anchor values are
// summed over the anchor's rows in the warp: one atomic per anchor and value.
__device__ __forceinline__ void row_epilogue(const Args &a, int an, int v, size_t gbase, const float dx[36],
                                             const float delta[3], float dist, const float dls[3],
                                             float *aPose) {
    const bool valid = an >= 0;
    const SegInfo si = seg_info(an);
    float dr[3] = {0.f, 0.f, 0.f};
    if (valid) {
        const float dot = delta[0] * dx[kFin] + delta[1] * dx[kFin + 1] + delta[2] * dx[kFin + 2];
        const float idist = 1.f / dist;
#pragma unroll
        for (int i = 0; i < 3; ++i) dr[i] = (dx[kFin + i] - delta[i] * dot) * idist + dx[kFin + 3] * delta[i];
        if ((a.mask & UPS_GRAD_POSE) && a.g_pose)
#pragma unroll
            for (int i = 0; i < 3; ++i) atomicAdd(aPose + 3 * v + i, -dr[i]);
    }
    if (!(a.mask & UPS_GRAD_ANCHOR)) return;
#pragma unroll 4
    for (int i = 0; i < kFin; ++i) {
        const float s = seg_scan(valid ? dx[i] : 0.f, si.ok);
        if (si.tail) atomicAdd(a.g_afeat + (size_t)an * kFin + i, s);
    }
    float dpos[3] = {dr[0], dr[1], dr[2]};
    for (int k = 0; k < a.K; ++k) {
        const float4 dm = valid ? a.d_mean_op[gbase + k] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float d3[3] = {dm.x, dm.y, dm.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dpos[c] += d3[c];
            const float s = seg_scan(d3[c], si.ok);
            if (si.tail) atomicAdd(a.g_offs + ((size_t)an * a.K + k) * 3 + c, s);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float sp = seg_scan(dpos[c], si.ok);
        const float sl = seg_scan(valid ? dls[c] : 0.f, si.ok);
        if (si.tail) {
            atomicAdd(a.g_pos + 3 * an + c, sp);
            atomicAdd(a.g_ascale + 3 * an + c, sl);
        }
    }
}

// Per-block pose flush: the camera centre o_c(xi) = t_wc - R_wc rho to first
// order, so dL/d rho = -R_cw dL/do_c (rotation rows of T_cw).
__device__ __forceinline__ void flush_pose(const Args &a, const ViewTable &vt, const float *aPose) {
    if (!((a.mask & UPS_GRAD_POSE) && a.g_pose)) return;
    for (int v = threadIdx.x; v < vt.n; v += blockDim.x) {
        const DevView &cam = vt.v[v];
        const float *go = aPose + 3 * v;
#pragma unroll
        for (int i = 0; i < 3; ++i)
            atomicAdd(a.g_pose + 6 * v + i,
                      -(cam.R[3 * i] * go[0] + cam.R[3 * i + 1] * go[1] + cam.R[3 * i + 2] * go[2]));
    }
}

// Called before (begin) and after each kernel launch of the decode backward
// (stage timing and launch counting in the context).
struct StageHook {
    void (*fn)(void *user, const char *name, bool begin, cudaStream_t st);
    void *user;
};

}  // namespace dbwd

// per-row kernels (decode.cu: FP32 on the CUDA cores; decode_bwd_tc.cu: BF16
// operands on the tensor cores) and the weight-gradient kernel
cudaError_t launch_decode_bwd_rows_fp32(const ViewTable &vt, const dbwd::Args &a, int num_sms, cudaStream_t st);
cudaError_t launch_decode_bwd_rows_tc(const ViewTable &vt, const dbwd::Args &a, int num_sms, cudaStream_t st);
size_t decode_bwd_rows_tc_smem(int NF, int K);
// rows the per-row kernel's resident grid covers in one pass (FP32: 3 CTAs of
// 128 rows per SM; tcgen05: 1 or 2 CTAs per SM by shared memory)
int decode_bwd_rows_wave(int bf16, int K, int NF, int num_sms);
bool decode_wgrad_tc_fits(int K, int NF);
cudaError_t launch_decode_wgrad_tc(const float *scratch, int ld, int nrows, int K, int NF, const ups_mlp &d_mlp,
                                   int *err, int num_sms, cudaStream_t st);

}  // namespace ups
