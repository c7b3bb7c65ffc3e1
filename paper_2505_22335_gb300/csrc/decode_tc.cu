// Decode (Eq. 8-9) on the 5th-generation tensor cores (tcgen05).
//
// One 128-thread CTA works on tiles of 128 (anchor, view) rows; thread t owns
// row t, which is also TMEM lane t.  Per MLP group g (opacity, covariance,
// colour, feature F_d):
//   Z_g[128 x 32]  = X[128 x Kin] . W1_g^T         (tcgen05.mma, D in TMEM)
//   H_g = act(Z_g + b1_g)                          (CUDA cores, back to smem)
//   Y_g[128 x 16m] = H_g[128 x 32] . W2_g'^T        (tcgen05.mma)
//   outputs = activation(Y_g + b2_g)               (CUDA cores, to HBM)
// W2_g' holds the group's output rows reordered component-major with 16 slots
// per component (slot = Gaussian index k < K), so each component of all K
// Gaussians is one aligned 16-column TMEM load.
//
// Precision: kBF16 rounds operands to BF16 (FP32 accumulation); kTF32 splits
// every operand into a TF32 high part and an FP32 remainder and accumulates
// hi*hi + hi*lo + lo*hi, which gives FP32-level results.
#include <algorithm>

#include "common.cuh"
#include "umma.cuh"

namespace ups {

namespace {

using namespace umma;

constexpr int kTCRows = 128;
constexpr int kH = 32;
constexpr int kFin = 32;
constexpr int kDin = kFin + 6;
constexpr uint32_t kTmemCols = 128;  // Z: [0, 32), Y chunk of <= 4 components: [32, 96)
constexpr int kChunk = 4;            // output components per Y chunk
constexpr int kWaitLimit = 1 << 22;

struct TcArgs {
    int A, K, NF;
    const float *pos, *afeat, *offs, *ascale;
    const float *w1, *b1, *w2, *b2;
    float4 *mean_op, *scale, *quat, *color;
    float *feat;
    int *err;
    int op_tanh;  // opacity = tanh(y) instead of sigmoid(y)
};

template <Kind KD> struct Prec {
    static constexpr int esize = KD == kBF16 ? 2 : 4;
    static constexpr int kin = KD == kBF16 ? 48 : 40;         // input width padded to the MMA K step
    static constexpr int xbytes = kin * esize;                 // bytes per X row
    static constexpr int hbytes = kH * esize;                  // bytes per H row
    static constexpr int kstep_bytes = 32;                     // K bytes per MMA instruction
};

__device__ __forceinline__ float sig(float x) { return 1.f / (1.f + __expf(-x)); }
__device__ __forceinline__ float softplus(float x) { return x > 20.f ? x : log1pf(__expf(x)); }

// store a value into a K-major operand (hi part, and lo part for TF32)
template <Kind KD>
__device__ __forceinline__ void put(unsigned char *hi, unsigned char *lo, int row, int k, int kbytes,
                                    float v) {
    const uint32_t off = kmajor_offset(row, k, kbytes, Prec<KD>::esize);
    if (KD == kBF16) {
        *reinterpret_cast<__nv_bfloat16 *>(hi + off) = __float2bfloat16_rn(v);
    } else {
        const float h = tf32_hi(v);
        *reinterpret_cast<float *>(hi + off) = h;
        *reinterpret_cast<float *>(lo + off) = v - h;
    }
}

// Issue D (+)= A . B^T over `ksteps` 32-byte K steps (all passes), then commit.
template <Kind KD>
__device__ __forceinline__ void gemm(uint32_t tmem_d, const unsigned char *a_hi, const unsigned char *a_lo,
                                     const unsigned char *b_hi, const unsigned char *b_lo, uint32_t a_kbytes,
                                     uint32_t b_kbytes, int ksteps, uint32_t id, uint64_t *mbar) {
    const uint32_t ah = smem_addr(a_hi), bh = smem_addr(b_hi);
    const uint32_t al = KD == kTF32 ? smem_addr(a_lo) : 0u, bl = KD == kTF32 ? smem_addr(b_lo) : 0u;
    uint32_t acc = 0;
    for (int ks = 0; ks < ksteps; ++ks) {
        const uint32_t o = (uint32_t)ks * 256;  // two core matrices along K per step
        mma<KD>(tmem_d, desc(ah + o, a_kbytes), desc(bh + o, b_kbytes), id, acc);
        acc = 1;
        if (KD == kTF32) {
            mma<KD>(tmem_d, desc(ah + o, a_kbytes), desc(bl + o, b_kbytes), id, 1);
            mma<KD>(tmem_d, desc(al + o, a_kbytes), desc(bh + o, b_kbytes), id, 1);
        }
    }
    commit(mbar);
}

struct TcLayout {
    int n_w2rows;  // rows of the reordered W2 (sum over groups of 16 m)
    int oX, oXl, oH, oHl, oW1, oW1l, oW2, oW2l, ob1, ob2, total;
};

template <Kind KD>
__host__ __device__ inline TcLayout tc_layout(int NF) {
    using P = Prec<KD>;
    TcLayout L;
    L.n_w2rows = 16 * (1 + 7 + 3 + NF);
    const int two = KD == kTF32 ? 1 : 0;
    int o = 0;
    auto take = [&](int bytes) { int r = o; o += (bytes + 1023) & ~1023; return r; };
    L.oX = take(kTCRows * P::xbytes);
    L.oXl = two ? take(kTCRows * P::xbytes) : L.oX;
    L.oH = take(kTCRows * P::hbytes);
    L.oHl = two ? take(kTCRows * P::hbytes) : L.oH;
    L.oW1 = take(4 * kH * P::xbytes);
    L.oW1l = two ? take(4 * kH * P::xbytes) : L.oW1;
    L.oW2 = take(L.n_w2rows * P::hbytes);
    L.oW2l = two ? take(L.n_w2rows * P::hbytes) : L.oW2;
    L.ob1 = take(4 * kH * 4);
    L.ob2 = take(L.n_w2rows * 4);
    L.total = o;
    return L;
}

// component-major reordered W2 row of (group g, component c, Gaussian k)
__host__ __device__ inline int w2_row_base(int g, int NF) {
    return g == 0 ? 0 : g == 1 ? 16 : g == 2 ? 16 * 8 : 16 * 11;
    (void)NF;
}

template <int NF, Kind KD>
__global__ void __launch_bounds__(kTCRows, 3) k_decode_fwd_tc(ViewTable vt, TcArgs a) {
    using P = Prec<KD>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const TcLayout L = tc_layout<KD>(NF);
    unsigned char *X = smem + L.oX, *Xl = smem + L.oXl, *Hs = smem + L.oH, *Hl = smem + L.oHl;
    unsigned char *W1 = smem + L.oW1, *W1l = smem + L.oW1l, *W2 = smem + L.oW2, *W2l = smem + L.oW2l;
    float *b1 = reinterpret_cast<float *>(smem + L.ob1), *b2 = reinterpret_cast<float *>(smem + L.ob2);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int K = a.K;
    // ---- weights: W1 rows per hidden unit (K-major over inputs), W2 reordered
    for (int i = tid; i < 4 * kH * P::kin; i += kTCRows) {
        const int h = i / P::kin, c = i - h * P::kin;
        put<KD>(W1, W1l, h, c, P::xbytes, c < kDin ? a.w1[h * kDin + c] : 0.f);
    }
    for (int i = tid; i < 4 * kH; i += kTCRows) b1[i] = a.b1[i];
    for (int i = tid; i < L.n_w2rows * kH; i += kTCRows) {
        const int rr = i / kH, j = i - rr * kH;
        // rr -> (group, component, slot k)
        int g, base;
        if (rr < 16) g = 0, base = 0;
        else if (rr < 16 * 8) g = 1, base = 16;
        else if (rr < 16 * 11) g = 2, base = 16 * 8;
        else g = 3, base = 16 * 11;
        const int m = g == 0 ? 1 : g == 1 ? 7 : g == 2 ? 3 : NF;
        const int r0 = g == 0 ? 0 : g == 1 ? K : g == 2 ? 8 * K : 11 * K;
        const int c = (rr - base) >> 4, k = (rr - base) & 15;
        float w = 0.f, bb = 0.f;
        if (k < K) {
            w = a.w2[(r0 + m * k + c) * kH + j];
            bb = a.b2[r0 + m * k + c];
        }
        put<KD>(W2, W2l, rr, j, P::hbytes, w);
        if (j == 0) b2[rr] = bb;
    }
    if (tid == 0) {
        mbar_init(&mbar, 1);
        s_fail = 0;
    }
    if (warp == 0) tmem_alloc(&tmem_base, kTmemCols);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    const int rows = a.A * vt.n;
    const int ntiles = (rows + kTCRows - 1) / kTCRows;
    const size_t NG = (size_t)a.A * K;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int row = tile * kTCRows + tid;
        const bool valid = row < rows;
        const int v = valid ? row / a.A : 0, an = valid ? row - v * a.A : 0;
        const DevView &cam = vt.v[v];
        // ---- MLP input of this row
        {
            float x[kDin];
            const float4 *f4 = reinterpret_cast<const float4 *>(a.afeat + (size_t)an * kFin);
#pragma unroll
            for (int i = 0; i < kFin / 4; ++i) {
                float4 f = f4[i];
                x[4 * i] = f.x;
                x[4 * i + 1] = f.y;
                x[4 * i + 2] = f.z;
                x[4 * i + 3] = f.w;
            }
            float oc[3], r[3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                oc[i] = -(cam.R[i] * cam.t[0] + cam.R[3 + i] * cam.t[1] + cam.R[6 + i] * cam.t[2]);
#pragma unroll
            for (int i = 0; i < 3; ++i) r[i] = a.pos[3 * an + i] - oc[i];
            const float dist = sqrtf(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
            const float id = 1.f / dist;
#pragma unroll
            for (int i = 0; i < 3; ++i) x[kFin + i] = r[i] * id;
            x[kFin + 3] = dist;
            float s, c;
            sincospif(cam.t_norm, &s, &c);
            x[kFin + 4] = s;
            x[kFin + 5] = c;
#pragma unroll
            for (int i = 0; i < P::kin; ++i) put<KD>(X, Xl, tid, i, P::xbytes, (valid && i < kDin) ? x[i] : 0.f);
        }
        fence_async_smem();
        __syncthreads();
        const size_t gbase = (size_t)v * NG + (size_t)an * K;
        float op[16], qw[16];
        for (int g = 0; g < 4 && ok; ++g) {
            const int m = g == 0 ? 1 : g == 1 ? 7 : g == 2 ? 3 : NF;
            if (m == 0) break;
            // Z_g = X . W1_g^T  -> TMEM columns [0, 32)
            if (tid == 0)
                gemm<KD>(tmem, X, Xl, W1 + g * kH * P::xbytes, W1l + g * kH * P::xbytes, P::xbytes, P::xbytes,
                         P::xbytes / P::kstep_bytes, idesc(KD, kTCRows, kH), &mbar);
            bool w_ok = mbar_wait(&mbar, phase, kWaitLimit);
            phase ^= 1u;
            if (__syncthreads_or(!w_ok)) {
                ok = false;
                break;
            }
            fence_after();
            {
                float z[32];
                float t16[16];
                tmem_ld16(lane_addr + 0, t16);
#pragma unroll
                for (int i = 0; i < 16; ++i) z[i] = t16[i];
                tmem_ld16(lane_addr + 16, t16);
#pragma unroll
                for (int i = 0; i < 16; ++i) z[16 + i] = t16[i];
#pragma unroll
                for (int j = 0; j < kH; ++j) {
                    const float zz = z[j] + b1[g * kH + j];
                    put<KD>(Hs, Hl, tid, j, P::hbytes, g < 3 ? fmaxf(zz, 0.f) : softplus(zz));
                }
            }
            fence_before();
            fence_async_smem();
            __syncthreads();
            fence_after();
            // Y_g in chunks of at most kChunk components (16 columns each) -> TMEM [32, 96)
            const int rbase = w2_row_base(g, NF);
            for (int c0 = 0; c0 < m && ok; c0 += kChunk) {
                const int nc = min(kChunk, m - c0);
                if (tid == 0)
                    gemm<KD>(tmem + 32, Hs, Hl, W2 + (rbase + 16 * c0) * P::hbytes,
                             W2l + (rbase + 16 * c0) * P::hbytes, P::hbytes, P::hbytes,
                             P::hbytes / P::kstep_bytes, idesc(KD, kTCRows, 16 * nc), &mbar);
                w_ok = mbar_wait(&mbar, phase, kWaitLimit);
                phase ^= 1u;
                if (__syncthreads_or(!w_ok)) {
                    ok = false;
                    break;
                }
                fence_after();
                // epilogue: component c of the K Gaussians is one 16-column load
                if (g == 0) {
                    float y[16];
                    tmem_ld16(lane_addr + 32, y);
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        op[k] = a.op_tanh ? tanhf(y[k] + b2[rbase + k]) : sig(y[k] + b2[rbase + k]);
                } else if (g == 1 && c0 == 0) {
                    // components 0..3 = scale x, y, z and quaternion w
                    float s0[16], s1[16], s2[16];
                    tmem_ld16(lane_addr + 32 + 0, s0);
                    tmem_ld16(lane_addr + 32 + 16, s1);
                    tmem_ld16(lane_addr + 32 + 32, s2);
                    const float lx = a.ascale[3 * an], ly = a.ascale[3 * an + 1], lz = a.ascale[3 * an + 2];
                    const float px = a.pos[3 * an], py = a.pos[3 * an + 1], pz = a.pos[3 * an + 2];
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        if (k < K && valid) {
                            a.scale[gbase + k] = make_float4(lx * sig(s0[k] + b2[rbase + k]),
                                                             ly * sig(s1[k] + b2[rbase + 16 + k]),
                                                             lz * sig(s2[k] + b2[rbase + 32 + k]), 0.f);
                            const float *o3 = a.offs + ((size_t)an * K + k) * 3;
                            a.mean_op[gbase + k] = make_float4(px + o3[0], py + o3[1], pz + o3[2], op[k]);
                        }
                    }
                    tmem_ld16(lane_addr + 32 + 48, qw);
#pragma unroll
                    for (int k = 0; k < 16; ++k) qw[k] += b2[rbase + 48 + k];
                } else if (g == 1) {
                    // components 4..6 = quaternion x, y, z
                    float q1[16], q2[16], q3[16];
                    tmem_ld16(lane_addr + 32 + 0, q1);
                    tmem_ld16(lane_addr + 32 + 16, q2);
                    tmem_ld16(lane_addr + 32 + 32, q3);
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < K && valid)
                            a.quat[gbase + k] = make_float4(qw[k], q1[k] + b2[rbase + 64 + k],
                                                            q2[k] + b2[rbase + 80 + k], q3[k] + b2[rbase + 96 + k]);
                } else if (g == 2) {
                    float c0v[16], c1v[16], c2v[16];
                    tmem_ld16(lane_addr + 32, c0v);
                    tmem_ld16(lane_addr + 48, c1v);
                    tmem_ld16(lane_addr + 64, c2v);
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < K && valid)
                            a.color[gbase + k] = make_float4(sig(c0v[k] + b2[rbase + k]), sig(c1v[k] + b2[rbase + 16 + k]),
                                                             sig(c2v[k] + b2[rbase + 32 + k]), 0.f);
                } else {
                    {
                        float f0[16], f1[16], f2[16], f3[16];
                        tmem_ld16(lane_addr + 32, f0);
                        tmem_ld16(lane_addr + 32 + 16, f1);
                        tmem_ld16(lane_addr + 32 + 32, f2);
                        tmem_ld16(lane_addr + 32 + 48, f3);
                        const int cc = c0;
                        const float *bb = b2 + rbase + 16 * cc;
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            if (k < K && valid)
                                *reinterpret_cast<float4 *>(a.feat + (gbase + k) * NF + cc) =
                                    make_float4(f0[k] + bb[k], f1[k] + bb[16 + k], f2[k] + bb[32 + k], f3[k] + bb[48 + k]);
                    }
                }
                fence_before();
                __syncthreads();
                fence_after();
            }
        }
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

size_t decode_tc_smem_bytes(int NF, int bf16) {
    return (size_t)(bf16 ? tc_layout<kBF16>(NF).total : tc_layout<kTF32>(NF).total);
}

cudaError_t launch_decode_fwd_tc(const ViewTable &vt, int A, int K, int NF, const ups_anchors &anc,
                                 const ups_mlp &mlp, const ups_gaussians &out, int bf16, int op_tanh, int *err,
                                 int num_sms, cudaStream_t st) {
    TcArgs a{A, K, NF, anc.pos, anc.feat, anc.offsets, anc.scaling, mlp.w1, mlp.b1, mlp.w2, mlp.b2,
             reinterpret_cast<float4 *>(out.mean_opacity), reinterpret_cast<float4 *>(out.scale),
             reinterpret_cast<float4 *>(out.quat), reinterpret_cast<float4 *>(out.color), out.feat, err, op_tanh};
    if (K < 1 || K > 16) return cudaErrorInvalidValue;
    const int rows = A * vt.n;
    const int tiles = (rows + kTCRows - 1) / kTCRows;
    // several CTAs per SM overlap one CTA's MMA waits with another's epilogue;
    // each holds 128 TMEM columns (4 x 128 = the SM's 512)
    const int blocks = std::max(1, std::min(tiles, num_sms * 3));
#define UPS_TC(NFV, KDV)                                                                             \
    do {                                                                                             \
        const size_t smem = (size_t)tc_layout<KDV>(NFV).total;                                      \
        if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;                                 \
        cudaFuncSetAttribute(k_decode_fwd_tc<NFV, KDV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                            \
        k_decode_fwd_tc<NFV, KDV><<<blocks, kTCRows, smem, st>>>(vt, a);                             \
    } while (0)
    if (bf16) {
        switch (NF) {
            case 0: UPS_TC(0, kBF16); break;
            case 16: UPS_TC(16, kBF16); break;
            case 32: UPS_TC(32, kBF16); break;
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (NF) {
            case 0: UPS_TC(0, kTF32); break;
            case 16: UPS_TC(16, kTF32); break;
            case 32: UPS_TC(32, kTF32); break;
            default: return cudaErrorInvalidValue;
        }
    }
#undef UPS_TC
    return cudaGetLastError();
}

}  // namespace ups
