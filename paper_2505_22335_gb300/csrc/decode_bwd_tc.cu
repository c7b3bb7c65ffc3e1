// Decode backward (Eq. 8-9 differentiated) with BF16 operands on the tcgen05
// tensor cores, the weight-gradient reduction shared with the FP32 path, and
// the host-side driver of both.
//
// k_decode_bwd_rows_tc: one 128-row tile per step, thread t = row t = TMEM lane
// t, rows anchor-major (row = anchor * V + view).  Per MLP group g:
//   Z_g  = X . W1_g^T                    (MMA)   H_g = act(Z_g + b1)
//   Y_g  = H_g . W2nl_g^T                (MMA, only the outputs whose activation
//                                         has a derivative: opacity, scale, colour)
//   DY_g = dL/dY (CUDA cores, from dL/dG through the output activations)
//   DH_g = DY_g . W2_g                   (MMA, a few output components per step)
//   DZ_g = DH_g * act'(Z_g)
//   DX  += DZ_g . W1_g                   (MMA, accumulated over the groups)
// then the per-row epilogue (camera centre, pose, per-anchor sums).  Z of all
// four groups is one MMA (N = 128) at the start of the tile.  DY is produced
// Gaussian-major (all components of a few Gaussians per chunk) so each thread
// reads its dL/dG records as whole float4s.  Operands are canonical K-major,
// no swizzle, in shared memory, written as 16-byte core-matrix rows;
// accumulators in TMEM: Z [0,128) Y [128,176) DH [176,208) DX [208,256).
//
// k_decode_wgrad: dW2_g = DY_g^T H_g (+ db2 = 1^T DY_g) and dW1 = DZ^T X (+ db1
// from the constant-1 column of X), FP32, over the feature-major scratch the
// per-row kernels wrote: 32-row chunks double-buffered into shared memory with
// cp.async, 4 x 8 register micro-tiles, one atomic per weight per block
// (db2 from per-feature sums of the staged DY).
#include <algorithm>

#include "decode_bwd.cuh"
#include "umma.cuh"

namespace ups {

using dbwd::kDin;
using dbwd::kFin;
using dbwd::kH;
using dbwd::kXW;

namespace {

using namespace umma;

constexpr int kRows = dbwd::kRowsPerBlock;
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t cZ = 0, cY = 128, cDH = 176, cDX = 208;  // Z of all groups, Y, DH, DX
constexpr int kWait = 1 << 22;
constexpr int kKin = 48;  // X / W1 K extent (38 inputs, zero padded)

__device__ __forceinline__ float sig(float x) { return 1.f / (1.f + __expf(-x)); }
__device__ __forceinline__ float softplus(float x) { return x > 20.f ? x : log1pf(__expf(x)); }

__device__ __forceinline__ void put(unsigned char *base, int row, int k, int kbytes, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + kmajor_offset(row, k, kbytes, 2)) = __float2bfloat16_rn(v);
}

__device__ __forceinline__ void mma_chain(uint32_t tmem_d, uint32_t a, uint32_t a_kbytes, uint32_t b,
                                          uint32_t b_kbytes, int ksteps, uint32_t id, bool accumulate) {
    for (int ks = 0; ks < ksteps; ++ks)
        mma<kBF16>(tmem_d, desc(a + 256u * ks, a_kbytes), desc(b + 256u * ks, b_kbytes), id,
                   (accumulate || ks > 0) ? 1u : 0u);
}

// nonlinear outputs of group g: opacity (1), scale (3), colour (3); rows of
// W2nl: g0 [0,16), g1 [16,64), g2 [64,112) (16 slots per component)
__host__ __device__ constexpr int nl_comps(int g) { return g == 0 ? 1 : g == 3 ? 0 : 3; }
__host__ __device__ constexpr int nl_base(int g) { return g == 0 ? 0 : g == 1 ? 16 : 64; }
// DY K index of output (Gaussian k, component c) of group g: k * mp + c, the
// components padded to mp; kc Gaussians fill one 64-element DY chunk
__host__ __device__ constexpr int mp_of(int g, int NF) { return g == 0 ? 1 : g == 1 ? 8 : g == 2 ? 4 : NF; }
__host__ __device__ constexpr int kc_of(int g, int NF) { return g == 0 ? 16 : NF == 0 && g == 3 ? 1 : 64 / mp_of(g, NF); }
// K extent of W2T_g: Gaussians padded so that every chunk is whole MMA K steps
__host__ __device__ inline int w2t_extent(int g, int NF, int K) {
    const int mp = mp_of(g, NF);
    if (mp == 0) return 0;
    const int step = mp >= 16 ? 1 : 16 / mp;
    return (K + step - 1) / step * step * mp;
}

struct Layout {
    int oW1, oW2nl, oW2T[4], eW2T[4], oW1T, ob1, ob2nl, oX, oH, oDY, oDZ, total;
};

__host__ __device__ inline Layout rows_layout(int NF, int K) {
    Layout L{};
    int o = 0;
    auto take = [&](int bytes) { const int r = o; o += (bytes + 1023) & ~1023; return r; };
    L.oW1 = take(128 * kKin * 2);
    L.oW2nl = take(112 * kH * 2);
    for (int g = 0; g < 4; ++g) {
        L.eW2T[g] = w2t_extent(g, NF, K);
        L.oW2T[g] = L.eW2T[g] ? take(kH * L.eW2T[g] * 2) : o;
    }
    L.oW1T = take(kKin * 128 * 2);
    L.ob1 = take(128 * 4);
    L.ob2nl = take(112 * 4);
    L.oX = take(kRows * kKin * 2);
    L.oH = take(kRows * kH * 2);
    L.oDY = take(kRows * 64 * 2);
    L.oDZ = take(kRows * kH * 2);
    L.total = o;
    return L;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a at the lower address
    return *reinterpret_cast<const uint32_t *>(&h);
}

// elements [8 k8, 8 k8 + 8) of operand row `row`: one core-matrix row, one
// 16-byte store (the 8 rows of a core matrix fill all banks once)
__device__ __forceinline__ void put8(unsigned char *base, int row, int k8, int kbytes, const float *v) {
    uint4 u;
    u.x = pack2(v[0], v[1]);
    u.y = pack2(v[2], v[3]);
    u.z = pack2(v[4], v[5]);
    u.w = pack2(v[6], v[7]);
    *reinterpret_cast<uint4 *>(base + kmajor_offset(row, 8 * k8, kbytes, 2)) = u;
}

struct Ctl {
    uint64_t *mbar;
    uint32_t phase;
    bool ok;
    // waits for the last commit; all threads agree on the outcome
    __device__ __forceinline__ bool wait() {
        const bool w = mbar_wait(mbar, phase, kWait);
        phase ^= 1u;
        if (__syncthreads_or(!w)) {
            ok = false;
            return false;
        }
        fence_after();
        return true;
    }
};

// operand writes by all threads -> visible to the MMA issued by thread 0
__device__ __forceinline__ void publish() {
    fence_before();
    fence_async_smem();
    __syncthreads();
    fence_after();
}

template <int G, int NF>
__device__ __forceinline__ void tc_group(const dbwd::Args &a, const Layout &L, unsigned char *smem, uint32_t sbase,
                                         uint32_t tmem, uint32_t lane, Ctl &ctl, int an, bool valid, size_t gbase,
                                         int lr, float dls[3]) {
    constexpr int M = G == 0 ? 1 : G == 1 ? 7 : G == 2 ? 3 : NF;
    constexpr int NNL = nl_comps(G);
    constexpr int MP = mp_of(G, NF);
    constexpr int KC = kc_of(G, NF);
    constexpr int NCH = (16 + KC - 1) / KC;  // chunks for K = 16
    constexpr int UNR = G < 3 ? NCH : 1;
    constexpr int NPUT = (KC * MP + 7) / 8;  // 16-byte stores per chunk row
    const int tid = threadIdx.x;
    const int K = a.K;
    const bool want_mlp = a.s.X != nullptr && valid;
    const int ld = a.s.ld;
    const float *b1 = reinterpret_cast<const float *>(smem + L.ob1);
    const float *b2nl = reinterpret_cast<const float *>(smem + L.ob2nl);
    // ---- H_g = act(Z_g + b1) from the Z columns of this group
    unsigned relu_on = 0;
    float hs[kH];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float z[16];
        tmem_ld16(lane + cZ + G * kH + 16 * half, z);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int jj = 16 * half + j;
            const float zz = z[j] + b1[G * kH + jj];
            if (G < 3) {
                relu_on |= (zz > 0.f ? 1u : 0u) << jj;
                hs[jj] = fmaxf(zz, 0.f);
            } else {
                hs[jj] = softplus(zz);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) put8(smem + L.oH, tid, q, kH * 2, hs + 8 * q);
    if (want_mlp)
#pragma unroll
        for (int j = 0; j < kH; ++j) a.s.H[(size_t)(G * kH + j) * ld + lr] = hs[j];
    publish();
    // ---- Y of the nonlinear outputs (columns 16 c + k)
    float ynl[NNL > 0 ? NNL : 1][16];
    if (NNL > 0) {
        if (tid == 0) {
            mma_chain(tmem + cY, sbase + L.oH, kH * 2, sbase + L.oW2nl + nl_base(G) * kH * 2, kH * 2, kH * 2 / 32,
                      idesc(kBF16, kRows, 16 * (NNL > 0 ? NNL : 1)), false);
            commit(ctl.mbar);
        }
        if (!ctl.wait()) return;
#pragma unroll
        for (int c = 0; c < NNL; ++c) {
            tmem_ld16(lane + cY + 16 * c, ynl[c]);
#pragma unroll
            for (int k = 0; k < 16; ++k) ynl[c][k] += b2nl[nl_base(G) + 16 * c + k];
        }
    }
    // ---- DY in chunks of KC Gaussians (all components); DH (+)= DY W2_g
    const int r0 = dbwd::grp_r0(G, K);
#pragma unroll UNR
    for (int ch = 0; ch < NCH; ++ch) {
        const int k0 = ch * KC;
        if (k0 >= K) break;
        float dyv[KC * MP > 0 ? KC * MP : 1];
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            const int k = k0 + kk;  // compile-time wherever ynl is indexed (G < 3)
            const bool live = k < K && valid;
            const size_t gi = gbase + (live ? k : 0);
            if (G == 0) {
                float dy = 0.f;
                if (live) {
                    if (a.op_tanh) {
                        const float t = tanhf(ynl[0][k & 15]);
                        dy = a.d_mean_op[gi].w * (1.f - t * t);
                    } else {
                        const float o = sig(ynl[0][k & 15]);
                        dy = a.d_mean_op[gi].w * o * (1.f - o);
                    }
                }
                dyv[kk] = dy;
            } else if (G == 1) {
                const float4 ds = live ? a.d_scale[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 dq = live ? a.d_quat[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float dsc[3] = {ds.x, ds.y, ds.z};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float s = sig(ynl[c < NNL ? c : 0][k & 15]);
                    dyv[kk * MP + c] = live ? dsc[c] * a.ascale[3 * an + c] * s * (1.f - s) : 0.f;
                    dls[c] += live ? dsc[c] * s : 0.f;
                }
                dyv[kk * MP + 3] = dq.x;
                dyv[kk * MP + 4] = dq.y;
                dyv[kk * MP + 5] = dq.z;
                dyv[kk * MP + 6] = dq.w;
                dyv[kk * MP + 7] = 0.f;
            } else if (G == 2) {
                const float4 dc = live ? a.d_color[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float dcc[3] = {dc.x, dc.y, dc.z};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float s = sig(ynl[c < NNL ? c : 0][k & 15]);
                    dyv[kk * MP + c] = dcc[c] * s * (1.f - s);
                }
                dyv[kk * MP + 3] = 0.f;
            } else {
#pragma unroll
                for (int q = 0; q < NF / 4; ++q) {
                    const float4 f = live ? reinterpret_cast<const float4 *>(a.d_feat + gi * NF)[q]
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
                    dyv[kk * MP + 4 * q] = f.x;
                    dyv[kk * MP + 4 * q + 1] = f.y;
                    dyv[kk * MP + 4 * q + 2] = f.z;
                    dyv[kk * MP + 4 * q + 3] = f.w;
                }
            }
            if (want_mlp && k < K)
#pragma unroll
                for (int c = 0; c < M; ++c) a.s.DY[(size_t)(r0 + M * k + c) * ld + lr] = dyv[kk * MP + c];
        }
#pragma unroll
        for (int q = 0; q < NPUT; ++q) put8(smem + L.oDY, tid, q, 64 * 2, dyv + 8 * q);
        publish();
        if (tid == 0) {
            const int steps = (min(KC, K - k0) * MP + 15) / 16;
            mma_chain(tmem + cDH, sbase + L.oDY, 64 * 2, sbase + L.oW2T[G] + (uint32_t)(k0 * MP * 2 / 16) * 128u,
                      L.eW2T[G] * 2, steps, idesc(kBF16, kRows, kH), ch > 0);
            commit(ctl.mbar);
        }
        if (!ctl.wait()) return;
    }
    // ---- DZ = DH * act'(Z): ReLU -> mask; SoftPlus -> sigmoid(Z) = 1 - exp(-H)
    float dz[kH];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float dh[16];
        tmem_ld16(lane + cDH + 16 * half, dh);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int jj = 16 * half + j;
            const float d = dh[j] * (G < 3 ? (float)((relu_on >> jj) & 1u) : -expm1f(-hs[jj]));
            dz[jj] = valid ? d : 0.f;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) put8(smem + L.oDZ, tid, q, kH * 2, dz + 8 * q);
    if (want_mlp)
#pragma unroll
        for (int j = 0; j < kH; ++j) a.s.DZ[(size_t)(G * kH + j) * ld + lr] = dz[j];
    publish();
    // ---- DX += DZ_g W1_g  (B = W1^T at K offset 32 g)
    if (tid == 0) {
        mma_chain(tmem + cDX, sbase + L.oDZ, kH * 2, sbase + L.oW1T + 512u * G, 128 * 2, kH * 2 / 32,
                  idesc(kBF16, kRows, kKin), G > 0);
        commit(ctl.mbar);
    }
    ctl.wait();
}

template <int NF>
__global__ void __launch_bounds__(kRows, 2) k_decode_bwd_rows_tc(ViewTable vt, dbwd::Args a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ float aPose[3 * UPS_MAX_VIEWS];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int K = a.K, V = vt.n;
    const Layout L = rows_layout(NF, K);
    // ---- weights as B operands (K-major BF16)
    for (int i = tid; i < 128 * kKin; i += kRows) {
        const int h = i / kKin, c = i - h * kKin;
        put(smem + L.oW1, h, c, kKin * 2, c < kDin ? a.w1[h * kDin + c] : 0.f);
    }
    for (int i = tid; i < kKin * 128; i += kRows) {  // W1T[i][h] = W1[h][i]
        const int ii = i / 128, h = i - ii * 128;
        put(smem + L.oW1T, ii, h, 128 * 2, ii < kDin ? a.w1[h * kDin + ii] : 0.f);
    }
    float *b1 = reinterpret_cast<float *>(smem + L.ob1);
    float *b2nl = reinterpret_cast<float *>(smem + L.ob2nl);
    for (int i = tid; i < 112 * kH; i += kRows) {
        const int rr = i / kH, j = i - rr * kH;
        const int g = rr < 16 ? 0 : rr < 64 ? 1 : 2;
        const int c = (rr - nl_base(g)) >> 4, k = (rr - nl_base(g)) & 15;
        float w = 0.f, bb = 0.f;
        if (k < K) {
            const int orow = dbwd::grp_r0(g, K) + dbwd::grp_m(g, NF) * k + c;
            w = a.w2[orow * kH + j];
            bb = a.b2[orow];
        }
        put(smem + L.oW2nl, rr, j, kH * 2, w);
        if (j == 0) b2nl[rr] = bb;
    }
    for (int g = 0; g < 4; ++g) {
        const int m = dbwd::grp_m(g, NF), mp = mp_of(g, NF), E = L.eW2T[g];
        for (int i = tid; i < kH * E; i += kRows) {  // W2T_g[j][k mp + c] = W2[r0 + m k + c][j]
            const int j = i / E, e = i - j * E, k = e / mp, c = e - k * mp;
            const float w = (k < K && c < m) ? a.w2[(dbwd::grp_r0(g, K) + m * k + c) * kH + j] : 0.f;
            put(smem + L.oW2T[g], j, e, E * 2, w);
        }
    }
    for (int i = tid; i < 128; i += kRows) b1[i] = a.b1[i];
    for (int i = tid; i < 3 * V; i += kRows) aPose[i] = 0.f;
    if (tid == 0) mbar_init(&mbar, 1);
    if (warp == 0) tmem_alloc(&tmem_base, kTmemCols);
    publish();
    const uint32_t tmem = tmem_base;
    const uint32_t lane = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t sbase = smem_addr(smem);
    Ctl ctl{&mbar, 0u, true};
    const size_t NG = (size_t)a.A * K;
    for (int base = a.row_begin + blockIdx.x * kRows; base < a.row_end && ctl.ok; base += gridDim.x * kRows) {
        const int row = base + tid;
        const bool valid = row < a.row_end;
        const int an = valid ? row / V : 0, v = valid ? row - an * V : 0;
        const int lr = row - a.row_begin;
        const DevView &cam = vt.v[v];
        const size_t gbase = (size_t)v * NG + (size_t)an * K;
        float delta[3], dist;
        {
            float x[kKin];
            dbwd::mlp_input(a, cam, an, x, delta, dist);
            if (a.s.X && valid)
#pragma unroll
                for (int i = 0; i < kXW; ++i) a.s.X[(size_t)i * a.s.ld + lr] = x[i];
#pragma unroll
            for (int i = 0; i < kKin; ++i) x[i] = (valid && i < kDin) ? x[i] : 0.f;
#pragma unroll
            for (int q = 0; q < kKin / 8; ++q) put8(smem + L.oX, tid, q, kKin * 2, x + 8 * q);
        }
        publish();
        // ---- Z of all four groups: X W1^T (N = 128)
        if (tid == 0) {
            mma_chain(tmem + cZ, sbase + L.oX, kKin * 2, sbase + L.oW1, kKin * 2, kKin * 2 / 32,
                      idesc(kBF16, kRows, 128), false);
            commit(&mbar);
        }
        if (!ctl.wait()) break;
        float dls[3] = {0.f, 0.f, 0.f};
        tc_group<0, NF>(a, L, smem, sbase, tmem, lane, ctl, an, valid, gbase, lr, dls);
        if (ctl.ok) tc_group<1, NF>(a, L, smem, sbase, tmem, lane, ctl, an, valid, gbase, lr, dls);
        if (ctl.ok) tc_group<2, NF>(a, L, smem, sbase, tmem, lane, ctl, an, valid, gbase, lr, dls);
        if (NF > 0 && ctl.ok) tc_group<3, NF>(a, L, smem, sbase, tmem, lane, ctl, an, valid, gbase, lr, dls);
        if (!ctl.ok) break;
        float dx[48];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            float t16[16];
            tmem_ld16(lane + cDX + 16 * q, t16);
#pragma unroll
            for (int i = 0; i < 16; ++i) dx[16 * q + i] = t16[i];
        }
        fence_before();
        dbwd::row_epilogue(a, valid ? an : -1, v, gbase, dx, delta, dist, dls, aPose);
        __syncthreads();
        fence_after();
    }
    if (!ctl.ok) {
        // a wait ran out: record it and give the outstanding MMA a bounded
        // chance to land before TMEM is released
        if (tid == 0) {
            atomicExch(a.err, 1);
            mbar_wait(&mbar, ctl.phase ^ 1u, kWait);
        }
    } else {
        __syncthreads();
        dbwd::flush_pose(a, vt, aPose);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// weight gradients
// ---------------------------------------------------------------------------

constexpr int kWR = 32;   // rows per staged chunk

// Staged feature index space: DY of group g at goff[g] (group sizes padded to
// 8), H at fH, DZ at fH + 128, X at fH + 256; each feature holds the chunk's
// 32 rows, float4 q at slot q ^ key(f) to spread shared-memory banks.
struct WLayout {
    int goff[4], gn[4], gr0[4], fH, F;
};

__host__ __device__ inline WLayout wlayout(int K, int NF) {
    WLayout w{};
    int o = 0;
    for (int g = 0; g < 4; ++g) {
        w.goff[g] = o;
        w.gn[g] = K * dbwd::grp_m(g, NF);
        w.gr0[g] = dbwd::grp_r0(g, K);
        o += (w.gn[g] + 7) & ~7;
    }
    w.fH = o;
    w.F = o + 128 + 128 + kXW;
    return w;
}

__device__ __forceinline__ int swz(int f, int q) { return q ^ ((f ^ (f >> 3)) & 7); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes));
}

struct WArgs {
    int nrows, K, NF;
    dbwd::Scratch s;
    float *g_w1, *g_b1, *g_w2, *g_b2;
};

// Micro-tile t: A features [fa, fa+4), B features [fb, fb+8); kind 0 = dW2
// (A = DY, B = H of the group), kind 1 = dW1 (A = DZ, B = X).
struct MT {
    int fa, fb, kind, g, o0, cb;
};

__device__ __forceinline__ MT mt_of(const WLayout &w, int t) {
    MT m{};
    if (t < w.fH) {
        int g = 0;
        while (g < 3 && t >= w.goff[g + 1]) ++g;
        const int l = t - w.goff[g], ob = l >> 2, cb = l & 3;
        m.kind = 0;
        m.g = g;
        m.o0 = 4 * ob;
        m.cb = cb;
        m.fa = w.goff[g] + 4 * ob;
        m.fb = w.fH + g * kH + 8 * cb;
    } else {
        const int l = t - w.fH, hb = l / 5, ib = l - hb * 5;
        m.kind = 1;
        m.o0 = 4 * hb;
        m.cb = ib;
        m.fa = w.fH + 128 + 4 * hb;
        m.fb = w.fH + 256 + 8 * ib;
    }
    return m;
}

// Issues the cp.async copies of local rows [r0, r0 + 32) of every feature
// (rows at or past nrows and group padding are zero-filled).
__device__ __forceinline__ void stage_chunk(const WArgs &wa, const WLayout &w, const int *tbl, float *buf, int r0) {
    const int n4 = w.F * (kWR / 4);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        const int f = i >> 3, q = i & 7;
        const int r = tbl[f];
        const int row = r0 + 4 * q;
        const int nb = r >= 0 ? 4 * max(0, min(4, wa.nrows - row)) : 0;
        // a valid address even when nothing is copied (zero fill)
        const float *src = wa.s.X + (nb > 0 ? (size_t)r * wa.s.ld + row : 0);
        cp_async16(buf + f * kWR + 4 * swz(f, q), src, nb);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// staged feature f -> its row in the scratch (X, H, DY, DZ are one buffer
// starting at X), -1 for group padding
__device__ __forceinline__ void build_table(const WArgs &wa, const WLayout &w, int *tbl) {
    const int n_out = dbwd::n_out(wa.K, wa.NF);
    for (int f = threadIdx.x; f < w.F; f += blockDim.x) {
        int r;
        if (f < w.fH) {
            int g = 0;
            while (g < 3 && f >= w.goff[g + 1]) ++g;
            const int l = f - w.goff[g];
            r = l < w.gn[g] ? kXW + 128 + w.gr0[g] + l : -1;
        } else if (f < w.fH + 128) {
            r = kXW + (f - w.fH);
        } else if (f < w.fH + 256) {
            r = kXW + 128 + n_out + (f - w.fH - 128);
        } else {
            r = f - w.fH - 256;
        }
        tbl[f] = r;
    }
}

template <int U, int kWT>
__global__ void __launch_bounds__(kWT) k_decode_wgrad(WArgs wa, int double_buffer) {
    extern __shared__ float4 ws4[];
    float *ws = reinterpret_cast<float *>(ws4);
    const WLayout w = wlayout(wa.K, wa.NF);
    const int n_mt = w.fH + 160;
    float *buf[2] = {ws, ws + (double_buffer ? w.F * kWR : 0)};
    int *tbl = reinterpret_cast<int *>(ws + (double_buffer ? 2 : 1) * w.F * kWR);
    build_table(wa, w, tbl);
    __syncthreads();
    float acc[U][4][8];
    int fa[U], fb[U];  // micro-tile operand features (the rest is recomputed at the flush)
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const MT m = mt_of(w, threadIdx.x + u * kWT);
        fa[u] = m.fa;
        fb[u] = m.fb;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[u][i][j] = 0.f;
    }
    // db2: thread t sums staged DY features t and t + kWT (group padding
    // included, as zeros)
    float bsum[2] = {0.f, 0.f};
    const int nchunks = (wa.nrows + kWR - 1) / kWR;
    auto compute = [&](const float *sb) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int fb = threadIdx.x + b * kWT;
            if (fb < w.fH) {
                float t = 0.f;
#pragma unroll
                for (int q = 0; q < kWR / 4; ++q) {
                    const float4 d = *reinterpret_cast<const float4 *>(sb + fb * kWR + 4 * swz(fb, q));
                    t += (d.x + d.y) + (d.z + d.w);
                }
                bsum[b] += t;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (threadIdx.x + u * kWT >= n_mt) continue;
            const int ma = fa[u], mb = fb[u];
#pragma unroll 1
            for (int q = 0; q < kWR / 4; ++q) {
                float4 av[4], bv[8];
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    av[i] = *reinterpret_cast<const float4 *>(sb + (ma + i) * kWR + 4 * swz(ma + i, q));
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    bv[j] = *reinterpret_cast<const float4 *>(sb + (mb + j) * kWR + 4 * swz(mb + j, q));
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float t = acc[u][i][j];
                        t = fmaf(av[i].x, bv[j].x, t);
                        t = fmaf(av[i].y, bv[j].y, t);
                        t = fmaf(av[i].z, bv[j].z, t);
                        t = fmaf(av[i].w, bv[j].w, t);
                        acc[u][i][j] = t;
                    }
            }
        }
    };
    if (double_buffer) {
        int ch = blockIdx.x;
        if (ch < nchunks) stage_chunk(wa, w, tbl, buf[0], ch * kWR);
        for (int it = 0; ch < nchunks; ch += gridDim.x, ++it) {
            const int nxt = ch + gridDim.x;
            if (nxt < nchunks) {
                stage_chunk(wa, w, tbl, buf[(it + 1) & 1], nxt * kWR);
                asm volatile("cp.async.wait_group 1;" ::: "memory");
            } else {
                asm volatile("cp.async.wait_group 0;" ::: "memory");
            }
            __syncthreads();
            compute(buf[it & 1]);
            __syncthreads();
        }
    } else {
        for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
            stage_chunk(wa, w, tbl, buf[0], ch * kWR);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();
            compute(buf[0]);
            __syncthreads();
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (threadIdx.x + u * kWT >= n_mt) continue;
        const MT m = mt_of(w, threadIdx.x + u * kWT);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (m.kind == 0) {
                const int o = m.o0 + i;
                if (o >= w.gn[m.g]) continue;
                const int orow = w.gr0[m.g] + o;
#pragma unroll
                for (int j = 0; j < 8; ++j) atomicAdd(wa.g_w2 + (size_t)orow * kH + 8 * m.cb + j, acc[u][i][j]);
            } else {
                const int h = m.o0 + i;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = 8 * m.cb + j;
                    if (c < kDin)
                        atomicAdd(wa.g_w1 + h * kDin + c, acc[u][i][j]);
                    else if (c == kDin)
                        atomicAdd(wa.g_b1 + h, acc[u][i][j]);
                }
            }
        }
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int fb = threadIdx.x + b * kWT;
        if (fb >= w.fH) continue;
        int g = 0;
        while (g < 3 && fb >= w.goff[g + 1]) ++g;
        const int o = fb - w.goff[g];
        if (o < w.gn[g]) atomicAdd(wa.g_b2 + w.gr0[g] + o, bsum[b]);
    }
}

// one staged chunk of rows (the kernel double-buffers when two fit)
size_t wgrad_chunk_smem(int K, int NF) { return sizeof(float) * (size_t)wlayout(K, NF).F * kWR; }

cudaError_t launch_decode_wgrad(const WArgs &wa, int num_sms, cudaStream_t st) {
    const WLayout w = wlayout(wa.K, wa.NF);
    const size_t one = wgrad_chunk_smem(wa.K, wa.NF), tbl = sizeof(int) * (size_t)w.F;
    const int db = 2 * one + tbl <= 227 * 1024 ? 1 : 0;
    const size_t smem = (db ? 2 * one : one) + tbl;
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    const int n_mt = w.fH + 160;
    const int chunks = (wa.nrows + kWR - 1) / kWR;
    const int blocks = std::max(1, std::min(chunks, num_sms));
#define UPS_WG(U, T)                                                                                   \
    do {                                                                                               \
        cudaFuncSetAttribute(k_decode_wgrad<U, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k_decode_wgrad<U, T><<<blocks, T, smem, st>>>(wa, db);                                         \
    } while (0)
    if (n_mt <= 512 && w.fH <= 1024)
        UPS_WG(1, 512);
    else if (n_mt <= 3 * 256 && w.fH <= 512)
        UPS_WG(3, 256);
    else
        return cudaErrorInvalidConfiguration;
#undef UPS_WG
    return cudaGetLastError();
}

// rows per scratch chunk of the decode backward
constexpr int kChunkRows = 1 << 18;

}  // namespace

size_t decode_bwd_rows_tc_smem(int NF, int K) { return (size_t)rows_layout(NF, K).total; }

// tcgen05 per-row kernel: resident CTAs per SM by shared memory
static int rows_tc_per_sm(int NF, int K) {
    const size_t smem = (size_t)rows_layout(NF, K).total;
    return (smem + 2048) * 2 <= 228 * 1024 ? 2 : 1;
}

int decode_bwd_rows_wave(int bf16, int K, int NF, int num_sms) {
    if (bf16) return std::max(1, num_sms) * rows_tc_per_sm(NF, K) * dbwd::kRowsPerBlock;
    return std::max(1, num_sms) * dbwd::kRowsCtasPerSm * dbwd::kRowsFp32;
}

cudaError_t launch_decode_bwd_rows_tc(const ViewTable &vt, const dbwd::Args &a, int num_sms, cudaStream_t st) {
    const size_t smem = (size_t)rows_layout(a.NF, a.K).total;
    if (smem + 1024 > 227 * 1024) return cudaErrorInvalidConfiguration;
    const int rows = a.row_end - a.row_begin;
    const int per_sm = rows_tc_per_sm(a.NF, a.K);
    const int blocks = std::max(1, std::min((rows + kRows - 1) / kRows, num_sms * per_sm));
#define UPS_BT(NFV)                                                                              \
    do {                                                                                         \
        cudaFuncSetAttribute(k_decode_bwd_rows_tc<NFV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                         \
        k_decode_bwd_rows_tc<NFV><<<blocks, kRows, smem, st>>>(vt, a);                           \
    } while (0)
    switch (a.NF) {
        case 0: UPS_BT(0); break;
        case 16: UPS_BT(16); break;
        case 32: UPS_BT(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef UPS_BT
    return cudaGetLastError();
}

// Scratch bytes the decode backward needs (MLP gradients only).
size_t decode_bwd_scratch_bytes(int A, int V, int K, int NF) {
    const int rows = std::min(A * V, kChunkRows);
    const int ld = (rows + 31) & ~31;
    return sizeof(float) * dbwd::scratch_floats(ld, dbwd::n_out(K, NF));
}

// Whether K and n_feat fit the backward kernels' shared memory and tiling.
bool decode_bwd_fits(int K, int NF) {
    return rows_layout(NF, K).total + 1024 <= 227 * 1024 &&
           wgrad_chunk_smem(K, NF) + sizeof(int) * wlayout(K, NF).F <= 227 * 1024 &&
           wlayout(K, NF).fH + 160 <= 3 * 256;
}

cudaError_t launch_decode_bwd(const ViewTable &vt, int A, int K, int NF, const ups_anchors &anc,
                              const ups_mlp &mlp, const ups_gaussians &dG, unsigned mask, const ups_mlp *d_mlp,
                              const ups_anchors *d_anc, float *d_pose, int bf16, int op_tanh, float *scratch,
                              int *err, int num_sms, const dbwd::StageHook &hook, cudaStream_t st) {
    dbwd::Args a{};
    a.op_tanh = op_tanh;
    a.A = A;
    a.K = K;
    a.NF = NF;
    a.pos = anc.pos;
    a.afeat = anc.feat;
    a.offs = anc.offsets;
    a.ascale = anc.scaling;
    a.w1 = mlp.w1;
    a.b1 = mlp.b1;
    a.w2 = mlp.w2;
    a.b2 = mlp.b2;
    a.d_mean_op = reinterpret_cast<const float4 *>(dG.mean_opacity);
    a.d_scale = reinterpret_cast<const float4 *>(dG.scale);
    a.d_quat = reinterpret_cast<const float4 *>(dG.quat);
    a.d_color = reinterpret_cast<const float4 *>(dG.color);
    a.d_feat = dG.feat;
    if (d_anc) {
        a.g_pos = d_anc->pos;
        a.g_afeat = d_anc->feat;
        a.g_offs = d_anc->offsets;
        a.g_ascale = d_anc->scaling;
    }
    a.g_pose = d_pose;
    a.mask = mask;
    a.err = err;
    const bool want_mlp = (mask & UPS_GRAD_MLP) && d_mlp;
    const int rows = A * vt.n;
    // chunks of whole passes of the per-row kernel's resident grid (a chunk of
    // 4.5 passes costs 5 on its slowest CTAs), at most kChunkRows rows
    const int wave = decode_bwd_rows_wave(bf16, K, NF, num_sms);
    int chunk = std::min(rows, kChunkRows);
    if (rows > kChunkRows && wave <= kChunkRows) chunk = (kChunkRows / wave) * wave;
    const int ld = (chunk + 31) & ~31;
    if (want_mlp) a.s = dbwd::scratch_at(scratch, ld, dbwd::n_out(K, NF));
    for (int r = 0; r < rows; r += chunk) {
        a.row_begin = r;
        a.row_end = std::min(rows, r + chunk);
        hook.fn(hook.user, "decode_bwd_rows", true, st);
        cudaError_t e = bf16 ? launch_decode_bwd_rows_tc(vt, a, num_sms, st)
                             : launch_decode_bwd_rows_fp32(vt, a, num_sms, st);
        hook.fn(hook.user, "decode_bwd_rows", false, st);
        if (e != cudaSuccess) return e;
        if (!want_mlp) continue;
        hook.fn(hook.user, "decode_wgrad", true, st);
        if (decode_wgrad_tc_fits(K, NF)) {
            e = launch_decode_wgrad_tc(scratch, ld, a.row_end - a.row_begin, K, NF, *d_mlp, err, num_sms, st);
        } else {
            WArgs wa{a.row_end - a.row_begin, K, NF, a.s, d_mlp->w1, d_mlp->b1, d_mlp->w2, d_mlp->b2};
            e = launch_decode_wgrad(wa, num_sms, st);
        }
        hook.fn(hook.user, "decode_wgrad", false, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ups
