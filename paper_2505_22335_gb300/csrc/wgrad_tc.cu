// Weight gradients of the decode MLPs (Eq. 8-9 differentiated) on the tcgen05
// tensor cores, FP32-accurate through split TF32 (3xTF32), summed over all
// rows (anchor, view) of the feature-major scratch that the per-row backward
// kernels write.  The reduction runs along rows, so rows are the MMA K
// dimension; a chunk of 16 rows is two K steps.
//
//   D_w2 [128 hidden x n_out] = H_all . DY^T     dW2[o][j] = D_w2[32 g(o) + j][o]
//   D_w1 [128 hidden x 48]    = DZ . X^T         dW1[h][i] = D_w1[h][i], db1 = column 38 (X row 38 = 1)
//   db2[o] = sum of DY[o] over rows (CUDA cores, while the operands are split)
// D_w2 keeps all four MLPs' hidden units as one M = 128 operand, so only the
// diagonal 32 x n_g blocks are used: fewer, wider MMAs (N up to 256) instead
// of one narrow MMA per (output tile, group).
//
// Each operand value x is split into hi = tf32(x) and lo = tf32(x - hi); the
// products hi*hi + hi*lo + lo*hi recover FP32 accuracy (the dropped lo*lo term
// is about 2^-22 relative), with FP32 accumulation in TMEM.
//
// Warp roles (one CTA per SM, persistent over chunks): warps 0-14 load a
// chunk's 16-row slice of every scratch feature (the next chunk's loads are
// in flight while the current one is split), split it and store hi and lo as
// canonical K-major no-swizzle operand tiles, then arrive on the stage's
// `full` mbarrier; warp 15 waits for `full`, issues the MMAs and commits them
// to the stage's `empty` mbarrier.  Three stages (two for the widest outputs).
#include <algorithm>

#include "decode_bwd.cuh"
#include "umma.cuh"

namespace ups {

namespace {

using namespace umma;
using dbwd::kDin;
using dbwd::kH;
using dbwd::kXW;

// 15 converter warps + the MMA warp: 512 threads at up to 128 registers
constexpr int kConv = 480;            // converter threads (warps 0-14)
constexpr int kT = kConv + 32;        // + the MMA warp
constexpr int kKR = 16;               // rows per chunk (2 TF32 K steps)
constexpr int kRowBytes = kKR * 4;    // bytes of one operand row per chunk
constexpr int kNX = 48;               // X operand rows (40 + zero padding)
constexpr int kMaxNB = 464;           // DY operand rows: D_w2 + D_w1 <= 512 TMEM columns
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxStages = 3;
constexpr int kMaxItems = 7;          // (feature, quad) items per converter thread
constexpr int kWait = 1 << 22;

struct WLay {
    int n_out, nb;       // DY rows, padded to 16 (MMA N granularity)
    int oA_h, oB_dy, oA_dz, oB_x, set_bytes;  // byte offsets in one (hi or lo) operand set
    int f_dz, f_h, f_x, f_end;  // item feature space: DY [0, nb), DZ, H, X (each a multiple of 8)
    int stages;                 // 3, or 2 where three do not fit
};

__host__ __device__ inline WLay wlay(int K, int NF) {
    WLay w{};
    w.n_out = dbwd::n_out(K, NF);
    w.nb = (w.n_out + 15) & ~15;
    int o = 0;
    w.oA_h = o;
    o += 128 * kRowBytes;
    w.oB_dy = o;
    o += w.nb * kRowBytes;
    w.oA_dz = o;
    o += 128 * kRowBytes;
    w.oB_x = o;
    o += kNX * kRowBytes;
    w.set_bytes = (o + 1023) & ~1023;
    w.f_dz = w.nb;
    w.f_h = w.f_dz + 128;
    w.f_x = w.f_h + 128;
    w.f_end = w.f_x + kXW;
    w.stages = 2 * w.set_bytes * 3 + 1024 <= 227 * 1024 ? 3 : 2;
    return w;
}

__host__ __device__ inline bool wlay_ok(const WLay &w) {
    return w.nb <= kMaxNB && 2 * w.set_bytes * w.stages + 1024 <= 227 * 1024 &&
           4 * w.f_end <= kMaxItems * kConv;
}

// byte offset of core-matrix row (operand row m, K quad q) in a K-major
// operand of 16 TF32 K elements per row
__device__ __forceinline__ int cm_off(int m, int q) { return ((m >> 3) * 4 + q) * 128 + (m & 7) * 16; }

struct WTArgs {
    int nrows, K, NF;
    const float *scratch;  // X [40][ld], H [128][ld], DY [n_out][ld], DZ [128][ld]
    int ld;
    float *g_w1, *g_b1, *g_w2, *g_b2;
    int *err;
};

// Item i of a chunk: feature f = 8 (i >> 5) + (i & 7), row quad q = (i >> 3) & 3,
// so the 8 lanes of a quarter warp store 8 different operand rows of one
// core-matrix column (all banks once) and a warp reads 8 features x 64 bytes.
__device__ __forceinline__ int item_feature(int i) { return 8 * (i >> 5) + (i & 7); }
__device__ __forceinline__ int item_quad(int i) { return (i >> 3) & 3; }

// scratch row of item feature f (-1: DY padding, nothing to load)
__device__ __forceinline__ int item_row(const WLay &w, int f) {
    if (f < w.f_dz) return f < w.n_out ? kXW + 128 + f : -1;  // DY
    if (f < w.f_h) return kXW + 128 + w.n_out + (f - w.f_dz);  // DZ
    if (f < w.f_x) return kXW + (f - w.f_h);                    // H
    return f - w.f_x;                                            // X
}

__device__ __forceinline__ int item_off(const WLay &w, int f, int q) {
    if (f < w.f_dz) return w.oB_dy + cm_off(f, q);
    if (f < w.f_h) return w.oA_dz + cm_off(f - w.f_dz, q);
    if (f < w.f_x) return w.oA_h + cm_off(f - w.f_h, q);
    return w.oB_x + cm_off(f - w.f_x, q);
}

__device__ __forceinline__ void split_store(unsigned char *hi, unsigned char *lo, int off, float4 v) {
    float4 h, l;
    h.x = tf32_hi(v.x);
    h.y = tf32_hi(v.y);
    h.z = tf32_hi(v.z);
    h.w = tf32_hi(v.w);
    l.x = tf32_hi(v.x - h.x);
    l.y = tf32_hi(v.y - h.y);
    l.z = tf32_hi(v.z - h.z);
    l.w = tf32_hi(v.w - h.w);
    *reinterpret_cast<float4 *>(hi + off) = h;
    *reinterpret_cast<float4 *>(lo + off) = l;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_addr(mbar)) : "memory");
}

// this converter thread's items of the chunk starting at row r0 (rows at or
// past nrows and DY padding read as zero)
__device__ __forceinline__ void load_items(const WTArgs &a, const WLay &w, int r0, float4 (&v)[kMaxItems]) {
    const int nitems = 4 * w.f_end;
#pragma unroll
    for (int k = 0; k < kMaxItems; ++k) {
        const int i = threadIdx.x + kConv * k;
        v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < nitems) {
            const int row = item_row(w, item_feature(i));
            if (row >= 0) {
                const float *src = a.scratch + (size_t)row * a.ld;
                const int rr = r0 + 4 * item_quad(i);
                if (rr + 4 <= a.nrows) {
                    v[k] = __ldg(reinterpret_cast<const float4 *>(src + rr));
                } else {
                    v[k].x = rr < a.nrows ? src[rr] : 0.f;
                    v[k].y = rr + 1 < a.nrows ? src[rr + 1] : 0.f;
                    v[k].z = rr + 2 < a.nrows ? src[rr + 2] : 0.f;
                    v[k].w = rr + 3 < a.nrows ? src[rr + 3] : 0.f;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kT, 1) k_decode_wgrad_tc(WTArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t full[kMaxStages], empty[kMaxStages];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const WLay w = wlay(a.K, a.NF);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nchunks = (a.nrows + kKR - 1) / kKR;
    const int nmine = nchunks > (int)blockIdx.x ? (nchunks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // zero the padding rows of every stage: DY rows [n_out, nb), X rows [40, 48)
    const int npad_dy = w.nb - w.n_out, npad = npad_dy + (kNX - kXW);
    const int S = w.stages;
    for (int s = 0; s < S; ++s)
        for (int i = tid; i < 4 * npad; i += kT) {
            const int r = i >> 2, q = i & 3;
            const int off = r < npad_dy ? w.oB_dy + cm_off(w.n_out + r, q) : w.oB_x + cm_off(kXW + r - npad_dy, q);
            unsigned char *hi = smem + (size_t)s * 2 * w.set_bytes;
            *reinterpret_cast<float4 *>(hi + off) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4 *>(hi + w.set_bytes + off) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], kConv);
            mbar_init(&empty[s], 1);
        }
        abort_flag = 0;
    }
    if (warp == 0) tmem_alloc(&tmem_base, kTmemCols);
    fence_before();
    fence_async_smem();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t cW2 = 0, cW1 = (uint32_t)w.nb;  // TMEM columns of D_w2, D_w1

    if (warp < kConv / 32) {
        // ---------------- converters
        const int nitems = 4 * w.f_end;
        float4 v[kMaxItems];
        float bs[kMaxItems];  // db2 partial sums of this thread's DY items
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k) bs[k] = 0.f;
        if (nmine > 0) load_items(a, w, (int)blockIdx.x * kKR, v);
        for (int it = 0; it < nmine; ++it) {
            const int s = it % S, use = it / S;
            if (use > 0 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1), kWait)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (*(volatile int *)&abort_flag) break;
            unsigned char *hi = smem + (size_t)s * 2 * w.set_bytes, *lo = hi + w.set_bytes;
#pragma unroll
            for (int k = 0; k < kMaxItems; ++k) {
                const int i = tid + kConv * k;
                if (i < nitems) {
                    const int f = item_feature(i);
                    if (f < w.n_out || f >= w.f_dz) split_store(hi, lo, item_off(w, f, item_quad(i)), v[k]);
                    if (f < w.f_dz) bs[k] += (v[k].x + v[k].y) + (v[k].z + v[k].w);
                }
            }
            fence_async_smem();
            mbar_arrive(&full[s]);
            if (it + 1 < nmine) load_items(a, w, ((int)blockIdx.x + (it + 1) * (int)gridDim.x) * kKR, v);
        }
        // db2: the four quads of a feature sit in lanes l, l + 8, l + 16, l + 24
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k) {
            float t = bs[k];
            t += __shfl_xor_sync(0xffffffffu, t, 8);
            t += __shfl_xor_sync(0xffffffffu, t, 16);
            const int i = tid + kConv * k;
            if (i < nitems && item_quad(i) == 0 && nmine > 0) {
                const int f = item_feature(i);
                if (f < w.n_out) atomicAdd(a.g_b2 + f, t);
            }
        }
    } else if (tid == kConv) {
        // ---------------- MMA issue (one thread of warp 15)
        const uint32_t id_w1 = idesc(kTF32, 128, kNX);
        for (int it = 0; it < nmine; ++it) {
            const int s = it % S, use = it / S;
            if (!mbar_wait(&full[s], (uint32_t)(use & 1), kWait)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            fence_after();
            const uint32_t hb = smem_addr(smem + (size_t)s * 2 * w.set_bytes), lb = hb + w.set_bytes;
            for (int pass = 0; pass < 3; ++pass) {
                // hi*hi, hi*lo, lo*hi
                const uint32_t ab = pass == 2 ? lb : hb, bb = pass == 1 ? lb : hb;
                for (int ks = 0; ks < 2; ++ks) {
                    const uint32_t acc = (it == 0 && pass == 0 && ks == 0) ? 0u : 1u;
                    const uint32_t ka = 256u * ks;
                    for (int n0 = 0; n0 < w.nb; n0 += 256) {
                        const int n = min(256, w.nb - n0);
                        mma<kTF32>(tmem + cW2 + n0, desc(ab + w.oA_h + ka, kRowBytes),
                                   desc(bb + w.oB_dy + n0 * kRowBytes + ka, kRowBytes), idesc(kTF32, 128, n), acc);
                    }
                    mma<kTF32>(tmem + cW1, desc(ab + w.oA_dz + ka, kRowBytes), desc(bb + w.oB_x + ka, kRowBytes),
                               id_w1, acc);
                }
            }
            commit(&empty[s]);
        }
    }
    __syncthreads();
    // all MMAs done: the last use of each stage completed
    if (tid == 0 && !abort_flag) {
        for (int s = 0; s < S && s < nmine; ++s) {
            const int last_use = (nmine - 1 - s) / S;
            if (!mbar_wait(&empty[s], (uint32_t)(last_use & 1), kWait)) {
                abort_flag = 1;
                break;
            }
        }
    }
    __syncthreads();
    fence_after();
    const bool ok = !abort_flag;
    if (ok && nmine > 0 && warp < 4) {
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        const int lane = tid & 31;
        // D_w2: warp g holds the hidden units of MLP g; its outputs are [r0, r0 + n)
        const int g = warp;
        const int r0 = dbwd::grp_r0(g, a.K), n = a.K * dbwd::grp_m(g, a.NF);
        for (int c0 = r0 & ~15; c0 < r0 + n; c0 += 16) {
            float d[16];
            tmem_ld16(lane_base + cW2 + c0, d);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int o = c0 + j;
                if (o >= r0 && o < r0 + n) atomicAdd(a.g_w2 + (size_t)o * kH + lane, d[j]);
            }
        }
        // D_w1: lane = hidden unit
        const int h = tid;
        for (int c0 = 0; c0 < kNX; c0 += 16) {
            float d[16];
            tmem_ld16(lane_base + cW1 + c0, d);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int i = c0 + j;
                if (i < kDin)
                    atomicAdd(a.g_w1 + h * kDin + i, d[j]);
                else if (i == kDin)
                    atomicAdd(a.g_b1 + h, d[j]);
            }
        }
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

bool decode_wgrad_tc_fits(int K, int NF) { return wlay_ok(wlay(K, NF)); }

cudaError_t launch_decode_wgrad_tc(const float *scratch, int ld, int nrows, int K, int NF, const ups_mlp &d_mlp,
                                   int *err, int num_sms, cudaStream_t st) {
    const WLay w = wlay(K, NF);
    if (!wlay_ok(w)) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)2 * w.set_bytes * w.stages;
    WTArgs a{nrows, K, NF, scratch, ld, d_mlp.w1, d_mlp.b1, d_mlp.w2, d_mlp.b2, err};
    const int chunks = (nrows + kKR - 1) / kKR;
    const int blocks = std::max(1, std::min(chunks, num_sms));
    cudaFuncSetAttribute(k_decode_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_decode_wgrad_tc<<<blocks, kT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ups
