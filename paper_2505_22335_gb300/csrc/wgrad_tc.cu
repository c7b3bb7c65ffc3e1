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
// of one narrow MMA per (output tile, group).  The B operands' padding rows
// (DY past n_out, X past 40) hold whatever features follow in the scratch;
// they only reach D columns that are not read.
//
// Each operand value x is split into hi = tf32(x) and lo = tf32(x - hi); the
// products hi*hi + hi*lo + lo*hi recover FP32 accuracy (the dropped lo*lo term
// is about 2^-22 relative), with FP32 accumulation in TMEM.
//
// A chunk's operands arrive by tiled TMA loads with 64-byte swizzle (one box
// of 16 rows x up to 256 features per operand region), already in the K-major
// layout the MMAs read; rows past the launch's end read as zero.
// Warp roles (one CTA per SM, persistent over chunks): warp 16 issues a
// chunk's loads into a free stage (waiting on the stage's `empty` barrier,
// completing on `loaded`); warps 0-14 wait for `loaded`, split each value in
// place (hi) and into the stage's lo tile set, then arrive on `full`; warp 15
// waits for `full`, issues the MMAs and commits them to `empty`.  Three
// stages (two for the widest outputs): the loads of the next chunks are in
// flight while one chunk is split and multiplied.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "decode_bwd.cuh"
#include "umma.cuh"

namespace ups {

namespace {

using namespace umma;
using dbwd::kDin;
using dbwd::kH;
using dbwd::kXW;

// 15 converter warps + the MMA warp + the load warp
constexpr int kConv = 480;            // converter threads (warps 0-14)
constexpr int kMmaTid = kConv;        // lane 0 of warp 15
constexpr int kLoadTid = kConv + 32;  // lane 0 of warp 16
constexpr int kT = kConv + 64;
constexpr int kKR = 16;               // rows per chunk (2 TF32 K steps)
constexpr int kRowBytes = kKR * 4;    // bytes of one operand row per chunk (one swizzle row)
constexpr int kNX = 48;               // X operand rows (40 + padding)
constexpr int kDyBox = 256;           // DY operand rows per load and MMA (the last may be narrower)
constexpr int kMaxNB = 464;           // DY operand rows: D_w2 + D_w1 <= 512 TMEM columns
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxStages = 3;
constexpr int kMaxItems = 7;          // float4 items per converter thread and chunk
constexpr int kWait = 1 << 22;

// One chunk's operand tile set (bytes; every region 512-byte aligned).
struct WLay {
    int n_out;
    int ndy, wlast, nb;             // DY: ndy boxes, the last wlast rows wide; nb rows in all
    int oA_h, oB_dy, oA_dz, oB_x;   // region offsets
    int block_bytes;                // bytes the loads of one chunk bring
    int set_bytes;                  // block_bytes rounded up to 1 KB
    int stages;                     // 3, or 2 where three do not fit
};

__host__ __device__ inline WLay wlay(int K, int NF) {
    WLay w{};
    w.n_out = dbwd::n_out(K, NF);
    w.ndy = (w.n_out + kDyBox - 1) / kDyBox;
    w.wlast = ((w.n_out - kDyBox * (w.ndy - 1)) + 15) & ~15;
    w.nb = kDyBox * (w.ndy - 1) + w.wlast;
    w.oA_h = 0;
    w.oB_dy = 128 * kRowBytes;
    w.oA_dz = w.oB_dy + w.nb * kRowBytes;
    w.oB_x = w.oA_dz + 128 * kRowBytes;
    w.block_bytes = w.oB_x + kNX * kRowBytes;
    w.set_bytes = (w.block_bytes + 1023) & ~1023;
    w.stages = 2 * w.set_bytes * 3 + 1024 <= 227 * 1024 ? 3 : 2;
    return w;
}

__host__ __device__ inline bool wlay_ok(const WLay &w) {
    return w.nb <= kMaxNB && 2 * w.set_bytes * w.stages + 1024 <= 227 * 1024 &&
           w.block_bytes / 16 <= kMaxItems * kConv;
}

struct WTArgs {
    int nrows, K, NF;
    float *g_w1, *g_b1, *g_w2, *g_b2;
    int *err;
};

// output index of the DY operand row holding the 16-byte item at byte offset
// `off` of a tile set (-1: not in the DY region)
__device__ __forceinline__ int dy_output_at(const WLay &w, int off) {
    if (off < w.oB_dy || off >= w.oA_dz) return -1;
    return (off - w.oB_dy) / kRowBytes;  // DY boxes are adjacent: row o of box j is output 256 j + o
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

// Tensor maps over the scratch (rows x features, 64-byte swizzle): boxes of
// 16 rows x 48 (X), 128 (H, DZ), 256 and the last width (DY) features.
struct WMaps {
    CUtensorMap x, h, dy, dy_last;
};

__global__ void __launch_bounds__(kT, 1) k_decode_wgrad_tc(const __grid_constant__ WMaps maps, WTArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t loaded[kMaxStages], full[kMaxStages], empty[kMaxStages];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, n_issued, n_mma;
    // operand regions on 1 KB boundaries (the swizzle pattern repeats every 512 bytes)
    unsigned char *smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const WLay w = wlay(a.K, a.NF);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nchunks = (a.nrows + kKR - 1) / kKR;
    const int nmine = nchunks > (int)blockIdx.x ? (nchunks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int S = w.stages;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&loaded[s], 1);
            mbar_init(&full[s], kConv);
            mbar_init(&empty[s], 1);
        }
        abort_flag = 0;
        n_issued = 0;
        n_mma = 0;
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
        const int nitems = w.block_bytes / 16;
        float bs[kMaxItems];  // db2 partial sums of this thread's DY items
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k) bs[k] = 0.f;
        for (int it = 0; it < nmine; ++it) {
            const int s = it % S, use = it / S;
            if (!mbar_wait(&loaded[s], (uint32_t)(use & 1), kWait)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (*(volatile int *)&abort_flag) break;
            unsigned char *hi = smem + (size_t)s * 2 * w.set_bytes, *lo = hi + w.set_bytes;
#pragma unroll
            for (int k = 0; k < kMaxItems; ++k) {
                const int i = tid + kConv * k;
                if (i < nitems) {
                    const float4 v = *reinterpret_cast<const float4 *>(hi + 16 * i);
                    split_store(hi, lo, 16 * i, v);
                    bs[k] += (v.x + v.y) + (v.z + v.w);
                }
            }
            fence_async_smem();
            mbar_arrive(&full[s]);
        }
        // db2: the four 16-byte items of a DY operand row (64 bytes, its 16
        // rows of the chunk in some order) sit in lanes 4 l .. 4 l + 3
#pragma unroll
        for (int k = 0; k < kMaxItems; ++k) {
            float t = bs[k];
            t += __shfl_xor_sync(0xffffffffu, t, 1);
            t += __shfl_xor_sync(0xffffffffu, t, 2);
            const int i = tid + kConv * k;
            if (i < nitems && (i & 3) == 0 && nmine > 0) {
                const int o = dy_output_at(w, 16 * i);
                if (o >= 0 && o < w.n_out) atomicAdd(a.g_b2 + o, t);
            }
        }
    } else if (tid == kMmaTid) {
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
                    const uint32_t ka = 32u * ks;  // 8 TF32 values of K
                    for (int j = 0; j < w.ndy; ++j) {
                        const int n = j + 1 < w.ndy ? kDyBox : w.wlast;
                        mma<kTF32>(tmem + cW2 + kDyBox * j, desc_sw64(ab + w.oA_h + ka),
                                   desc_sw64(bb + w.oB_dy + kDyBox * kRowBytes * j + ka), idesc(kTF32, 128, n), acc);
                    }
                    mma<kTF32>(tmem + cW1, desc_sw64(ab + w.oA_dz + ka), desc_sw64(bb + w.oB_x + ka), id_w1, acc);
                }
            }
            commit(&empty[s]);
            n_mma = it + 1;
        }
    } else if (tid == kLoadTid) {
        // ---------------- tiled loads (one thread of warp 16)
        const int fH = kXW, fDY = kXW + 128, fDZ = kXW + 128 + w.n_out;  // first scratch feature of each region
        for (int it = 0; it < nmine; ++it) {
            const int s = it % S, use = it / S;
            if (use > 0 && !mbar_wait(&empty[s], (uint32_t)((use - 1) & 1), kWait)) {
                atomicExch(&abort_flag, 1);
                break;
            }
            if (*(volatile int *)&abort_flag) break;
            const int r0 = ((int)blockIdx.x + it * (int)gridDim.x) * kKR;
            unsigned char *hi = smem + (size_t)s * 2 * w.set_bytes;
            mbar_arrive_expect(&loaded[s], (uint32_t)w.block_bytes);
            tma_load_2d(hi + w.oB_x, &maps.x, r0, 0, &loaded[s]);
            tma_load_2d(hi + w.oA_h, &maps.h, r0, fH, &loaded[s]);
            for (int j = 0; j < w.ndy; ++j)
                tma_load_2d(hi + w.oB_dy + kDyBox * kRowBytes * j, j + 1 < w.ndy ? &maps.dy : &maps.dy_last, r0,
                            fDY + kDyBox * j, &loaded[s]);
            tma_load_2d(hi + w.oA_dz, &maps.h, r0, fDZ, &loaded[s]);
            n_issued = it + 1;
        }
    }
    __syncthreads();
    // Before the TMEM reads (and before exit): every issued load has landed
    // and every issued MMA has completed, each waited for (bounded) through
    // the last use of its stage.
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            if (s < n_issued) {
                const int last = (n_issued - 1 - s) / S;
                if (!mbar_wait(&loaded[s], (uint32_t)(last & 1), kWait)) abort_flag = 1;
            }
            if (s < n_mma) {
                const int last = (n_mma - 1 - s) / S;
                if (!mbar_wait(&empty[s], (uint32_t)(last & 1), kWait)) abort_flag = 1;
            }
        }
        if (n_mma < nmine) abort_flag = 1;
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

// the driver's tensor-map encoder, looked up once
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// rows x features view of the feature-major scratch (feature f of row r at
// [f * ld + r]); boxes of 16 rows x box_f features, 64-byte swizzle, rows
// past nrows and features past nfeat read as zero
bool make_map(CUtensorMap *m, const float *scratch, int ld, int nrows, int nfeat, int box_f) {
    const auto fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)nrows, (cuuint64_t)nfeat};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kKR, (cuuint32_t)box_f};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(scratch), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool decode_wgrad_tc_fits(int K, int NF) { return wlay_ok(wlay(K, NF)); }

cudaError_t launch_decode_wgrad_tc(const float *scratch, int ld, int nrows, int K, int NF, const ups_mlp &d_mlp,
                                   int *err, int num_sms, cudaStream_t st) {
    const WLay w = wlay(K, NF);
    if (!wlay_ok(w)) return cudaErrorInvalidConfiguration;
    if (nrows <= 0) return cudaSuccess;
    // TMA: 16-byte aligned base and row stride
    if ((reinterpret_cast<uintptr_t>(scratch) & 15) != 0 || (ld & 3) != 0 || ld < nrows)
        return cudaErrorInvalidValue;
    const int nfeat = kXW + 128 + w.n_out + 128;
    WMaps maps;
    if (!make_map(&maps.x, scratch, ld, nrows, nfeat, kNX) || !make_map(&maps.h, scratch, ld, nrows, nfeat, 128) ||
        !make_map(&maps.dy, scratch, ld, nrows, nfeat, kDyBox) ||
        !make_map(&maps.dy_last, scratch, ld, nrows, nfeat, w.wlast))
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * w.set_bytes * w.stages + 1024;
    WTArgs a{nrows, K, NF, d_mlp.w1, d_mlp.b1, d_mlp.w2, d_mlp.b2, err};
    const int chunks = (nrows + kKR - 1) / kKR;
    const int blocks = std::max(1, std::min(chunks, num_sms));
    cudaFuncSetAttribute(k_decode_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_decode_wgrad_tc<<<blocks, kT, smem, st>>>(maps, a);
    return cudaGetLastError();
}

}  // namespace ups
