// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/ups.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "ups.h"

namespace ups {

constexpr int kTile = 16;          // image tile edge (pixels)
constexpr int kTilePix = kTile * kTile;

// One view as the kernels see it (passed by value in kernel parameters).
struct DevView {
    float fx, fy, cx, cy;
    int W, H;
    int tiles_x, tiles_y;
    int tile_base;  // index of this view's tile 0 among all views' tiles
    int pix_off;    // P_v: pixel offset of this view in concatenated images
    float R[9];     // rotation of T_cw (row-major)
    float t[3];     // translation of T_cw
    float limx, limy;  // frustum guard on |X/Z|, |Y/Z|
    float t_norm;
    int set;        // the Gaussian set this view reads (attribute index set * n + g)
    int set_first;  // 1: the first view reading that set
};

struct ViewTable {
    int n;
    int total_tiles;
    DevView v[UPS_MAX_VIEWS];
};

struct BlendParams {
    float alpha_min, alpha_max, t_min, dilation, near_z;
};

// Per-Gaussian-view 2D gradient record (floats, 16-byte aligned groups):
//  0 du, 1 dv, 2 dz, 3 dopacity, 4 dconic_a, 5 dconic_b, 6 dconic_c, 7 pad,
//  8..10 dcolor, 11 pad, 12.. dfeat[n_feat]
constexpr int kG2Base = 12;
__host__ __device__ inline int g2_stride(int n_feat) { return kG2Base + n_feat; }

// View index of global tile `t` (views are few; linear scan).
__device__ __forceinline__ int view_of_tile(const ViewTable &vt, int t) {
    int v = 0;
    while (v + 1 < vt.n && vt.v[v + 1].tile_base <= t) ++v;
    return v;
}

// ---------------------------------------------------------------------------
// host-side helpers (implemented in ctx.cu)
// ---------------------------------------------------------------------------

// Packed pairs of f32 (first element in the low half) for fma.rn.f32x2: two
// channels per instruction, each rounded exactly as a scalar fmaf.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_make(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ void f2_split(f2 a, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}
__device__ __forceinline__ float f2_lo(f2 a) {
    float lo, hi;
    f2_split(a, lo, hi);
    (void)hi;
    return lo;
}
__device__ __forceinline__ float f2_hi(f2 a) {
    float lo, hi;
    f2_split(a, lo, hi);
    (void)lo;
    return hi;
}

// Device buffer that only grows.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t want);
    void release();
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// Radix sort of (key, value) pairs over bits [0, end_bit); stable.  Keys are
// uint32 or uint64, values uint32.  On return *key_io/*val_io point at the
// buffer (one of the two given) that holds the sorted data.
struct SortScratch {
    DevBuf hist;
};
size_t radix_hist_bytes(size_t n);
cudaError_t radix_sort_u32(uint32_t **key_io, uint32_t **key_alt, uint32_t **val_io,
                           uint32_t **val_alt, size_t n, int end_bit, SortScratch &s,
                           cudaStream_t st);
cudaError_t radix_sort_u64(uint64_t **key_io, uint64_t **key_alt, uint32_t **val_io,
                           uint32_t **val_alt, size_t n, int end_bit, SortScratch &s,
                           cudaStream_t st);
// One-pass stable sort of (key, value) pairs by keys < nbins <= kMaxBucketBins
// (tile ids).  Bucket d keeps its first min(count_d, cap) values (cap =
// kNoListCap: all; a finite cap needs cap <= kMaxListCap and nbins <
// kMaxBucketBins), written in key order to vals_out; ranges[d] is the kept
// [start, end) and bit d of trunc[(nbins + 31) / 32] is set when bucket d
// lost values to the cap.  scratch: bucket_sort_scratch_bytes.  gate (no
// cap only): when non-null the kernels do nothing unless *gate != 0.
constexpr int kMaxBucketBins = 1 << 14;
constexpr int kMaxListCap = 32767;
constexpr uint32_t kNoListCap = 0xffffffffu;
size_t bucket_sort_scratch_bytes(size_t n, int nbins, int num_sms);
cudaError_t bucket_sort_u32(const uint32_t *keys, const uint32_t *vals, uint32_t *vals_out, size_t n, int nbins,
                            uint32_t cap, uint2 *ranges, uint32_t *trunc, void *scratch, size_t scratch_bytes,
                            int num_sms, cudaStream_t st, const int *gate = nullptr);
// keys[i] = t for every i in ranges[t] (the sorted keys of a bucket sort)
cudaError_t keys_from_ranges(const uint2 *ranges, int nbins, uint32_t *keys, cudaStream_t st);
// C (column-major m x n, leading dimension ldc) = alpha op(A) op(B) + beta C
// in FP32 on the CUDA cores (op = transpose when ta / tb); column-major A
// (m x k, or k x m when ta) and B (k x n, or n x k when tb).  Splits K over
// several CTAs (atomic adds) when the output alone would not fill the GPU.
// *launches (may be null) counts the kernels launched.
cudaError_t gemm_f32(cudaStream_t st, bool ta, bool tb, int m, int n, int k, float alpha, const float *A, int lda,
                     const float *B, int ldb, float beta, float *C, int ldc, int num_sms, int *launches);
// Exclusive scan of n uint32 into uint64 (out has n+1 entries; out[n] = total).
size_t scan_scratch_bytes(size_t n);
cudaError_t exclusive_scan_u32_u64(const uint32_t *in, uint64_t *out, size_t n, void *scratch,
                                   cudaStream_t st);

}  // namespace ups
