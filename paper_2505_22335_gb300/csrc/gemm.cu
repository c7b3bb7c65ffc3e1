// Plain FP32 matrix product on the CUDA cores for the library's small and
// weight-sized contractions (feature lifting, uncertainty MLP):
//   C = alpha op(A) op(B) + beta C
// column-major like the BLAS convention (element (i, j) of an m x n matrix
// with leading dimension ld at [i + j ld]); op(X) = X or X^T.  Every product
// is a sequence of fmaf in FP32.
//
// 64 x 64 output tiles, 256 threads, 4 x 4 outputs per thread, K staged 16 at
// a time in shared memory (K-major, so a thread reads its 4 rows and 4
// columns as two 16-byte loads).  Loads follow the operand's contiguous axis.
// A product whose tiles are too few to fill the GPU is split along K over
// grid.z, the parts added with atomics into C after C was scaled by beta.
#include <algorithm>

#include "common.cuh"

namespace ups {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_f32(int m, int n, int k, int kchunk, float alpha,
                                                  const float *__restrict__ A, int lda, const float *__restrict__ B,
                                                  int ldb, float beta, float *__restrict__ C, int ldc, int split) {
    // rows padded by 4 floats: the transposed-operand stores hit 8 banks, not 1
    __shared__ __align__(16) float As[kBK][kBM + 4];
    __shared__ __align__(16) float Bs[kBK][kBN + 4];
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * kBM, j0 = blockIdx.y * kBN;
    const int k_beg = blockIdx.z * kchunk, k_end = min(k, k_beg + kchunk);
    const int ti = (tid & 15) * 4, tj = (tid >> 4) * 4;
    float acc[4][4] = {};
    for (int kk = k_beg; kk < k_end; kk += kBK) {
        // 1024 elements of each operand tile, 4 per thread, along the
        // operand's contiguous axis
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + 256 * e;
            int r, c;  // r: along M (A) or N (B), c: along K
            if (!TA) {
                r = idx & (kBM - 1);
                c = idx >> 6;
            } else {
                c = idx & (kBK - 1);
                r = idx >> 4;
            }
            const int gi = i0 + r, gk = kk + c;
            float a = 0.f;
            if (gi < m && gk < k_end) a = TA ? A[gk + (size_t)gi * lda] : A[gi + (size_t)gk * lda];
            As[c][r] = a;
            if (!TB) {
                c = idx & (kBK - 1);
                r = idx >> 4;
            } else {
                r = idx & (kBN - 1);
                c = idx >> 6;
            }
            const int gj = j0 + r, gk2 = kk + c;
            float b = 0.f;
            if (gj < n && gk2 < k_end) b = TB ? B[gj + (size_t)gk2 * ldb] : B[gk2 + (size_t)gj * ldb];
            Bs[c][r] = b;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kBK; ++c) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[c][ti]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[c][tj]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gi = i0 + ti + x, gj = j0 + tj + y;
            if (gi >= m || gj >= n) continue;
            float *cp = C + gi + (size_t)gj * ldc;
            if (split)
                atomicAdd(cp, alpha * acc[x][y]);
            else
                *cp = beta == 0.f ? alpha * acc[x][y] : fmaf(beta, *cp, alpha * acc[x][y]);
        }
}

__global__ void k_scale_cols(int m, int n, float beta, float *__restrict__ C, int ldc) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)m * n) return;
    const int i = (int)(idx % m), j = (int)(idx / m);
    float *cp = C + i + (size_t)j * ldc;
    *cp = beta == 0.f ? 0.f : beta * *cp;
}

}  // namespace

cudaError_t gemm_f32(cudaStream_t st, bool ta, bool tb, int m, int n, int k, float alpha, const float *A, int lda,
                     const float *B, int ldb, float beta, float *C, int ldc, int num_sms, int *launches) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int gm = (m + kBM - 1) / kBM, gn = (n + kBN - 1) / kBN;
    // split K when the output tiles alone would leave most SMs idle
    int split = 1, kchunk = 0;
    if (k > 0) {
        const int tiles = gm * gn;
        if (tiles < 2 * num_sms && k > 4 * kBK)
            split = std::min((2 * num_sms + tiles - 1) / tiles, (k + 255) / 256);
        split = std::max(1, std::min(split, 65535));
        kchunk = (k + split - 1) / split;
        kchunk = (kchunk + kBK - 1) / kBK * kBK;
        split = std::max(1, (k + kchunk - 1) / kchunk);
    }
    if (split > 1 && beta != 1.f) {
        const size_t total = (size_t)m * n;
        k_scale_cols<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(m, n, beta, C, ldc);
        if (launches) ++*launches;
    }
    const dim3 grid(gm, gn, split);
#define UPS_GEMM(TA, TB) \
    k_gemm_f32<TA, TB><<<grid, 256, 0, st>>>(m, n, k, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, split > 1)
    if (!ta && !tb) UPS_GEMM(false, false);
    else if (!ta && tb) UPS_GEMM(false, true);
    else if (ta && !tb) UPS_GEMM(true, false);
    else UPS_GEMM(true, true);
#undef UPS_GEMM
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace ups
