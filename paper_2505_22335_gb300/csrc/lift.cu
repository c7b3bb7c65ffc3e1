// Feature lifting F_m and the distillation loss L_d (Sec. 3.3, Eq. 11, Eq. 12;
// App. "MLP Implementation Details"): the rendered N_l-channel feature map F~
// goes through a per-pixel (1x1 convolution) MLP N_l -> 128 -> ReLU -> N_h to
// F^, compared by cosine with the DINO feature F of the pixel, bilinearly
// upsampled from the view's patch grid (Sec. 3.2):
//   L_d = (1 / P) sum_p (1 - cos(F_p, F^_p)),   cos = 0 where a vector is 0.
//
// The two layers and their backward are plain GEMMs over the pixels of a
// view; they run as cuBLAS TF32 tensor-core GEMMs on the planar image layout
// (channel c of pixel p at [c * HW + p] is a column-major HW x C matrix, so
// no repacking is needed).  The kernels here do the rest: bias + ReLU, the
// bilinear upsampling with the cosine, the loss and dL/dF^, the ReLU mask and
// the bias sums.
#include <cublas_v2.h>

#include "common.cuh"

namespace ups {

namespace {

constexpr int kLiftHidden = 128;

__global__ void k_bias_relu(float *__restrict__ z, const float *__restrict__ b, size_t HW) {
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= HW) return;
    float *row = z + (size_t)blockIdx.y * HW;
    row[p] = fmaxf(row[p] + b[blockIdx.y], 0.f);
}

// dZ = dH where H > 0 (ReLU derivative), in place
__global__ void k_relu_mask(float *__restrict__ dh, const float *__restrict__ h, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(h[i] > 0.f)) dh[i] = 0.f;
}

// out[r] += sum_p m[r * HW + p]: blockIdx.y = row, blockIdx.x = a chunk of
// kSumChunk pixels, one atomic per block
constexpr int kSumChunk = 8192;
__global__ void __launch_bounds__(256) k_row_sums(const float *__restrict__ m, size_t HW, float *__restrict__ out) {
    const float *row = m + (size_t)blockIdx.y * HW;
    const size_t p0 = (size_t)blockIdx.x * kSumChunk;
    const size_t p1 = min(HW, p0 + kSumChunk);
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    size_t p = p0 + threadIdx.x;
    for (; p + 768 < p1; p += 1024) {
        s0 += row[p];
        s1 += row[p + 256];
        s2 += row[p + 512];
        s3 += row[p + 768];
    }
    for (; p < p1; p += 256) s0 += row[p];
    float s = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(out + blockIdx.y, t);
    }
}

// Per pixel: F^ = Fh + b2 (Fh = H W2^T of the view), F bilinear from the
// patch grid [hp][wp][nh] at patch coordinate ((x + 0.5) / patch - 0.5,
// (y + 0.5) / patch - 0.5) clamped to the grid; loss += g (1 - cos); Fh is
// overwritten with g dL_d/dF^ = g (cos F^ / |F^|^2 - F / (|F| |F^|)), with g =
// scale / P.  Zero vectors: cos = 0 and no gradient.
__global__ void __launch_bounds__(256) k_lift_cos(float *__restrict__ fh, const float *__restrict__ b2, int W,
                                                  int H, int nh, const float *__restrict__ grid, int wp, int hp,
                                                  int patch, float g0, const float *__restrict__ weight,
                                                  float *__restrict__ loss) {
    const size_t HW = (size_t)W * H;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float term = 0.f;
    if (p < HW) {
        const float wpx = weight ? weight[p] : 1.f;  // per-pixel weight (the mask of Eq. 14)
        const float g = g0 * wpx;
        const int y = (int)(p / (size_t)W), x = (int)(p - (size_t)y * W);
        const float inv = 1.f / (float)patch;
        const float u = fminf(fmaxf(((float)x + 0.5f) * inv - 0.5f, 0.f), (float)(wp - 1));
        const float v = fminf(fmaxf(((float)y + 0.5f) * inv - 0.5f, 0.f), (float)(hp - 1));
        const int x0 = (int)u, y0 = (int)v;
        const int x1 = min(x0 + 1, wp - 1), y1 = min(y0 + 1, hp - 1);
        const float ax = u - (float)x0, ay = v - (float)y0;
        const float w00 = (1.f - ax) * (1.f - ay), w01 = ax * (1.f - ay), w10 = (1.f - ax) * ay, w11 = ax * ay;
        // the four patch vectors, four channels per 16-byte load (nh % 4 == 0)
        const float4 *g00 = reinterpret_cast<const float4 *>(grid + ((size_t)y0 * wp + x0) * nh);
        const float4 *g01 = reinterpret_cast<const float4 *>(grid + ((size_t)y0 * wp + x1) * nh);
        const float4 *g10 = reinterpret_cast<const float4 *>(grid + ((size_t)y1 * wp + x0) * nh);
        const float4 *g11 = reinterpret_cast<const float4 *>(grid + ((size_t)y1 * wp + x1) * nh);
        const float4 *b4 = reinterpret_cast<const float4 *>(b2);
        auto target = [&](int q) {
            const float4 a = __ldg(g00 + q), b = __ldg(g01 + q), c = __ldg(g10 + q), d = __ldg(g11 + q);
            return make_float4(w00 * a.x + w01 * b.x + w10 * c.x + w11 * d.x,
                               w00 * a.y + w01 * b.y + w10 * c.y + w11 * d.y,
                               w00 * a.z + w01 * b.z + w10 * c.z + w11 * d.z,
                               w00 * a.w + w01 * b.w + w10 * c.w + w11 * d.w);
        };
        float dot = 0.f, na = 0.f, nb = 0.f;
        const int nq = nh >> 2;
#pragma unroll 2
        for (int q = 0; q < nq; ++q) {
            const float4 f = target(q), bb = __ldg(b4 + q);
            const float *col = fh + (size_t)(4 * q) * HW + p;
            const float f4[4] = {f.x, f.y, f.z, f.w};
            const float fb4[4] = {col[0] + bb.x, col[HW] + bb.y, col[2 * HW] + bb.z, col[3 * HW] + bb.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                dot = fmaf(f4[k], fb4[k], dot);
                na = fmaf(f4[k], f4[k], na);
                nb = fmaf(fb4[k], fb4[k], nb);
            }
        }
        const bool ok = na > 0.f && nb > 0.f;
        const float ia = ok ? rsqrtf(na) : 0.f, ib = ok ? rsqrtf(nb) : 0.f;
        const float cs = dot * ia * ib;
        term = wpx * (1.f - cs);
        const float k1 = g * cs * ib * ib, k2 = g * ia * ib;
#pragma unroll 2
        for (int q = 0; q < nq; ++q) {
            const float4 f = target(q), bb = __ldg(b4 + q);
            float *col = fh + (size_t)(4 * q) * HW + p;
            const float f4[4] = {f.x, f.y, f.z, f.w};
            const float b4v[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float fb = col[k * HW] + b4v[k];
                col[k * HW] = ok ? k1 * fb - k2 * f4[k] : 0.f;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(loss, g0 * t);
    }
}

cudaError_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const float *A,
                 int lda, const float *B, int ldb, float beta, float *Cm, int ldc) {
    const float alpha = 1.f;
    const cublasStatus_t s = cublasGemmEx(h, ta, tb, m, n, k, &alpha, A, CUDA_R_32F, lda, B, CUDA_R_32F, ldb, &beta,
                                          Cm, CUDA_R_32F, ldc, CUBLAS_COMPUTE_32F_FAST_TF32, CUBLAS_GEMM_DEFAULT);
    return s == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown;
}

}  // namespace

size_t lift_scratch_floats(size_t max_hw, int nh) { return max_hw * (2 * kLiftHidden + (size_t)nh); }

cudaError_t lift_handle(void **handle) {
    if (*handle) return cudaSuccess;
    cublasHandle_t h = nullptr;
    if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    *handle = h;
    return cudaSuccess;
}

void lift_handle_destroy(void *handle) {
    if (handle) cublasDestroy(static_cast<cublasHandle_t>(handle));
}

// One view: forward, loss and backward.  feat / d_feat: the view's planes
// [nf][HW]; grid: its patch grid; weight: its per-pixel weights (null: 1);
// scratch: lift_scratch_floats(HW, nh).
// d_w1 [128][nf], d_b1 [128], d_w2 [nh][128], d_b2 [nh] and d_feat are
// accumulated (may be null: that gradient is skipped).
cudaError_t lift_view(void *handle, cudaStream_t st, int W, int H, int nf, int nh, int patch, const float *feat,
                      const float *grid, int wp, int hp, const float *w1, const float *b1, const float *w2,
                      const float *b2, float g, const float *weight, float *loss, float *d_w1, float *d_b1,
                      float *d_w2, float *d_b2, float *d_feat, float *scratch, int *launches) {
    cublasHandle_t h = static_cast<cublasHandle_t>(handle);
    if (cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    const int HW = W * H;
    const int NH = kLiftHidden;
    float *Hm = scratch;                       // [128][HW] hidden (post-ReLU)
    float *Fh = Hm + (size_t)NH * HW;          // [nh][HW] F^ - b2, then g dL/dF^
    float *dZ = Fh + (size_t)nh * HW;          // [128][HW] dL/dZ1
    const dim3 blk(256);
    const unsigned gx = (unsigned)((HW + 255) / 256);
    cudaError_t e;
    // Z1 = F~ W1^T, H = relu(Z1 + b1)
    if ((e = gemm(h, CUBLAS_OP_N, CUBLAS_OP_N, HW, NH, nf, feat, HW, w1, nf, 0.f, Hm, HW)) != cudaSuccess) return e;
    k_bias_relu<<<dim3(gx, NH), blk, 0, st>>>(Hm, b1, (size_t)HW);
    // F^ - b2 = H W2^T
    if ((e = gemm(h, CUBLAS_OP_N, CUBLAS_OP_N, HW, nh, NH, Hm, HW, w2, NH, 0.f, Fh, HW)) != cudaSuccess) return e;
    k_lift_cos<<<gx, blk, 0, st>>>(Fh, b2, W, H, nh, grid, wp, hp, patch, g, weight, loss);
    *launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool want_w = d_w1 || d_b1 || d_w2 || d_b2;
    if (!want_w && !d_feat) return cudaSuccess;
    if (d_b2) {
        k_row_sums<<<dim3((unsigned)((HW + kSumChunk - 1) / kSumChunk), nh), blk, 0, st>>>(Fh, (size_t)HW, d_b2);
        ++*launches;
    }
    // dW2 += H^T dF^  ([128 x nh] column-major = [nh][128] row-major)
    if (d_w2 && (e = gemm(h, CUBLAS_OP_T, CUBLAS_OP_N, NH, nh, HW, Hm, HW, Fh, HW, 1.f, d_w2, NH)) != cudaSuccess)
        return e;
    // dZ1 = (dF^ W2) * relu'(Z1)
    if ((e = gemm(h, CUBLAS_OP_N, CUBLAS_OP_T, HW, NH, nh, Fh, HW, w2, NH, 0.f, dZ, HW)) != cudaSuccess) return e;
    k_relu_mask<<<std::min<unsigned>(4096u, (unsigned)(((size_t)NH * HW + 255) / 256)), blk, 0, st>>>(
        dZ, Hm, (size_t)NH * HW);
    ++*launches;
    if (d_b1) {
        k_row_sums<<<dim3((unsigned)((HW + kSumChunk - 1) / kSumChunk), NH), blk, 0, st>>>(dZ, (size_t)HW, d_b1);
        ++*launches;
    }
    // dW1 += F~^T dZ1 ([nf x 128] column-major = [128][nf] row-major)
    if (d_w1 && (e = gemm(h, CUBLAS_OP_T, CUBLAS_OP_N, nf, NH, HW, feat, HW, dZ, HW, 1.f, d_w1, nf)) != cudaSuccess)
        return e;
    // dF~ += dZ1 W1
    if (d_feat && (e = gemm(h, CUBLAS_OP_N, CUBLAS_OP_T, HW, nf, NH, dZ, HW, w1, nf, 1.f, d_feat, HW)) != cudaSuccess)
        return e;
    return cudaGetLastError();
}

}  // namespace ups
