// Front-to-back alpha blending of colour, depth, an N_l-channel feature map
// and transmittance (Eq. 3, Eq. 10), the per-pixel weighted loss (Eq. 4 /
// Eq. 14), and the reverse-order blending backward.
//
// One 256-thread CTA per 16x16 image tile, one pixel per thread.  The tile's
// depth-ordered Gaussian list is walked in batches of 256 staged in shared
// memory; a CTA stops when every pixel has terminated.  The backward walks
// the same list from each pixel's last blended Gaussian to the front,
// recomputing transmittance by division from the stored final T, and reduces
// per-Gaussian gradients across the warp (transposed butterfly: each lane
// ends up owning one or two of the record's values) before one coalesced
// atomic add per warp.
#include <algorithm>

#include "common.cuh"

namespace ups {

namespace {

constexpr int kBatch = 256;

struct TileCtx {
    int v, tx, ty, px, py;
    bool inside;
    const DevView *cam;
};

__device__ __forceinline__ TileCtx tile_ctx(const ViewTable &vt) {
    TileCtx c;
    const int t = blockIdx.x;
    c.v = view_of_tile(vt, t);
    c.cam = &vt.v[c.v];
    int local = t - c.cam->tile_base;
    c.ty = local / c.cam->tiles_x;
    c.tx = local - c.ty * c.cam->tiles_x;
    c.px = c.tx * kTile + (threadIdx.x & (kTile - 1));
    c.py = c.ty * kTile + (threadIdx.x / kTile);
    c.inside = c.px < c.cam->W && c.py < c.cam->H;
    return c;
}

template <int NF>
struct Stage {
    float4 xyzo[kBatch];
    float4 conic[kBatch];
    float4 color[kBatch];
    float feat[NF > 0 ? NF : 1][kBatch];  // channel-major: conflict-free broadcast reads
    uint32_t gv[kBatch];
};

template <int NF>
__device__ __forceinline__ void stage_load(Stage<NF> &S, int slot, uint32_t gv, int gs,
                                           const float4 *__restrict__ xyzo,
                                           const float4 *__restrict__ conic,
                                           const float4 *__restrict__ color,
                                           const float *__restrict__ feat) {
    S.gv[slot] = gv;
    S.xyzo[slot] = xyzo[gv];
    S.conic[slot] = conic[gv];
    S.color[slot] = color[gs];
    if (NF > 0) {
        const float4 *f4 = reinterpret_cast<const float4 *>(feat + (size_t)gs * NF);
#pragma unroll
        for (int c = 0; c < NF / 4; ++c) {
            float4 f = f4[c];
            S.feat[4 * c + 0][slot] = f.x;
            S.feat[4 * c + 1][slot] = f.y;
            S.feat[4 * c + 2][slot] = f.z;
            S.feat[4 * c + 3][slot] = f.w;
        }
    }
}

// Each thread owns two pixels of the tile, (x, y) and (x, y + 8): the staged
// Gaussian is read from shared memory once for both.
constexpr int kThreadsBlend = 128;

struct Tile2 {
    int v, px, py0;
    bool in0, in1;
    const DevView *cam;
};

__device__ __forceinline__ Tile2 tile2(const ViewTable &vt) {
    Tile2 c;
    const int t = blockIdx.x;
    c.v = view_of_tile(vt, t);
    c.cam = &vt.v[c.v];
    int local = t - c.cam->tile_base;
    int ty = local / c.cam->tiles_x;
    int tx = local - ty * c.cam->tiles_x;
    c.px = tx * kTile + (threadIdx.x & (kTile - 1));
    c.py0 = ty * kTile + (threadIdx.x / kTile);
    c.in0 = c.px < c.cam->W && c.py0 < c.cam->H;
    c.in1 = c.px < c.cam->W && c.py0 + 8 < c.cam->H;
    return c;
}

template <int NF>
__global__ void __launch_bounds__(kThreadsBlend) k_composite_fwd(
    ViewTable vt, BlendParams bp, int N, int per_view, const uint2 *__restrict__ ranges,
    const uint32_t *__restrict__ ival, const float4 *__restrict__ xyzo,
    const float4 *__restrict__ conic, const float4 *__restrict__ color,
    const float *__restrict__ feat, float *__restrict__ out_color, float *__restrict__ out_depth,
    float *__restrict__ out_feat, float *__restrict__ out_T, uint32_t *__restrict__ out_nc) {
    __shared__ Stage<NF> S;
    const Tile2 tc = tile2(vt);
    const uint2 rg = ranges[blockIdx.x];
    const float fx = (float)tc.px;
    const float fy[2] = {(float)tc.py0, (float)(tc.py0 + 8)};
    float T[2] = {1.f, 1.f}, C0[2] = {0.f, 0.f}, C1[2] = {0.f, 0.f}, C2[2] = {0.f, 0.f},
          D[2] = {0.f, 0.f};
    float F[2][NF > 0 ? NF : 1];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < NF; ++c) F[q][c] = 0.f;
    uint32_t last[2] = {0u, 0u};
    bool done[2] = {!tc.in0, !tc.in1};
    const int set_base = per_view ? 0 : tc.v * N;
    for (uint32_t base = rg.x; base < rg.y; base += kBatch) {
        if (__syncthreads_count(done[0] && done[1]) == kThreadsBlend) break;
#pragma unroll
        for (int h = 0; h < kBatch / kThreadsBlend; ++h) {
            uint32_t i = base + threadIdx.x + h * kThreadsBlend;
            if (i < rg.y) {
                uint32_t gv = ival[i];
                stage_load<NF>(S, threadIdx.x + h * kThreadsBlend, gv, (int)gv - set_base, xyzo,
                               conic, color, feat);
            }
        }
        __syncthreads();
        const int n = min((int)(rg.y - base), kBatch);
        for (int j = 0; j < n && !(done[0] && done[1]); ++j) {
            const float4 g = S.xyzo[j];
            const float4 cn = S.conic[j];
            const float dx = fx - g.x;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (done[q]) continue;
                const float dy = fy[q] - g.y;
                const float power = -0.5f * (cn.x * dx * dx + cn.z * dy * dy) - cn.y * dx * dy;
                const float alpha = fminf(bp.alpha_max, g.w * __expf(power));
                if (alpha < bp.alpha_min) continue;
                const float Tn = T[q] * (1.f - alpha);
                if (Tn < bp.t_min) {
                    done[q] = true;
                    continue;
                }
                const float w = alpha * T[q];
                const float4 col = S.color[j];
                C0[q] = fmaf(w, col.x, C0[q]);
                C1[q] = fmaf(w, col.y, C1[q]);
                C2[q] = fmaf(w, col.z, C2[q]);
                D[q] = fmaf(w, g.z, D[q]);
#pragma unroll
                for (int c = 0; c < NF; ++c) F[q][c] = fmaf(w, S.feat[c][j], F[q][c]);
                T[q] = Tn;
                last[q] = base - rg.x + j + 1;
            }
        }
    }
    const DevView &cam = *tc.cam;
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t P = (size_t)cam.pix_off;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (!(q == 0 ? tc.in0 : tc.in1)) continue;
        const size_t p = (size_t)(tc.py0 + 8 * q) * cam.W + tc.px;
        out_color[3 * P + p] = C0[q];
        out_color[3 * P + HW + p] = C1[q];
        out_color[3 * P + 2 * HW + p] = C2[q];
        out_depth[P + p] = D[q];
#pragma unroll
        for (int c = 0; c < NF; ++c) out_feat[NF * P + c * HW + p] = F[q][c];
        out_T[P + p] = T[q];
        out_nc[P + p] = last[q];
    }
}

// ---------------------------------------------------------------------------
// loss
// ---------------------------------------------------------------------------

template <int NF>
__global__ void __launch_bounds__(256) k_loss(
    ViewTable vt, int v0, int tgt_base, float lc, float ld, float lf, int l2, float inv_norm,
    const float *__restrict__ color, const float *__restrict__ depth,
    const float *__restrict__ feat, const float *__restrict__ t_color,
    const float *__restrict__ t_depth, const float *__restrict__ t_feat,
    const float *__restrict__ weight, float *__restrict__ g_color, float *__restrict__ g_depth,
    float *__restrict__ g_feat, float *__restrict__ loss) {
    // view v0 + blockIdx.y; targets and weights are indexed from pixel tgt_base
    const DevView &cam = vt.v[v0 + blockIdx.y];
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t P = (size_t)cam.pix_off;
    const size_t PT = P - (size_t)tgt_base;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    if (p < HW) {
        float w = weight ? weight[PT + p] : 1.f;
        auto term = [&](float r, float lam, float *g, size_t idx) {
            float val = l2 ? r * r : fabsf(r);
            float der = l2 ? 2.f * r : (float)((r > 0.f) - (r < 0.f));
            acc += w * lam * val;
            g[idx] = w * lam * der * inv_norm;
        };
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            size_t idx = 3 * P + c * HW + p;
            term(color[idx] - t_color[3 * PT + c * HW + p], lc, g_color, idx);
        }
        term(depth[P + p] - t_depth[PT + p], ld, g_depth, P + p);
#pragma unroll
        for (int c = 0; c < NF; ++c) {
            size_t idx = NF * P + c * HW + p;
            term(feat[idx] - t_feat[NF * PT + c * HW + p], lf, g_feat, idx);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s * inv_norm);
    }
}

// lambda * mean(s) over all Gaussian scales
__global__ void k_scale_mean(const float4 *__restrict__ scale, size_t n, float coef,
                             float *__restrict__ loss) {
    float acc = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float4 s = scale[i];
        acc += s.x + s.y + s.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(loss, s * coef);
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

// Number of record slots reduced per warp: next power of two >= 12 + NF.
template <int NF> struct RecPad { static constexpr int value = NF == 0 ? 16 : (NF <= 20 ? 32 : 64); };

// Transposed butterfly reduction of RP values over the 32 lanes.  On return
// v[0..max(RP/32,1)-1] holds the warp sums of record indices idx_of(lane, i).
template <int RP>
__device__ __forceinline__ void warp_transpose_reduce(float (&v)[RP], int lane) {
    constexpr unsigned full = 0xffffffffu;
    int n = RP;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (n > 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < RP / 2; ++i) {
                if (i < n / 2) {
                    float send = up ? v[i] : v[i + n / 2];
                    float keep = up ? v[i + n / 2] : v[i];
                    v[i] = keep + __shfl_xor_sync(full, send, o);
                }
            }
            n >>= 1;
        } else {
            v[0] += __shfl_xor_sync(full, v[0], o);
        }
    }
}

template <int NF>
__global__ void __launch_bounds__(kThreadsBlend) k_composite_bwd(
    ViewTable vt, BlendParams bp, int N, int per_view, const uint2 *__restrict__ ranges,
    const uint32_t *__restrict__ ival, const float4 *__restrict__ xyzo,
    const float4 *__restrict__ conic, const float4 *__restrict__ color,
    const float *__restrict__ feat, const float *__restrict__ in_T,
    const uint32_t *__restrict__ in_nc, const float *__restrict__ dC,
    const float *__restrict__ dD, const float *__restrict__ dF, const float *__restrict__ dT,
    float *__restrict__ g2) {
    constexpr int RP = RecPad<NF>::value;
    constexpr int STRIDE = kG2Base + NF;
    __shared__ Stage<NF> S;
    __shared__ uint32_t s_max[kThreadsBlend / 32];
    const Tile2 tc = tile2(vt);
    const int lane = threadIdx.x & 31;
    const uint2 rg = ranges[blockIdx.x];
    const float fx = (float)tc.px;
    const float fy[2] = {(float)tc.py0, (float)(tc.py0 + 8)};
    const DevView &cam = *tc.cam;
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t P = (size_t)cam.pix_off;
    float T[2] = {1.f, 1.f}, acc[2] = {0.f, 0.f}, gC0[2] = {0.f, 0.f}, gC1[2] = {0.f, 0.f},
          gC2[2] = {0.f, 0.f}, gD[2] = {0.f, 0.f};
    float gF[2][NF > 0 ? NF : 1];
    uint32_t nc[2] = {0u, 0u};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int c = 0; c < NF; ++c) gF[q][c] = 0.f;
        if (!(q == 0 ? tc.in0 : tc.in1)) continue;
        const size_t p = (size_t)(tc.py0 + 8 * q) * cam.W + tc.px;
        T[q] = in_T[P + p];
        nc[q] = in_nc[P + p];
        if (dC) {
            gC0[q] = dC[3 * P + p];
            gC1[q] = dC[3 * P + HW + p];
            gC2[q] = dC[3 * P + 2 * HW + p];
        }
        if (dD) gD[q] = dD[P + p];
        if (dF)
#pragma unroll
            for (int c = 0; c < NF; ++c) gF[q][c] = dF[NF * P + c * HW + p];
        if (dT) acc[q] = dT[P + p] * T[q];
    }
    // longest blended prefix over the tile
    uint32_t m = __reduce_max_sync(0xffffffffu, max(nc[0], nc[1]));
    if (lane == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    uint32_t max_nc = 0;
#pragma unroll
    for (int w = 0; w < kThreadsBlend / 32; ++w) max_nc = max(max_nc, s_max[w]);
    const uint32_t my_nc = max(nc[0], nc[1]);
    const int set_base = per_view ? 0 : tc.v * N;
    for (int hi = (int)max_nc; hi > 0; hi -= kBatch) {
        const int lo = max(0, hi - kBatch);
        __syncthreads();
#pragma unroll
        for (int h = 0; h < kBatch / kThreadsBlend; ++h) {
            int i = lo + threadIdx.x + h * kThreadsBlend;
            if (i < hi) {
                uint32_t gv = ival[rg.x + i];
                stage_load<NF>(S, threadIdx.x + h * kThreadsBlend, gv, (int)gv - set_base, xyzo,
                               conic, color, feat);
            }
        }
        __syncthreads();
        // warps whose pixels all stop earlier skip the tail of the batch
        const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, my_nc);
        int jstart = min(hi - lo, (int)warp_nc - lo) - 1;
        for (int j = jstart; j >= 0; --j) {
            const int idx = lo + j;
            const float4 g = S.xyzo[j];
            const float4 cn = S.conic[j];
            const float4 col = S.color[j];
            const float dx = fx - g.x;
            float v[RP];
#pragma unroll
            for (int k = 0; k < RP; ++k) v[k] = 0.f;
            bool any = false;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (idx >= (int)nc[q]) continue;
                const float dy = fy[q] - g.y;
                const float power = -0.5f * (cn.x * dx * dx + cn.z * dy * dy) - cn.y * dx * dy;
                const float G = __expf(power);
                const float raw = g.w * G;
                const float alpha = fminf(bp.alpha_max, raw);
                if (alpha < bp.alpha_min) continue;
                any = true;
                const float om = 1.f - alpha;
                T[q] = T[q] / om;  // transmittance in front of this Gaussian
                const float w = alpha * T[q];
                float xg = col.x * gC0[q] + col.y * gC1[q] + col.z * gC2[q] + g.z * gD[q];
#pragma unroll
                for (int c = 0; c < NF; ++c) {
                    xg = fmaf(S.feat[c][j], gF[q][c], xg);
                    v[kG2Base + c] = fmaf(w, gF[q][c], v[kG2Base + c]);
                }
                const float dalpha = T[q] * xg - acc[q] / om;
                acc[q] = fmaf(w, xg, acc[q]);
                float dq = 0.f;
                if (raw < bp.alpha_max) {
                    v[3] = fmaf(dalpha, G, v[3]);
                    dq = dalpha * (-0.5f * alpha);
                }
                v[0] = fmaf(dq * (-2.f), cn.x * dx + cn.y * dy, v[0]);
                v[1] = fmaf(dq * (-2.f), cn.y * dx + cn.z * dy, v[1]);
                v[2] = fmaf(w, gD[q], v[2]);
                v[4] = fmaf(dq, dx * dx, v[4]);
                v[5] = fmaf(dq, 2.f * dx * dy, v[5]);
                v[6] = fmaf(dq, dy * dy, v[6]);
                v[8] = fmaf(w, gC0[q], v[8]);
                v[9] = fmaf(w, gC1[q], v[9]);
                v[10] = fmaf(w, gC2[q], v[10]);
            }
            if (__any_sync(0xffffffffu, any)) {
                warp_transpose_reduce<RP>(v, lane);
                float *rec = g2 + (size_t)S.gv[j] * STRIDE;
                if (RP == 16) {
                    int k = lane >> 1;
                    if (!(lane & 1) && k != 7 && k != 11 && k < STRIDE) atomicAdd(rec + k, v[0]);
                } else if (RP == 32) {
                    int k = lane;
                    if (k != 7 && k != 11 && k < STRIDE) atomicAdd(rec + k, v[0]);
                } else {
#pragma unroll
                    for (int e = 0; e < RP / 32; ++e) {
                        int k = (RP / 32) * lane + e;
                        if (k != 7 && k != 11 && k < STRIDE) atomicAdd(rec + k, v[e]);
                    }
                }
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_composite_fwd(const ViewTable &vt, const BlendParams &bp, int n_feat, int N,
                                 int per_view, const uint2 *ranges, const uint32_t *ival,
                                 const float4 *xyzo, const float4 *conic, const float4 *color,
                                 const float *feat, const ups_images &out, cudaStream_t st) {
    dim3 grid(vt.total_tiles), block(kThreadsBlend);
    if (vt.total_tiles == 0) return cudaSuccess;
#define UPS_FWD(NFV)                                                                          \
    k_composite_fwd<NFV><<<grid, block, 0, st>>>(vt, bp, N, per_view, ranges, ival, xyzo, conic, \
                                                 color, feat, out.color, out.depth, out.feat,  \
                                                 out.T, out.n_contrib)
    switch (n_feat) {
        case 0: UPS_FWD(0); break;
        case 16: UPS_FWD(16); break;
        case 32: UPS_FWD(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef UPS_FWD
    return cudaGetLastError();
}

cudaError_t launch_loss(const ViewTable &vt, int n_feat, int max_hw, float lc, float ld, float lf,
                        int l2, float inv_norm, const ups_images &img, const ups_targets &tgt,
                        const ups_images &grad, float *loss, cudaStream_t st, int v0, int v1) {
    if (v1 < 0) v1 = vt.n;
    if (v1 <= v0) return cudaSuccess;
    const int tgt_base = vt.v[v0].pix_off;
    dim3 grid((max_hw + 255) / 256, v1 - v0), block(256);
#define UPS_LOSS(NFV)                                                                          \
    k_loss<NFV><<<grid, block, 0, st>>>(vt, v0, tgt_base, lc, ld, lf, l2, inv_norm, img.color, img.depth, \
                                        img.feat, tgt.color, tgt.depth, tgt.feat, tgt.weight,   \
                                        grad.color, grad.depth, grad.feat, loss)
    switch (n_feat) {
        case 0: UPS_LOSS(0); break;
        case 16: UPS_LOSS(16); break;
        case 32: UPS_LOSS(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef UPS_LOSS
    return cudaGetLastError();
}

cudaError_t launch_scale_mean(const float4 *scale, size_t n, float coef, float *loss,
                              cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int blocks = (int)std::min<size_t>((n + 255) / 256, 1024);
    k_scale_mean<<<blocks, 256, 0, st>>>(scale, n, coef, loss);
    return cudaGetLastError();
}

cudaError_t launch_composite_bwd(const ViewTable &vt, const BlendParams &bp, int n_feat, int N,
                                 int per_view, const uint2 *ranges, const uint32_t *ival,
                                 const float4 *xyzo, const float4 *conic, const float4 *color,
                                 const float *feat, const float *T, const uint32_t *nc,
                                 const ups_image_grads &dL, float *g2, cudaStream_t st) {
    dim3 grid(vt.total_tiles), block(kThreadsBlend);
    if (vt.total_tiles == 0) return cudaSuccess;
#define UPS_BWD(NFV)                                                                          \
    k_composite_bwd<NFV><<<grid, block, 0, st>>>(vt, bp, N, per_view, ranges, ival, xyzo, conic, \
                                                 color, feat, T, nc, dL.color, dL.depth,       \
                                                 dL.feat, dL.T, g2)
    switch (n_feat) {
        case 0: UPS_BWD(0); break;
        case 16: UPS_BWD(16); break;
        case 32: UPS_BWD(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef UPS_BWD
    return cudaGetLastError();
}

}  // namespace ups
