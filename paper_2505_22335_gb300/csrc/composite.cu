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

template <int NF>
__global__ void __launch_bounds__(256) k_composite_fwd(
    ViewTable vt, BlendParams bp, int N, int per_view, const uint2 *__restrict__ ranges,
    const uint32_t *__restrict__ ival, const float4 *__restrict__ xyzo,
    const float4 *__restrict__ conic, const float4 *__restrict__ color,
    const float *__restrict__ feat, float *__restrict__ out_color, float *__restrict__ out_depth,
    float *__restrict__ out_feat, float *__restrict__ out_T, uint32_t *__restrict__ out_nc) {
    __shared__ Stage<NF> S;
    const TileCtx tc = tile_ctx(vt);
    const uint2 rg = ranges[blockIdx.x];
    const float fx = (float)tc.px, fy = (float)tc.py;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    float F[NF > 0 ? NF : 1];
#pragma unroll
    for (int c = 0; c < NF; ++c) F[c] = 0.f;
    uint32_t last = 0;
    bool done = !tc.inside;
    const int set_base = per_view ? 0 : tc.v * N;
    for (uint32_t base = rg.x; base < rg.y; base += kBatch) {
        if (__syncthreads_count(done) == kBatch) break;
        uint32_t i = base + threadIdx.x;
        if (i < rg.y) {
            uint32_t gv = ival[i];
            stage_load<NF>(S, threadIdx.x, gv, (int)gv - set_base, xyzo, conic, color, feat);
        }
        __syncthreads();
        int n = min((int)(rg.y - base), kBatch);
        if (!done) {
            for (int j = 0; j < n; ++j) {
                float4 g = S.xyzo[j];
                float4 cn = S.conic[j];
                float dx = fx - g.x, dy = fy - g.y;
                float power = -0.5f * (cn.x * dx * dx + cn.z * dy * dy) - cn.y * dx * dy;
                float alpha = fminf(bp.alpha_max, g.w * __expf(power));
                if (alpha < bp.alpha_min) continue;
                float Tn = T * (1.f - alpha);
                if (Tn < bp.t_min) {
                    done = true;
                    break;
                }
                float w = alpha * T;
                float4 col = S.color[j];
                C0 = fmaf(w, col.x, C0);
                C1 = fmaf(w, col.y, C1);
                C2 = fmaf(w, col.z, C2);
                D = fmaf(w, g.z, D);
#pragma unroll
                for (int c = 0; c < NF; ++c) F[c] = fmaf(w, S.feat[c][j], F[c]);
                T = Tn;
                last = base - rg.x + j + 1;
            }
        }
    }
    if (tc.inside) {
        const DevView &cam = *tc.cam;
        const size_t HW = (size_t)cam.W * cam.H;
        const size_t p = (size_t)tc.py * cam.W + tc.px;
        const size_t P = (size_t)cam.pix_off;
        out_color[3 * P + p] = C0;
        out_color[3 * P + HW + p] = C1;
        out_color[3 * P + 2 * HW + p] = C2;
        out_depth[P + p] = D;
#pragma unroll
        for (int c = 0; c < NF; ++c) out_feat[NF * P + c * HW + p] = F[c];
        out_T[P + p] = T;
        out_nc[P + p] = last;
    }
}

// ---------------------------------------------------------------------------
// loss
// ---------------------------------------------------------------------------

template <int NF>
__global__ void __launch_bounds__(256) k_loss(
    ViewTable vt, float lc, float ld, float lf, int l2, float inv_norm,
    const float *__restrict__ color, const float *__restrict__ depth,
    const float *__restrict__ feat, const float *__restrict__ t_color,
    const float *__restrict__ t_depth, const float *__restrict__ t_feat,
    const float *__restrict__ weight, float *__restrict__ g_color, float *__restrict__ g_depth,
    float *__restrict__ g_feat, float *__restrict__ loss) {
    const DevView &cam = vt.v[blockIdx.y];
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t P = (size_t)cam.pix_off;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    if (p < HW) {
        float w = weight ? weight[P + p] : 1.f;
        auto term = [&](float r, float lam, float *g, size_t idx) {
            float val = l2 ? r * r : fabsf(r);
            float der = l2 ? 2.f * r : (float)((r > 0.f) - (r < 0.f));
            acc += w * lam * val;
            g[idx] = w * lam * der * inv_norm;
        };
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            size_t idx = 3 * P + c * HW + p;
            term(color[idx] - t_color[idx], lc, g_color, idx);
        }
        term(depth[P + p] - t_depth[P + p], ld, g_depth, P + p);
#pragma unroll
        for (int c = 0; c < NF; ++c) {
            size_t idx = NF * P + c * HW + p;
            term(feat[idx] - t_feat[idx], lf, g_feat, idx);
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
__global__ void __launch_bounds__(256) k_composite_bwd(
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
    __shared__ uint32_t s_max[8];
    const TileCtx tc = tile_ctx(vt);
    const int lane = threadIdx.x & 31;
    const uint2 rg = ranges[blockIdx.x];
    const float fx = (float)tc.px, fy = (float)tc.py;
    const DevView &cam = *tc.cam;
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t P = (size_t)cam.pix_off;
    const size_t p = (size_t)(tc.inside ? tc.py : 0) * cam.W + (tc.inside ? tc.px : 0);
    float T = 1.f, acc = 0.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f;
    float gF[NF > 0 ? NF : 1];
#pragma unroll
    for (int c = 0; c < NF; ++c) gF[c] = 0.f;
    uint32_t nc = 0;
    if (tc.inside) {
        T = in_T[P + p];
        nc = in_nc[P + p];
        if (dC) {
            gC0 = dC[3 * P + p];
            gC1 = dC[3 * P + HW + p];
            gC2 = dC[3 * P + 2 * HW + p];
        }
        if (dD) gD = dD[P + p];
#pragma unroll
        for (int c = 0; c < NF; ++c) gF[c] = dF ? dF[NF * P + c * HW + p] : 0.f;
        if (dT) acc = dT[P + p] * T;
    }
    // longest blended prefix over the tile
    uint32_t m = __reduce_max_sync(0xffffffffu, nc);
    if (lane == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    uint32_t max_nc = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) max_nc = max(max_nc, s_max[w]);
    const int set_base = per_view ? 0 : tc.v * N;
    for (int hi = (int)max_nc; hi > 0; hi -= kBatch) {
        const int lo = max(0, hi - kBatch);
        __syncthreads();
        {
            int i = lo + threadIdx.x;
            if (i < hi) {
                uint32_t gv = ival[rg.x + i];
                stage_load<NF>(S, threadIdx.x, gv, (int)gv - set_base, xyzo, conic, color, feat);
            }
        }
        __syncthreads();
        for (int j = hi - lo - 1; j >= 0; --j) {
            const int idx = lo + j;
            bool contrib = idx < (int)nc;
            float v[RP];
#pragma unroll
            for (int k = 0; k < RP; ++k) v[k] = 0.f;
            if (contrib) {
                float4 g = S.xyzo[j];
                float4 cn = S.conic[j];
                float dx = fx - g.x, dy = fy - g.y;
                float power = -0.5f * (cn.x * dx * dx + cn.z * dy * dy) - cn.y * dx * dy;
                float G = __expf(power);
                float raw = g.w * G;
                float alpha = fminf(bp.alpha_max, raw);
                if (alpha < bp.alpha_min) {
                    contrib = false;
                } else {
                    float om = 1.f - alpha;
                    T = T / om;  // transmittance in front of this Gaussian
                    float w = alpha * T;
                    float4 col = S.color[j];
                    float xg = col.x * gC0 + col.y * gC1 + col.z * gC2 + g.z * gD;
#pragma unroll
                    for (int c = 0; c < NF; ++c) {
                        float f = S.feat[c][j];
                        xg = fmaf(f, gF[c], xg);
                        v[kG2Base + c] = w * gF[c];
                    }
                    float dalpha = T * xg - acc / om;
                    acc = fmaf(w, xg, acc);
                    float dq = 0.f;
                    if (raw < bp.alpha_max) {
                        v[3] = dalpha * G;
                        dq = dalpha * (-0.5f * alpha);
                    }
                    v[0] = dq * (-2.f) * (cn.x * dx + cn.y * dy);
                    v[1] = dq * (-2.f) * (cn.y * dx + cn.z * dy);
                    v[2] = w * gD;
                    v[4] = dq * dx * dx;
                    v[5] = dq * 2.f * dx * dy;
                    v[6] = dq * dy * dy;
                    v[8] = w * gC0;
                    v[9] = w * gC1;
                    v[10] = w * gC2;
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
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
    dim3 grid(vt.total_tiles), block(256);
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
                        const ups_images &grad, float *loss, cudaStream_t st) {
    dim3 grid((max_hw + 255) / 256, vt.n), block(256);
#define UPS_LOSS(NFV)                                                                          \
    k_loss<NFV><<<grid, block, 0, st>>>(vt, lc, ld, lf, l2, inv_norm, img.color, img.depth,    \
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
    dim3 grid(vt.total_tiles), block(256);
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
