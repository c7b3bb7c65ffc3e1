// Front-to-back alpha blending of colour, depth, an N_l-channel feature map
// and transmittance (Eq. 3, Eq. 10), the per-pixel weighted loss (Eq. 4 /
// Eq. 14), and the reverse-order blending backward.
//
// One CTA per 16x16 image tile, PX pixels per thread (forward 2; backward 4
// for up to 16 feature channels, 2 for 32: registers).  The tile's
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

// channels [c, c + 4) of staged Gaussian j as two pairs
template <int NF, class St>
__device__ __forceinline__ ulonglong2 feat4(const St &S, int j, int c) {
    return *reinterpret_cast<const ulonglong2 *>(&S.feat[j][c]);
}

template <int NF>
struct Stage {
    float4 xyzo[kBatch];
    float4 conic[kBatch];
    float4 color[kBatch];
    // Gaussian-major, rows padded by 4 floats: 16-byte broadcast reads of four
    // channels, conflict-free 16-byte staging stores
    float feat[kBatch][NF > 0 ? NF + 4 : 1];
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
            *reinterpret_cast<float4 *>(&S.feat[slot][4 * c]) = f;
        }
    }
}

// Each thread owns PX pixels of the tile, (x, y + (16 / PX) q) for q < PX:
// the staged Gaussian is read from shared memory once for all of them (and,
// in the backward, reduced across the warp once for all of them).
template <int PX> struct Px {
    static constexpr int NT = kTilePix / PX;  // threads per tile
    static constexpr int RS = kTile / PX;     // row step between a thread's pixels
};

template <int PX>
struct TileP {
    int v, px, py0;
    bool in[PX];
    const DevView *cam;
};

template <int PX>
__device__ __forceinline__ TileP<PX> tilep(const ViewTable &vt) {
    TileP<PX> c;
    const int t = blockIdx.x;
    c.v = view_of_tile(vt, t);
    c.cam = &vt.v[c.v];
    int local = t - c.cam->tile_base;
    int ty = local / c.cam->tiles_x;
    int tx = local - ty * c.cam->tiles_x;
    c.px = tx * kTile + (threadIdx.x & (kTile - 1));
    c.py0 = ty * kTile + (threadIdx.x / kTile);
#pragma unroll
    for (int q = 0; q < PX; ++q) c.in[q] = c.px < c.cam->W && c.py0 + Px<PX>::RS * q < c.cam->H;
    return c;
}

// pixels per thread: forward 2; backward 4 up to 16 feature channels (the
// per-Gaussian warp reduction is shared by more pixels), 2 for 32 (registers)
__host__ __device__ constexpr int blend_px_fwd(int nf) { return 2; }
__host__ __device__ constexpr int blend_px_bwd(int nf) { return nf <= 16 ? 4 : 2; }

template <int NF, int PX>
__global__ void __launch_bounds__(Px<PX>::NT) k_composite_fwd(
    ViewTable vt, BlendParams bp, int N, int per_view, const uint2 *__restrict__ ranges,
    const uint32_t *__restrict__ ival, const float4 *__restrict__ xyzo,
    const float4 *__restrict__ conic, const float4 *__restrict__ color,
    const float *__restrict__ feat, float *__restrict__ out_color, float *__restrict__ out_depth,
    float *__restrict__ out_feat, float *__restrict__ out_T, uint32_t *__restrict__ out_nc,
    const uint32_t *__restrict__ trunc, int *__restrict__ trunc_flag, const int *__restrict__ gate) {
    // gate: when non-null, blend only if *gate != 0 (a pass enqueued ahead of
    // the GPU's decision to run it)
    if (gate && *gate == 0) return;
    constexpr int NT = Px<PX>::NT, RS = Px<PX>::RS;
    __shared__ Stage<NF> S;
    const TileP<PX> tc = tilep<PX>(vt);
    const uint2 rg = ranges[blockIdx.x];
    const float fx = (float)tc.px;
    float fy[PX], T[PX], C0[PX], C1[PX], C2[PX], D[PX];
    f2 F[PX][NF > 0 ? NF / 2 : 1];  // feature accumulators, channel pairs
    uint32_t last[PX];
    bool done[PX];
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        fy[q] = (float)(tc.py0 + RS * q);
        T[q] = 1.f;
        C0[q] = C1[q] = C2[q] = D[q] = 0.f;
#pragma unroll
        for (int c = 0; c < NF / 2; ++c) F[q][c] = 0ull;
        last[q] = 0u;
        done[q] = !tc.in[q];
    }
    auto all_done = [&]() {
        bool d = true;
#pragma unroll
        for (int q = 0; q < PX; ++q) d = d && done[q];
        return d;
    };
    const int set_base = per_view ? 0 : tc.v * N;
    for (uint32_t base = rg.x; base < rg.y; base += kBatch) {
        if (__syncthreads_count(all_done()) == NT) break;
#pragma unroll
        for (int h = 0; h < kBatch / NT; ++h) {
            uint32_t i = base + threadIdx.x + h * NT;
            if (i < rg.y) {
                uint32_t gv = ival[i];
                stage_load<NF>(S, threadIdx.x + h * NT, gv, (int)gv - set_base, xyzo, conic, color, feat);
            }
        }
        __syncthreads();
        const int n = min((int)(rg.y - base), kBatch);
        for (int j = 0; j < n && !all_done(); ++j) {
            const float4 g = S.xyzo[j];
            const float4 cn = S.conic[j];
            const float dx = fx - g.x;
#pragma unroll
            for (int q = 0; q < PX; ++q) {
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
                const f2 w2 = f2_make(w, w);
#pragma unroll
                for (int c = 0; c < NF; c += 4) {
                    const ulonglong2 f = feat4<NF>(S, j, c);
                    F[q][c / 2] = f2_fma(w2, f.x, F[q][c / 2]);
                    F[q][c / 2 + 1] = f2_fma(w2, f.y, F[q][c / 2 + 1]);
                }
                T[q] = Tn;
                last[q] = base - rg.x + j + 1;
            }
        }
    }
    // a list cut short by the list cap is exact only if every pixel stopped
    // inside it; otherwise the caller blends the tile again from a full list
    if (trunc && ((trunc[blockIdx.x >> 5] >> (blockIdx.x & 31)) & 1u))
        if (__syncthreads_count(all_done()) != NT && threadIdx.x == 0) atomicOr(trunc_flag, 1);
    const DevView &cam = *tc.cam;
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t P = (size_t)cam.pix_off;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        if (!tc.in[q]) continue;
        const size_t p = (size_t)(tc.py0 + RS * q) * cam.W + tc.px;
        out_color[3 * P + p] = C0[q];
        out_color[3 * P + HW + p] = C1[q];
        out_color[3 * P + 2 * HW + p] = C2[q];
        out_depth[P + p] = D[q];
#pragma unroll
        for (int c = 0; c < NF / 2; ++c) {
            out_feat[NF * P + 2 * c * HW + p] = f2_lo(F[q][c]);
            out_feat[NF * P + (2 * c + 1) * HW + p] = f2_hi(F[q][c]);
        }
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

template <int NF, int PX>
__global__ void __launch_bounds__(Px<PX>::NT) k_composite_bwd(
    ViewTable vt, BlendParams bp, int N, int per_view, const uint2 *__restrict__ ranges,
    const uint32_t *__restrict__ ival, const float4 *__restrict__ xyzo,
    const float4 *__restrict__ conic, const float4 *__restrict__ color,
    const float *__restrict__ feat, const float *__restrict__ in_T,
    const uint32_t *__restrict__ in_nc, const float *__restrict__ dC,
    const float *__restrict__ dD, const float *__restrict__ dF, const float *__restrict__ dT,
    float *__restrict__ g2) {
    constexpr int NT = Px<PX>::NT, RS = Px<PX>::RS;
    constexpr int RP = RecPad<NF>::value;
    constexpr int STRIDE = kG2Base + NF;
    __shared__ Stage<NF> S;
    __shared__ uint32_t s_max[NT / 32];
    const TileP<PX> tc = tilep<PX>(vt);
    const int lane = threadIdx.x & 31;
    const uint2 rg = ranges[blockIdx.x];
    const float fx = (float)tc.px;
    const DevView &cam = *tc.cam;
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t P = (size_t)cam.pix_off;
    float fy[PX], T[PX], acc[PX], gC0[PX], gC1[PX], gC2[PX], gD[PX];
    f2 gF[PX][NF > 0 ? NF / 2 : 1];  // dL/d(feature image), channel pairs
    uint32_t nc[PX];
    uint32_t my_nc = 0;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        fy[q] = (float)(tc.py0 + RS * q);
        T[q] = 1.f;
        acc[q] = gC0[q] = gC1[q] = gC2[q] = gD[q] = 0.f;
        nc[q] = 0u;
#pragma unroll
        for (int c = 0; c < NF / 2; ++c) gF[q][c] = 0ull;
        if (!tc.in[q]) continue;
        const size_t p = (size_t)(tc.py0 + RS * q) * cam.W + tc.px;
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
            for (int c = 0; c < NF / 2; ++c)
                gF[q][c] = f2_make(dF[NF * P + 2 * c * HW + p], dF[NF * P + (2 * c + 1) * HW + p]);
        if (dT) acc[q] = dT[P + p] * T[q];
        my_nc = max(my_nc, nc[q]);
    }
    // longest blended prefix over the tile
    uint32_t m = __reduce_max_sync(0xffffffffu, my_nc);
    if (lane == 0) s_max[threadIdx.x >> 5] = m;
    __syncthreads();
    uint32_t max_nc = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) max_nc = max(max_nc, s_max[w]);
    const int set_base = per_view ? 0 : tc.v * N;
    for (int hi = (int)max_nc; hi > 0; hi -= kBatch) {
        const int lo = max(0, hi - kBatch);
        __syncthreads();
#pragma unroll
        for (int h = 0; h < kBatch / NT; ++h) {
            int i = lo + threadIdx.x + h * NT;
            if (i < hi) {
                uint32_t gv = ival[rg.x + i];
                stage_load<NF>(S, threadIdx.x + h * NT, gv, (int)gv - set_base, xyzo, conic, color, feat);
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
            f2 vF[NF > 0 ? NF / 2 : 1];  // feature-gradient sums, channel pairs
#pragma unroll
            for (int c = 0; c < NF / 2; ++c) vF[c] = 0ull;
            bool any = false;
#pragma unroll
            for (int q = 0; q < PX; ++q) {
                if (idx >= (int)nc[q]) continue;
                const float dy = fy[q] - g.y;
                const float power = -0.5f * (cn.x * dx * dx + cn.z * dy * dy) - cn.y * dx * dy;
                const float G = __expf(power);
                const float raw = g.w * G;
                const float alpha = fminf(bp.alpha_max, raw);
                if (alpha < bp.alpha_min) continue;
                any = true;
                const float om = 1.f - alpha;
                const float rom = __frcp_rn(om);
                T[q] = T[q] * rom;  // transmittance in front of this Gaussian
                const float w = alpha * T[q];
                const f2 w2 = f2_make(w, w);
                f2 xg2 = 0ull;
#pragma unroll
                for (int c = 0; c < NF; c += 4) {
                    const ulonglong2 f = feat4<NF>(S, j, c);
                    xg2 = f2_fma(f.x, gF[q][c / 2], xg2);
                    xg2 = f2_fma(f.y, gF[q][c / 2 + 1], xg2);
                    vF[c / 2] = f2_fma(w2, gF[q][c / 2], vF[c / 2]);
                    vF[c / 2 + 1] = f2_fma(w2, gF[q][c / 2 + 1], vF[c / 2 + 1]);
                }
                const float xg = col.x * gC0[q] + col.y * gC1[q] + col.z * gC2[q] + g.z * gD[q] +
                                 (NF > 0 ? f2_lo(xg2) + f2_hi(xg2) : 0.f);
                const float dalpha = T[q] * xg - acc[q] * rom;
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
#pragma unroll
            for (int c = 0; c < NF / 2; ++c) {
                v[kG2Base + 2 * c] = f2_lo(vF[c]);
                v[kG2Base + 2 * c + 1] = f2_hi(vF[c]);
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
                                 const float *feat, const ups_images &out, cudaStream_t st,
                                 const uint32_t *trunc, int *trunc_flag, const int *gate) {
    if (vt.total_tiles == 0) return cudaSuccess;
#define UPS_FWD(NFV)                                                                                  \
    k_composite_fwd<NFV, blend_px_fwd(NFV)><<<vt.total_tiles, Px<blend_px_fwd(NFV)>::NT, 0, st>>>(              \
        vt, bp, N, per_view, ranges, ival, xyzo, conic, color, feat, out.color, out.depth, out.feat, out.T, \
        out.n_contrib, trunc, trunc_flag, gate)
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
    if (vt.total_tiles == 0) return cudaSuccess;
#define UPS_BWD(NFV)                                                                                \
    k_composite_bwd<NFV, blend_px_bwd(NFV)><<<vt.total_tiles, Px<blend_px_bwd(NFV)>::NT, 0, st>>>(            \
        vt, bp, N, per_view, ranges, ival, xyzo, conic, color, feat, T, nc, dL.color, dL.depth, dL.feat, \
        dL.T, g2)
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
