// Front-to-back alpha blending of colour, depth, an N_l-channel feature map
// and transmittance (Eq. 3, Eq. 10), the per-pixel weighted loss (Eq. 4 /
// Eq. 14), and the reverse-order blending backward.
//
// One CTA per 16x16 image tile, PX pixels per thread (forward 2; backward 4
// for up to 16 feature channels, 2 for 32: registers).  The tile's
// depth-ordered Gaussian list is staged in shared memory in batches of list
// entries by the bulk-copy (TMA) engine: one cp.async.bulk per attribute
// record of an entry, completed on the batch's mbarrier, in a ring of stages
// so that the next batches load while one is blended.  A CTA stops when every
// pixel has terminated.  The backward walks the same list from each pixel's
// last blended Gaussian to the front, recomputing transmittance by division
// from the stored final T, and reduces per-Gaussian gradients over the warp
// through a shared-memory transpose before one vector atomic add per record
// group.
//
// Per (pixel, Gaussian) the exponent is evaluated as p(dy) = pa + dy (pb + pc
// dy), the quadratic form of the conic with the Gaussian's column offset dx
// fixed per thread (pa = -a dx^2 / 2, pb = -b dx, pc = -c / 2, all times
// log2 e for a base-2 exponential); the forward
// and the backward share this evaluation, so both take the same alpha
// decisions.  The four pixels of a thread are processed without branches
// (a pixel that takes no part contributes zero), which lets their independent
// dependency chains interleave.
#include <algorithm>

#include "common.cuh"
#include "umma.cuh"

namespace ups {

namespace {

constexpr int kWaitPolls = 1 << 22;

// Batch sizes and ring depths (compile-time tuning; a batch has at most one
// entry per thread): the forward stops early, so it takes few large batches;
// the backward walks whole prefixes.
#ifndef UPS_FWD_BATCH
#define UPS_FWD_BATCH 128
#endif
#ifndef UPS_FWD_STAGES
#define UPS_FWD_STAGES 2
#endif
#ifndef UPS_BWD_BATCH
#define UPS_BWD_BATCH 64
#endif

// one staged batch: attribute records of KB list entries
template <int NF, int KB>
struct Stage {
    float4 xyzo[KB];
    float4 conic[KB];
    float4 color[KB];
    float feat[KB][NF > 0 ? NF : 4];  // 16-byte rows
    uint32_t gv[KB];
};

template <int NF> struct StageBytes { static constexpr uint32_t value = 48u + 4u * NF; };

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     umma::smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(umma::smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(umma::smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// Entry t of a batch: its Gaussian-view id to shared memory, its four
// attribute records by bulk copies completing on mbar.
template <int NF, int KB>
__device__ __forceinline__ void stage_entry(Stage<NF, KB> &S, int t, uint32_t gv, int gs, const float4 *__restrict__ xyzo,
                                            const float4 *__restrict__ conic, const float4 *__restrict__ color,
                                            const float *__restrict__ feat, uint64_t *mbar) {
    S.gv[t] = gv;
    bulk_load(&S.xyzo[t], xyzo + gv, 16, mbar);
    bulk_load(&S.conic[t], conic + gv, 16, mbar);
    bulk_load(&S.color[t], color + gs, 16, mbar);
    if (NF > 0) bulk_load(&S.feat[t][0], feat + (size_t)gs * NF, 4 * NF, mbar);
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
#ifndef UPS_FWD_PX
#define UPS_FWD_PX 2
#endif
__host__ __device__ constexpr int blend_px_fwd(int nf) { return UPS_FWD_PX; }
__host__ __device__ constexpr int blend_px_bwd(int nf) { return nf <= 16 ? 4 : 2; }

// Exponent coefficients of a staged Gaussian for a thread's pixel column, in
// base 2: exp(p) = 2^(p log2 e), so the coefficients carry the factor log2 e
// and the falloff is one hardware base-2 exponential per pixel.
constexpr float kLog2e = 1.44269504088896341f;
struct Expo {
    float pa, pb, pc;
};
__device__ __forceinline__ Expo expo(float4 cn, float dx) {
    return Expo{(-0.5f * kLog2e) * cn.x * dx * dx, (-kLog2e * cn.y) * dx, (-0.5f * kLog2e) * cn.z};
}
__device__ __forceinline__ float expo_at(const Expo &e, float dy) { return fmaf(dy, fmaf(e.pc, dy, e.pb), e.pa); }
// G = 2^x (x = expo_at(...) <= 0 for a positive definite conic)
__device__ __forceinline__ float falloff(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Waits (bounded) for the batches issued but not yet consumed, so that no
// bulk copy is still writing this CTA's shared memory when it exits.
__device__ __forceinline__ void drain(uint64_t *mbar, int consumed, int issued, int ns, int *err) {
    for (int b = consumed; b < issued; ++b)
        if (!umma::mbar_wait(&mbar[b % ns], (uint32_t)((b / ns) & 1), kWaitPolls) && err) *err = 1;
}

constexpr int kFwdStages = UPS_FWD_STAGES;
constexpr int kFwdBatch = UPS_FWD_BATCH;

template <int NF, int PX>
__global__ void __launch_bounds__(Px<PX>::NT) k_composite_fwd(
    ViewTable vt, BlendParams bp, int N, int per_view, const uint2 *__restrict__ ranges,
    const uint32_t *__restrict__ ival, const float4 *__restrict__ xyzo,
    const float4 *__restrict__ conic, const float4 *__restrict__ color,
    const float *__restrict__ feat, float *__restrict__ out_color, float *__restrict__ out_depth,
    float *__restrict__ out_feat, float *__restrict__ out_T, uint32_t *__restrict__ out_nc,
    const uint32_t *__restrict__ trunc, int *__restrict__ trunc_flag, const int *__restrict__ gate,
    int *__restrict__ err) {
    // gate: when non-null, blend only if *gate != 0 (a pass enqueued ahead of
    // the GPU's decision to run it)
    if (gate && *gate == 0) return;
    constexpr int NT = Px<PX>::NT, RS = Px<PX>::RS, NS = kFwdStages, KB = kFwdBatch;
    static_assert(NT >= KB, "one thread per staged entry");
    __shared__ __align__(128) Stage<NF, KB> ring[NS];
    __shared__ __align__(8) uint64_t mbar[NS];
    const TileP<PX> tc = tilep<PX>(vt);
    const uint2 rg = ranges[blockIdx.x];
    const int n_list = (int)(rg.y - rg.x);
    const int nb = (n_list + KB - 1) / KB;
    const int set_base = (tc.v - tc.cam->set) * N;  // gv - set_base: attribute index
    const int tid = threadIdx.x;
    if (tid == 0)
        for (int s = 0; s < NS; ++s) umma::mbar_init(&mbar[s], 1);
    __syncthreads();
    // a thread's entry of batch b (t < KB)
    auto issue = [&](int b, uint32_t gv) {
        const int cnt = min(KB, n_list - b * KB);
        Stage<NF, KB> &S = ring[b % NS];
        if (tid == 0) mbar_expect(&mbar[b % NS], (uint32_t)cnt * StageBytes<NF>::value);
        if (tid < cnt) stage_entry<NF, KB>(S, tid, gv, (int)gv - set_base, xyzo, conic, color, feat, &mbar[b % NS]);
    };
    auto entry_gv = [&](int b) -> uint32_t {
        const int i = b * KB + tid;
        return (tid < KB && i < n_list) ? ival[rg.x + i] : 0u;
    };
    int issued = min(NS, nb);
    {
        uint32_t pg[NS];
#pragma unroll
        for (int b0 = 0; b0 < NS; ++b0) pg[b0] = b0 < issued ? entry_gv(b0) : 0u;
#pragma unroll
        for (int b0 = 0; b0 < NS; ++b0)
            if (b0 < issued) issue(b0, pg[b0]);
    }

    const float fx = (float)tc.px;
    float fy[PX], T[PX];
    f2 Ca[PX], Cb[PX];  // blended (r, g), (b, depth)
    f2 F[PX][NF > 0 ? NF / 2 : 1];  // feature accumulators, channel pairs
    uint32_t last[PX];
    bool done[PX];
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        fy[q] = (float)(tc.py0 + RS * q);
        T[q] = 1.f;
        Ca[q] = Cb[q] = 0ull;
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
    int b = 0;
    bool ok_wait = true;
    for (; b < nb; ++b) {
        // prefetch the id of this thread's entry of the batch that will reuse this slot
        const uint32_t nxt = issued < nb ? entry_gv(issued) : 0u;
        const bool arrived = umma::mbar_wait(&mbar[b % NS], (uint32_t)((b / NS) & 1), kWaitPolls);
        if (__syncthreads_or(!arrived)) {
            ok_wait = false;  // the drain below waits for this batch again
            if (err && tid == 0) *err = 1;
            break;
        }
        const Stage<NF, KB> &S = ring[b % NS];
        const int n = min(KB, n_list - b * KB);
        for (int j = 0; j < n; ++j) {
            if (__all_sync(0xffffffffu, all_done())) break;
            const float4 g = S.xyzo[j];
            const float4 cn = S.conic[j];
            const Expo ex = expo(cn, fx - g.x);
            const uint32_t pos = (uint32_t)(b * KB + j + 1);
            // alpha and the stopping test of every pixel first (independent
            // chains), then the weighted sums only where a pixel blends
            float alpha[PX], Tn[PX];
            bool use[PX];
            bool any = false;
#pragma unroll
            for (int q = 0; q < PX; ++q) {
                alpha[q] = fminf(bp.alpha_max, g.w * falloff(expo_at(ex, fy[q] - g.y)));
                Tn[q] = T[q] * (1.f - alpha[q]);
                use[q] = !done[q] && alpha[q] >= bp.alpha_min;
                const bool stop = use[q] && Tn[q] < bp.t_min;
                done[q] = done[q] || stop;
                use[q] = use[q] && !stop;
                any = any || use[q];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const float4 col = S.color[j];
            const f2 ca = f2_make(col.x, col.y), cb = f2_make(col.z, g.z);
#pragma unroll
            for (int q = 0; q < PX; ++q) {
                if (!use[q]) continue;
                const float w = alpha[q] * T[q];
                const f2 w2 = f2_make(w, w);
                Ca[q] = f2_fma(w2, ca, Ca[q]);
                Cb[q] = f2_fma(w2, cb, Cb[q]);
#pragma unroll
                for (int c = 0; c < NF; c += 4) {
                    const ulonglong2 f = *reinterpret_cast<const ulonglong2 *>(&S.feat[j][c]);
                    F[q][c / 2] = f2_fma(w2, f.x, F[q][c / 2]);
                    F[q][c / 2 + 1] = f2_fma(w2, f.y, F[q][c / 2 + 1]);
                }
                T[q] = Tn[q];
                last[q] = pos;
            }
        }
        // every thread is done with this slot (and with the batch) here
        const bool finished = __syncthreads_count(all_done()) == NT;
        if (finished) {
            ++b;
            break;
        }
        if (issued < nb) {
            umma::fence_async_smem();
            issue(issued, nxt);
            ++issued;
        }
    }
    drain(mbar, b, issued, NS, err);
    if (!ok_wait) return;
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
        float c0, c1, c2, d;
        f2_split(Ca[q], c0, c1);
        f2_split(Cb[q], c2, d);
        out_color[3 * P + p] = c0;
        out_color[3 * P + HW + p] = c1;
        out_color[3 * P + 2 * HW + p] = c2;
        out_depth[P + p] = d;
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

#ifndef UPS_BWD_STAGES
#define UPS_BWD_STAGES 3
#endif
constexpr int kBwdStages = UPS_BWD_STAGES;
// Tuning of the backward (compile-time): CTAs per SM the register allocation
// targets at 4 pixels per thread (8 caps registers at 128), and whether a warp
// skips a pixel row no lane of it blends (a vote per row) or runs it masked.
#ifndef UPS_BWD_MIN_BLOCKS
#define UPS_BWD_MIN_BLOCKS 6
#endif
#ifndef UPS_BWD_ROW_SKIP
#define UPS_BWD_ROW_SKIP 0
#endif
constexpr int kBwdMinBlocks = UPS_BWD_MIN_BLOCKS;
constexpr int kRedStride = 36;  // floats per lane row of the reduction scratch

// Sums over the warp of the per-lane gradient record values v (float4 groups
// 0..NG-1 of the record: du dv dz do | dca dcb dcc - | dr dg db - | df...) and
// adds them to rec (16-byte aligned) with one vector atomic per group.  The
// lanes write their groups to a [32][kRedStride] scratch row (16-byte stores,
// conflict-free), lane l then sums rows 8 (l / 8) .. 8 (l / 8) + 7 of column
// group l % 8 (a 32-float chunk at a time) in packed pairs, and two butterfly
// steps over l / 8 finish the sums.  All 32 lanes must call it.
template <int NG>
__device__ __forceinline__ void warp_record_add(const float4 (&v)[NG], float (*red)[kRedStride], int lane,
                                                float *rec) {
    const int col = lane & 7, rq = lane >> 3;
#pragma unroll
    for (int c0 = 0; c0 < NG; c0 += 8) {
        constexpr int kMax = 8;
#pragma unroll
        for (int k = 0; k < kMax; ++k)
            if (c0 + k < NG) *reinterpret_cast<float4 *>(&red[lane][4 * k]) = v[c0 + k];
        __syncwarp();
        f2 s01 = 0ull, s23 = 0ull;  // packed pairs of the group's four sums
        if (c0 + col < NG) {
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(&red[8 * rq + r][4 * col]);
                s01 = r == 0 ? x.x : f2_add(s01, x.x);
                s23 = r == 0 ? x.y : f2_add(s23, x.y);
            }
        }
#pragma unroll
        for (int o = 8; o <= 16; o <<= 1) {
            s01 = f2_add(s01, __shfl_xor_sync(0xffffffffu, s01, o));
            s23 = f2_add(s23, __shfl_xor_sync(0xffffffffu, s23, o));
        }
        float4 sum;
        f2_split(s01, sum.x, sum.y);
        f2_split(s23, sum.z, sum.w);
        if (rq == 0 && c0 + col < NG) atomicAdd(reinterpret_cast<float4 *>(rec) + c0 + col, sum);
        __syncwarp();
    }
}

template <int NF, int PX>
__global__ void __launch_bounds__(Px<PX>::NT, PX == 4 ? kBwdMinBlocks : 1) k_composite_bwd(
    ViewTable vt, BlendParams bp, int N, int per_view, const uint2 *__restrict__ ranges,
    const uint32_t *__restrict__ ival, const float4 *__restrict__ xyzo,
    const float4 *__restrict__ conic, const float4 *__restrict__ color,
    const float *__restrict__ feat, const float *__restrict__ in_T,
    const uint32_t *__restrict__ in_nc, const float *__restrict__ dC,
    const float *__restrict__ dD, const float *__restrict__ dF, const float *__restrict__ dT,
    float *__restrict__ g2, int *__restrict__ err) {
    constexpr int NT = Px<PX>::NT, RS = Px<PX>::RS, NW = NT / 32, NS = kBwdStages;
    constexpr int KB = NF > 16 ? 32 : UPS_BWD_BATCH;
    constexpr int STRIDE = kG2Base + NF;  // record floats, a multiple of 4
    constexpr int NG = STRIDE / 4;
    static_assert(NT >= KB, "one thread per staged entry");
    __shared__ __align__(128) Stage<NF, KB> ring[NS];
    __shared__ __align__(8) uint64_t mbar[NS];
    __shared__ __align__(16) float red[NW][32][kRedStride];
    __shared__ uint32_t s_max[NW];
    const TileP<PX> tc = tilep<PX>(vt);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint2 rg = ranges[blockIdx.x];
    const float fx = (float)tc.px;
    const DevView &cam = *tc.cam;
    const size_t HW = (size_t)cam.W * cam.H;
    const size_t P = (size_t)cam.pix_off;
    float T[PX], acc[PX];
    f2 gCa[PX], gCb[PX];             // (dL/dC_r, dL/dC_g), (dL/dC_b, dL/dD) per pixel
    f2 gF[PX][NF > 0 ? NF / 2 : 1];  // dL/d(feature image), channel pairs
    uint32_t nc[PX];
    uint32_t my_nc = 0;
#pragma unroll
    for (int q = 0; q < PX; ++q) {
        T[q] = 1.f;
        acc[q] = 0.f;
        gCa[q] = gCb[q] = 0ull;
        nc[q] = 0u;
#pragma unroll
        for (int c = 0; c < NF / 2; ++c) gF[q][c] = 0ull;
        if (!tc.in[q]) continue;
        const size_t p = (size_t)(tc.py0 + RS * q) * cam.W + tc.px;
        T[q] = in_T[P + p];
        nc[q] = in_nc[P + p];
        gCa[q] = f2_make(dC ? dC[3 * P + p] : 0.f, dC ? dC[3 * P + HW + p] : 0.f);
        gCb[q] = f2_make(dC ? dC[3 * P + 2 * HW + p] : 0.f, dD ? dD[P + p] : 0.f);
        if (dF)
#pragma unroll
            for (int c = 0; c < NF / 2; ++c)
                gF[q][c] = f2_make(dF[NF * P + 2 * c * HW + p], dF[NF * P + (2 * c + 1) * HW + p]);
        if (dT) acc[q] = dT[P + p] * T[q];
        my_nc = max(my_nc, nc[q]);
    }
    if (tid == 0)
        for (int s = 0; s < NS; ++s) umma::mbar_init(&mbar[s], 1);
    // longest blended prefix over the tile
    const uint32_t warp_nc = __reduce_max_sync(0xffffffffu, my_nc);
    if (lane == 0) s_max[wid] = warp_nc;
    __syncthreads();
    int max_nc = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) max_nc = max(max_nc, (int)s_max[w]);
    // batch b holds list positions [max(0, max_nc - (b + 1) KB), max_nc - b KB), back to front
    const int nb = (max_nc + KB - 1) / KB;
    const int set_base = (tc.v - tc.cam->set) * N;  // gv - set_base: attribute index
    auto lo_of = [&](int b) { return max(0, max_nc - (b + 1) * KB); };
    auto entry_gv = [&](int b) -> uint32_t {
        const int lo = lo_of(b), i = lo + tid;
        return (tid < KB && i < max_nc - b * KB) ? ival[rg.x + i] : 0u;
    };
    auto issue = [&](int b, uint32_t gv) {
        const int lo = lo_of(b), cnt = max_nc - b * KB - lo;
        Stage<NF, KB> &S = ring[b % NS];
        if (tid == 0) mbar_expect(&mbar[b % NS], (uint32_t)cnt * StageBytes<NF>::value);
        if (tid < cnt) stage_entry<NF, KB>(S, tid, gv, (int)gv - set_base, xyzo, conic, color, feat, &mbar[b % NS]);
    };
    int issued = min(NS, nb);
    {
        uint32_t pg[NS];
#pragma unroll
        for (int b0 = 0; b0 < NS; ++b0) pg[b0] = b0 < issued ? entry_gv(b0) : 0u;
#pragma unroll
        for (int b0 = 0; b0 < NS; ++b0)
            if (b0 < issued) issue(b0, pg[b0]);
    }
    float fy[PX];
#pragma unroll
    for (int q = 0; q < PX; ++q) fy[q] = (float)(tc.py0 + RS * q);
    int b = 0;
    for (; b < nb; ++b) {
        const uint32_t nxt = issued < nb ? entry_gv(issued) : 0u;
        const bool arrived = umma::mbar_wait(&mbar[b % NS], (uint32_t)((b / NS) & 1), kWaitPolls);
        if (__syncthreads_or(!arrived)) {
            if (err && tid == 0) *err = 1;
            break;  // the drain below waits for this batch again
        }
        const Stage<NF, KB> &S = ring[b % NS];
        const int lo = lo_of(b), hi = max_nc - b * KB;
        // warps whose pixels all stop earlier skip the tail of the batch
        const int jstart = min(hi, (int)warp_nc) - lo - 1;
        for (int j = jstart; j >= 0; --j) {
            const int idx = lo + j;
            const float4 g = S.xyzo[j];
            const float4 cn = S.conic[j];
            const float dx = fx - g.x;
            const Expo ex = expo(cn, dx);
            float G[PX], alpha[PX], dy[PX];
            bool use[PX];
            bool any = false;
#pragma unroll
            for (int q = 0; q < PX; ++q) {
                dy[q] = fy[q] - g.y;
                G[q] = falloff(expo_at(ex, dy[q]));
                alpha[q] = fminf(bp.alpha_max, g.w * G[q]);
                use[q] = idx < (int)nc[q] && alpha[q] >= bp.alpha_min;
                any = any || use[q];
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const float4 col = S.color[j];
            const f2 ca = f2_make(col.x, col.y), cb = f2_make(col.z, g.z);
            f2 fj[NF > 0 ? NF / 2 : 1];
#pragma unroll
            for (int c = 0; c < NF; c += 4) {
                const ulonglong2 f = *reinterpret_cast<const ulonglong2 *>(&S.feat[j][c]);
                fj[c / 2] = f.x;
                fj[c / 2 + 1] = f.y;
            }
            // per-thread sums over its pixels.  With t = dL/dalpha * G for an
            // unclamped alpha (0 otherwise), dL/do = sum t and the exponent
            // p = pa + dy (pb + pc dy) has dL/dp = o t per pixel, so the conic
            // and mean terms need only sum t, sum t dy and sum t dy^2 (dx is
            // the thread's), scaled by o once per Gaussian.
            float sop = 0.f, sty = 0.f, styy = 0.f;
            f2 sca = 0ull, scb = 0ull;  // sum w (dL/dC_r, dL/dC_g), sum w (dL/dC_b, dL/dD)
            f2 vF[NF > 0 ? NF / 2 : 1];
#pragma unroll
            for (int c = 0; c < NF / 2; ++c) vF[c] = 0ull;
#pragma unroll
            for (int q = 0; q < PX; ++q) {
                if (UPS_BWD_ROW_SKIP && !__any_sync(0xffffffffu, use[q])) continue;
                const float a = use[q] ? alpha[q] : 0.f;
                const float rom = use[q] ? __fdividef(1.f, 1.f - a) : 1.f;
                T[q] *= rom;  // transmittance in front of this Gaussian
                const float w = a * T[q];
                const f2 w2 = f2_make(w, w);
                f2 xg2 = f2_fma(cb, gCb[q], f2_fma(ca, gCa[q], 0ull));
#pragma unroll
                for (int c = 0; c < NF / 2; ++c) {
                    xg2 = f2_fma(fj[c], gF[q][c], xg2);
                    vF[c] = f2_fma(w2, gF[q][c], vF[c]);
                }
                float xlo, xhi;
                f2_split(xg2, xlo, xhi);
                const float xg = xlo + xhi;  // dL/d(blended value) . (c, z, f) of this Gaussian
                // dL/dalpha where alpha is not clamped, 0 elsewhere
                const float dal = use[q] && alpha[q] < bp.alpha_max ? T[q] * xg - acc[q] * rom : 0.f;
                acc[q] = fmaf(w, xg, acc[q]);
                const float t = dal * G[q];
                sop += t;
                const float ty = t * dy[q];
                sty += ty;
                styy = fmaf(ty, dy[q], styy);
                sca = f2_fma(w2, gCa[q], sca);
                scb = f2_fma(w2, gCb[q], scb);
            }
            // record groups: du dv dz do | dca dcb dcc - | dr dg db - | df...
            float4 v[NG];
            // d(u, v) = o sum t (a dx + b dy, b dx + c dy) (dx, dy: pixel minus
            // mean); d(a, b, c) = -o/2 sum t (dx^2, 2 dx dy, dy^2)
            const float ho = -0.5f * g.w;
            float sc0, sc1, sc2, sz;
            f2_split(sca, sc0, sc1);
            f2_split(scb, sc2, sz);
            v[0] = make_float4(g.w * fmaf(cn.x * dx, sop, cn.y * sty), g.w * fmaf(cn.y * dx, sop, cn.z * sty), sz,
                               sop);
            v[1] = make_float4(ho * dx * dx * sop, -g.w * dx * sty, ho * styy, 0.f);
            v[2] = make_float4(sc0, sc1, sc2, 0.f);
#pragma unroll
            for (int c = 0; c < NF / 4; ++c) {
                float a0, a1, a2, a3;
                f2_split(vF[2 * c], a0, a1);
                f2_split(vF[2 * c + 1], a2, a3);
                v[3 + c] = make_float4(a0, a1, a2, a3);
            }
            warp_record_add<NG>(v, red[wid], lane, g2 + (size_t)S.gv[j] * STRIDE);
        }
        __syncthreads();  // every thread is done with this slot
        if (issued < nb) {
            umma::fence_async_smem();
            issue(issued, nxt);
            ++issued;
        }
    }
    drain(mbar, b, issued, NS, err);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_composite_fwd(const ViewTable &vt, const BlendParams &bp, int n_feat, int N,
                                 int per_view, const uint2 *ranges, const uint32_t *ival,
                                 const float4 *xyzo, const float4 *conic, const float4 *color,
                                 const float *feat, const ups_images &out, cudaStream_t st,
                                 const uint32_t *trunc, int *trunc_flag, const int *gate, int *err) {
    if (vt.total_tiles == 0) return cudaSuccess;
#define UPS_FWD(NFV)                                                                                  \
    k_composite_fwd<NFV, blend_px_fwd(NFV)><<<vt.total_tiles, Px<blend_px_fwd(NFV)>::NT, 0, st>>>(              \
        vt, bp, N, per_view, ranges, ival, xyzo, conic, color, feat, out.color, out.depth, out.feat, out.T, \
        out.n_contrib, trunc, trunc_flag, gate, err)
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
                                 const ups_image_grads &dL, float *g2, cudaStream_t st, int *err) {
    if (vt.total_tiles == 0) return cudaSuccess;
#define UPS_BWD(NFV)                                                                                \
    k_composite_bwd<NFV, blend_px_bwd(NFV)><<<vt.total_tiles, Px<blend_px_bwd(NFV)>::NT, 0, st>>>(            \
        vt, bp, N, per_view, ranges, ival, xyzo, conic, color, feat, T, nc, dL.color, dL.depth, dL.feat, \
        dL.T, g2, err)
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
