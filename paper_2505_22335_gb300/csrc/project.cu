// EWA projection of 3D Gaussians (Eq. 1-2), depth keys, tile-instance
// emission and tile ranges, and the projection backward into mean, scale,
// rotation and SE(3) pose gradients.
//
// One thread per Gaussian-view; attributes are read as float4 records.
#include "common.cuh"

namespace ups {

namespace {

struct Geo {
    float p[3];       // camera-space mean
    float W[9];       // rotation of T_cw
    float Rq[9];      // rotation of the normalised quaternion
    float qn[4], qinv;  // normalised quaternion and 1/|q|
    float s[3];
    float T[6];       // J W (2x3)
    float Sig[6];     // world covariance (xx, xy, xz, yy, yz, zz)
    float A, B, C;    // Sigma' (with dilation)
};

__device__ __forceinline__ void quat_rot(const float q[4], float R[9]) {
    float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - w * z);
    R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);
    R[7] = 2.f * (y * z + w * x);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

// camera-space mean; returns validity (near plane, frustum guard, opacity)
__device__ __forceinline__ bool camera_point(const DevView &cam, const BlendParams &bp, float4 m,
                                             float p[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
        p[i] = fmaf(cam.R[3 * i], m.x, fmaf(cam.R[3 * i + 1], m.y, fmaf(cam.R[3 * i + 2], m.z, cam.t[i])));
    if (!(p[2] > bp.near_z)) return false;
    if (fabsf(p[0] / p[2]) > cam.limx || fabsf(p[1] / p[2]) > cam.limy) return false;
    return m.w >= bp.alpha_min;
}

// Sigma = R S S^T R^T, Sigma' = (J W) Sigma (J W)^T + dilation I
__device__ __forceinline__ void covariance(const DevView &cam, const BlendParams &bp, float4 sc,
                                           float4 q, Geo &G) {
    float qs = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    G.qinv = 1.f / qs;
    G.qn[0] = q.x * G.qinv;
    G.qn[1] = q.y * G.qinv;
    G.qn[2] = q.z * G.qinv;
    G.qn[3] = q.w * G.qinv;
    quat_rot(G.qn, G.Rq);
    G.s[0] = sc.x;
    G.s[1] = sc.y;
    G.s[2] = sc.z;
    float M[9];  // R S
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = G.Rq[3 * i + j] * G.s[j];
    G.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    G.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    G.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    G.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    G.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    G.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
#pragma unroll
    for (int i = 0; i < 9; ++i) G.W[i] = cam.R[i];
    float iz = 1.f / G.p[2];
    float j00 = cam.fx * iz, j02 = -cam.fx * G.p[0] * iz * iz;
    float j11 = cam.fy * iz, j12 = -cam.fy * G.p[1] * iz * iz;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        G.T[j] = j00 * G.W[j] + j02 * G.W[6 + j];
        G.T[3 + j] = j11 * G.W[3 + j] + j12 * G.W[6 + j];
    }
    const float *S = G.Sig;
    // rows of T times Sigma
    float t0[3], t1[3];
    t0[0] = G.T[0] * S[0] + G.T[1] * S[1] + G.T[2] * S[2];
    t0[1] = G.T[0] * S[1] + G.T[1] * S[3] + G.T[2] * S[4];
    t0[2] = G.T[0] * S[2] + G.T[1] * S[4] + G.T[2] * S[5];
    t1[0] = G.T[3] * S[0] + G.T[4] * S[1] + G.T[5] * S[2];
    t1[1] = G.T[3] * S[1] + G.T[4] * S[3] + G.T[5] * S[4];
    t1[2] = G.T[3] * S[2] + G.T[4] * S[4] + G.T[5] * S[5];
    G.A = t0[0] * G.T[0] + t0[1] * G.T[1] + t0[2] * G.T[2] + bp.dilation;
    G.B = t0[0] * G.T[3] + t0[1] * G.T[4] + t0[2] * G.T[5];
    G.C = t1[0] * G.T[3] + t1[1] * G.T[4] + t1[2] * G.T[5] + bp.dilation;
}

// The alpha >= alpha_min ellipse q(d) = a dx^2 + 2 b dx dy + c dy^2 <= k2,
// k2 = 2 ln(o / alpha_min), of a projected Gaussian at (u, v), conic (a, b, c).
// Tile decisions use a margin so that FP32 rounding never drops a tile the
// blend uses: k2 grown by kMarginQ (relative) and every tile's box of pixel
// centres grown by kMarginPx on each side; the rectangle is the box of that
// grown ellipse, grown by kMarginPx.  A list may thus hold, besides the exact
// tiles, tiles whose box the exact ellipse misses by less than the margin.
constexpr float kMarginQ = 1e-4f;
constexpr float kMarginPx = 1e-3f;

struct Ellipse {
    float u, v, a, b, k2, detc, ry, dyr;
};

__device__ __forceinline__ Ellipse ellipse_of(float4 xo, float4 cn, float alpha_min) {
    Ellipse e;
    e.u = xo.x;
    e.v = xo.y;
    e.a = cn.x;
    e.b = cn.y;
    // a relative margin so FP32 rounding never drops a tile the blend uses
    e.k2 = 2.f * logf(xo.w / alpha_min) * (1.f + kMarginQ);
    e.detc = cn.x * cn.z - cn.y * cn.y;
    e.ry = sqrtf(e.k2 * cn.x / e.detc);               // half-extent in y
    e.dyr = -cn.y * sqrtf(e.k2 / (cn.z * e.detc));    // dy of the point of largest x
    return e;
}

// Tile columns [c0, c1] of tile row ty (clipped to the rect's columns
// [x0, x1]; c0 > c1: none) whose box of pixel centres the ellipse meets.  The
// ellipse's slice through the row's band of pixel centres is an x interval;
// its ends are the right-most and left-most boundary points, whose dy is the
// unconstrained extreme clamped to the band (the boundary's x is concave /
// convex in dy).
__device__ __forceinline__ int2 row_cols(const Ellipse &e, int ty, int W, int H, int x0, int x1) {
    const float yb0 = (float)(ty * kTile) - kMarginPx,
                yb1 = fminf((float)(ty * kTile + kTile - 1), (float)(H - 1)) + kMarginPx;
    const float lo = fmaxf(yb0 - e.v, -e.ry), hi = fminf(yb1 - e.v, e.ry);
    if (!(lo <= hi)) return make_int2(1, 0);
    const float dr = fminf(fmaxf(e.dyr, lo), hi), dl = fminf(fmaxf(-e.dyr, lo), hi);
    const float ia = 1.f / e.a;
    const float xr = (-e.b * dr + sqrtf(fmaxf(e.a * e.k2 - e.detc * dr * dr, 0.f))) * ia;
    const float xl = (-e.b * dl - sqrtf(fmaxf(e.a * e.k2 - e.detc * dl * dl, 0.f))) * ia;
    const float xlo = fmaxf(e.u + xl - kMarginPx, 0.f), xhi = fminf(e.u + xr + kMarginPx, (float)(W - 1));
    if (!(xlo <= xhi)) return make_int2(1, 0);
    // tile tx holds pixel centres [16 tx, 16 tx + 15]: the first whose box
    // reaches xlo, the last whose box starts at or before xhi
    return make_int2(max((int)ceilf((xlo - (float)(kTile - 1)) * (1.f / kTile)), x0),
                     min((int)floorf(xhi * (1.f / kTile)), x1));
}

__global__ void __launch_bounds__(256) k_project(
    ViewTable vt, BlendParams bp, int N, int per_view, int total,
    const float4 *__restrict__ mean_op, const float4 *__restrict__ scale,
    const float4 *__restrict__ quat, float4 *__restrict__ xyzo, float4 *__restrict__ conic,
    uint2 *__restrict__ rect, uint32_t *__restrict__ count, uint64_t *__restrict__ dkey,
    uint32_t *__restrict__ dval, uint32_t *__restrict__ dkey32, int vbits32) {
    int gv = blockIdx.x * blockDim.x + threadIdx.x;
    if (gv >= total) return;
    int v = gv / N;
    const DevView &cam = vt.v[v];
    int gs = cam.set * N + (gv - v * N);
    float4 m = mean_op[gs];
    Geo G;
    bool ok = camera_point(cam, bp, m, G.p);
    uint32_t cnt = 0;
    uint2 rc = make_uint2(0u, 0u);
    float4 xo = make_float4(0.f, 0.f, G.p[2], m.w);
    float4 cn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ok) {
        covariance(cam, bp, scale[gs], quat[gs], G);
        float det = G.A * G.C - G.B * G.B;
        float idet = 1.f / det;
        cn = make_float4(G.C * idet, -G.B * idet, G.A * idet, 0.f);
        float iz = 1.f / G.p[2];
        float u = fmaf(cam.fx * G.p[0], iz, cam.cx);
        float vv = fmaf(cam.fy * G.p[1], iz, cam.cy);
        xo.x = u;
        xo.y = vv;
        // bounding box of the ellipse o exp(-q/2) >= alpha_min, with the
        // margin of the tile decisions
        float k2 = 2.f * logf(m.w / bp.alpha_min) * (1.f + kMarginQ);
        float rx = sqrtf(k2 * G.A) + kMarginPx, ry = sqrtf(k2 * G.C) + kMarginPx;
        float xlo = fmaxf(u - rx, 0.f), xhi = fminf(u + rx, (float)(cam.W - 1));
        float ylo = fmaxf(vv - ry, 0.f), yhi = fminf(vv + ry, (float)(cam.H - 1));
        if (xlo <= xhi && ylo <= yhi) {
            int x0 = (int)floorf(xlo * (1.f / kTile)), x1 = (int)floorf(xhi * (1.f / kTile));
            int y0 = (int)floorf(ylo * (1.f / kTile)), y1 = (int)floorf(yhi * (1.f / kTile));
            // tiles of the rect that the ellipse meets (same arithmetic as k_emit)
            const Ellipse e = ellipse_of(xo, cn, bp.alpha_min);
            for (int ty = y0; ty <= y1; ++ty) {
                const int2 cc = row_cols(e, ty, cam.W, cam.H, x0, x1);
                if (cc.x <= cc.y) cnt += (uint32_t)(cc.y - cc.x + 1);
            }
            rc = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
        }
    }
    xyzo[gv] = xo;
    conic[gv] = cn;
    rect[gv] = rc;
    count[gv] = cnt;
    if (vbits32 < 0) {
        uint32_t zb = cnt ? __float_as_uint(G.p[2]) : 0xffffffffu;
        dkey[gv] = ((uint64_t)v << 32) | zb;
    } else {
        // 32-bit key: view in the top vbits32 bits, float bits of z above
        // 0.125 m below (exact while z < 2^(32 - vbits32) ulps above 0.125 m;
        // larger depths saturate and fall back to id order)
        const uint32_t zmask = vbits32 == 0 ? 0xffffffffu : (0xffffffffu >> vbits32);
        uint32_t zf = zmask;
        if (cnt) zf = min(__float_as_uint(G.p[2]) - 0x3e000000u, zmask);
        dkey32[gv] = (vbits32 == 0 ? 0u : ((uint32_t)v << (32 - vbits32))) | zf;
    }
    dval[gv] = (uint32_t)gv;
}

__global__ void k_gather_counts(const uint32_t *__restrict__ sorted_gv,
                                const uint32_t *__restrict__ count, uint32_t *__restrict__ out,
                                int total) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < total) out[s] = count[sorted_gv[s]];
}

// Instances of 32 consecutive depth-ordered Gaussian-views are written by one
// warp: the warp walks its contiguous instance range 32 at a time, each lane
// finds its source Gaussian by a binary search over the lanes' start offsets,
// so stores are coalesced whatever the per-Gaussian tile counts are.  Each
// owner lane first tabulates its Gaussian's met columns per tile row (first
// column and running instance count) in shared memory, up to kEmitRows rows;
// taller Gaussians (rare) recompute the rows per instance.
constexpr int kEmitRows = 8;

__global__ void __launch_bounds__(256) k_emit(ViewTable vt, BlendParams bp, int N, int total,
                                              const uint32_t *__restrict__ sorted_gv,
                                              const uint64_t *__restrict__ off,
                                              const uint2 *__restrict__ rect,
                                              const float4 *__restrict__ xyzo,
                                              const float4 *__restrict__ conic,
                                              uint32_t *__restrict__ ikey,
                                              uint32_t *__restrict__ ival) {
    __shared__ uint32_t s_rows[256 / 32][32][kEmitRows];  // first column | (instances before the row << 16)
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int s0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
    if (s0 >= total) return;  // warp-uniform
    const int s = s0 + lane;
    const bool in = s < total;
    const uint64_t o = off[in ? s : total];
    const uint64_t o_end = off[min(s0 + 32, total)];
    const uint64_t o_beg = __shfl_sync(full, o, 0);
    uint32_t gv = in ? sorted_gv[s] : 0u;
    uint2 rc = make_uint2(0u, 0u);
    float4 xo = make_float4(0.f, 0.f, 0.f, 1.f), cn = make_float4(1.f, 0.f, 1.f, 0.f);
    const bool mine = in && off[s + 1] > o;
    if (mine) {
        rc = rect[gv];
        xo = xyzo[gv];
        cn = conic[gv];
        const int v = (int)(gv / (uint32_t)N);
        const DevView &cam = vt.v[v];
        const int x0 = rc.x & 0xffff, y0 = rc.x >> 16, x1 = rc.y & 0xffff, y1 = rc.y >> 16;
        if (y1 - y0 < kEmitRows) {
            const Ellipse e = ellipse_of(xo, cn, bp.alpha_min);
            uint32_t before = 0;
            for (int r = y0; r <= y1; ++r) {
                const int2 cc = row_cols(e, r, cam.W, cam.H, x0, x1);
                s_rows[wid][lane][r - y0] = (uint32_t)max(cc.x, 0) | (before << 16);
                if (cc.x <= cc.y) before += (uint32_t)(cc.y - cc.x + 1);
            }
        }
    }
    __syncwarp();
    for (uint64_t b = o_beg; b < o_end; b += 32) {
        const uint64_t i = b + lane;
        int L = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            uint64_t oc = __shfl_sync(full, o, L + step);
            if (oc <= i) L += step;
        }
        const uint32_t g = __shfl_sync(full, gv, L);
        const uint32_t r0 = __shfl_sync(full, rc.x, L);
        const uint32_t r1 = __shfl_sync(full, rc.y, L);
        const uint64_t oL = __shfl_sync(full, o, L);
        if (i < o_end) {
            const int v = (int)(g / (uint32_t)N);
            const DevView &cam = vt.v[v];
            const int x0 = r0 & 0xffff, y0 = r0 >> 16, x1 = r1 & 0xffff, y1 = r1 >> 16;
            const int j = (int)(i - oL);
            int tx = x0, ty = y0;
            if (y1 - y0 < kEmitRows) {
                // last tabulated row whose running count is <= j
                int r = 0;
                for (int k = 1; k <= y1 - y0; ++k)
                    if ((int)(s_rows[wid][L][k] >> 16) <= j) r = k;
                const uint32_t e = s_rows[wid][L][r];
                tx = (int)(e & 0xffff) + j - (int)(e >> 16);
                ty = y0 + r;
            } else {
                const Ellipse e = ellipse_of(xyzo[g], conic[g], bp.alpha_min);
                int jj = j;
                for (int r = y0; r <= y1; ++r) {
                    const int2 cc = row_cols(e, r, cam.W, cam.H, x0, x1);
                    const int n = cc.x <= cc.y ? cc.y - cc.x + 1 : 0;
                    if (jj < n) {
                        tx = cc.x + jj;
                        ty = r;
                        break;
                    }
                    jj -= n;
                }
            }
            ikey[i] = (uint32_t)(cam.tile_base + ty * cam.tiles_x + tx);
            ival[i] = g;
        }
    }
}

__global__ void k_ranges(const uint32_t *__restrict__ ikey, uint32_t n, uint2 *__restrict__ ranges) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = ikey[i];
    if (i == 0 || ikey[i - 1] != k) ranges[k].x = i;
    if (i == n - 1 || ikey[i + 1] != k) ranges[k].y = i + 1;
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_project_bwd(
    ViewTable vt, BlendParams bp, int N, int direct, int total, int n_feat, unsigned mask,
    float scale_grad, const float4 *__restrict__ mean_op, const float4 *__restrict__ scale,
    const float4 *__restrict__ quat, const float *__restrict__ g2, float4 *__restrict__ d_mean_op,
    float4 *__restrict__ d_scale, float4 *__restrict__ d_quat, float4 *__restrict__ d_color,
    float *__restrict__ d_feat, float *__restrict__ d_pose) {
    int gv = blockIdx.x * blockDim.x + threadIdx.x;
    bool in = gv < total;
    int v = in ? gv / N : vt.n - 1;
    // direct: every set is read by one view, so its gradient is written, not
    // accumulated (else the caller zeroed the gradient and views add into it)
    int gs = vt.v[v].set * N + (gv - v * N);
    float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (in) {
        const DevView &cam = vt.v[v];
        float4 m = mean_op[gs];
        Geo G;
        bool ok = camera_point(cam, bp, m, G.p);
        const int stride = g2_stride(n_feat);
        const float *r = g2 + (size_t)gv * stride;
        float dmu[3] = {0.f, 0.f, 0.f}, ds[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
        float dop = 0.f;
        if (ok) {
            covariance(cam, bp, scale[gs], quat[gs], G);
            float4 ra = *reinterpret_cast<const float4 *>(r);
            float4 rb = *reinterpret_cast<const float4 *>(r + 4);
            float gu = ra.x, gvv = ra.y, gz = ra.z;
            dop = ra.w;
            float ga = rb.x, gb = rb.y, gc = rb.z;
            float A = G.A, B = G.B, Cc = G.C;
            float D = A * Cc - B * B;
            float iD2 = 1.f / (D * D);
            float gA = (-Cc * Cc * ga + B * Cc * gb - B * B * gc) * iD2;
            float gB = (2.f * B * Cc * ga - (A * Cc + B * B) * gb + 2.f * A * B * gc) * iD2;
            float gC = (-B * B * ga + B * A * gb - A * A * gc) * iD2;
            // G2 = [[gA, gB/2], [gB/2, gC]]; Sigma' = T Sigma T^T
            float h = 0.5f * gB;
            const float *T = G.T;
            const float *S = G.Sig;
            // G2 T (2x3)
            float gt0[3], gt1[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                gt0[j] = gA * T[j] + h * T[3 + j];
                gt1[j] = h * T[j] + gC * T[3 + j];
            }
            // dL/dSigma = T^T G2 T (symmetric 3x3, full)
            float GS[9];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) GS[3 * i + j] = T[i] * gt0[j] + T[3 + i] * gt1[j];
            // dL/dT = 2 G2 T Sigma
            float Sf[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
            float GT[6];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                GT[j] = 2.f * (gt0[0] * Sf[j] + gt0[1] * Sf[3 + j] + gt0[2] * Sf[6 + j]);
                GT[3 + j] = 2.f * (gt1[0] * Sf[j] + gt1[1] * Sf[3 + j] + gt1[2] * Sf[6 + j]);
            }
            // T = J W: dL/dJ = GT W^T, dL/dW(cov) = J^T GT
            const float *W = G.W;
            float GJ[6];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    GJ[3 * a + j] = GT[3 * a] * W[3 * j] + GT[3 * a + 1] * W[3 * j + 1] +
                                    GT[3 * a + 2] * W[3 * j + 2];
            float iz = 1.f / G.p[2], iz2 = iz * iz, iz3 = iz2 * iz;
            float fx = cam.fx, fy = cam.fy;
            float gp[3];
            gp[0] = GJ[2] * (-fx * iz2) + gu * fx * iz;
            gp[1] = GJ[5] * (-fy * iz2) + gvv * fy * iz;
            gp[2] = GJ[0] * (-fx * iz2) + GJ[2] * (2.f * fx * G.p[0] * iz3) + GJ[4] * (-fy * iz2) +
                    GJ[5] * (2.f * fy * G.p[1] * iz3) - gu * fx * G.p[0] * iz2 -
                    gvv * fy * G.p[1] * iz2 + gz;
#pragma unroll
            for (int i = 0; i < 3; ++i) dmu[i] = W[i] * gp[0] + W[3 + i] * gp[1] + W[6 + i] * gp[2];
            if (mask & UPS_GRAD_POSE) {
                // dW(cov) = J^T GT; J = [[j00 0 j02][0 j11 j12]]
                float j00 = fx * iz, j02 = -fx * G.p[0] * iz2, j11 = fy * iz, j12 = -fy * G.p[1] * iz2;
                float GW[9];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    GW[j] = j00 * GT[j];
                    GW[3 + j] = j11 * GT[3 + j];
                    GW[6 + j] = j02 * GT[j] + j12 * GT[3 + j];
                }
                // A = W GW^T; d phi += vee(A)
                float Am[9];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        Am[3 * i + j] = W[3 * i] * GW[3 * j] + W[3 * i + 1] * GW[3 * j + 1] +
                                        W[3 * i + 2] * GW[3 * j + 2];
                const float *p = G.p;
                pose[0] = gp[0];
                pose[1] = gp[1];
                pose[2] = gp[2];
                pose[3] = p[1] * gp[2] - p[2] * gp[1] + Am[5] - Am[7];
                pose[4] = p[2] * gp[0] - p[0] * gp[2] + Am[6] - Am[2];
                pose[5] = p[0] * gp[1] - p[1] * gp[0] + Am[1] - Am[3];
            }
            if (mask & UPS_GRAD_GAUSS) {
                // Sigma = (R S)(R S)^T: dL/d(RS) = 2 GS (R S)
                float GR[9];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float acc = 0.f;
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        float grs = 2.f * (GS[3 * i] * G.Rq[j] * G.s[j] + GS[3 * i + 1] * G.Rq[3 + j] * G.s[j] +
                                           GS[3 * i + 2] * G.Rq[6 + j] * G.s[j]);
                        GR[3 * i + j] = grs * G.s[j];
                        acc += grs * G.Rq[3 * i + j];
                    }
                    ds[j] = acc;
                }
                float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
                float dqn[4];
                dqn[0] = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
                dqn[1] = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] +
                                z * GR[6] + w * GR[7] - 2.f * x * GR[8]);
                dqn[2] = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] -
                                w * GR[6] + z * GR[7] - 2.f * y * GR[8]);
                dqn[3] = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] +
                                y * GR[5] + x * GR[6] + y * GR[7]);
                float dot = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
#pragma unroll
                for (int i = 0; i < 4; ++i) dq[i] = (dqn[i] - G.qn[i] * dot) * G.qinv;
            }
        }
        if (mask & UPS_GRAD_GAUSS) {
            // the mean-scale term enters each set's scale gradient once
            float sreg = vt.v[v].set_first ? scale_grad : 0.f;
            float4 rc = *reinterpret_cast<const float4 *>(r + 8);  // dr dg db -
            if (direct) {
                d_mean_op[gs] = make_float4(dmu[0], dmu[1], dmu[2], dop);
                d_scale[gs] = make_float4(ds[0] + sreg, ds[1] + sreg, ds[2] + sreg, 0.f);
                d_quat[gs] = make_float4(dq[0], dq[1], dq[2], dq[3]);
                d_color[gs] = make_float4(rc.x, rc.y, rc.z, 0.f);
                // feature gradients as 16-byte moves (n_feat is a multiple of 4; the
                // record's feature part starts 48 bytes into a 16-byte aligned record)
                const float4 *rf = reinterpret_cast<const float4 *>(r + kG2Base);
                float4 *df = reinterpret_cast<float4 *>(d_feat + (size_t)gs * n_feat);
                for (int c = 0; c < n_feat / 4; ++c) df[c] = rf[c];
            } else {
                float *dm = reinterpret_cast<float *>(d_mean_op + gs);
                float *dsc = reinterpret_cast<float *>(d_scale + gs);
                float *dqq = reinterpret_cast<float *>(d_quat + gs);
                float *dc = reinterpret_cast<float *>(d_color + gs);
                if (ok) {
                    atomicAdd(dm + 0, dmu[0]);
                    atomicAdd(dm + 1, dmu[1]);
                    atomicAdd(dm + 2, dmu[2]);
                    atomicAdd(dm + 3, dop);
                    atomicAdd(dsc + 0, ds[0]);
                    atomicAdd(dsc + 1, ds[1]);
                    atomicAdd(dsc + 2, ds[2]);
                    for (int i = 0; i < 4; ++i) atomicAdd(dqq + i, dq[i]);
                    atomicAdd(dc + 0, rc.x);
                    atomicAdd(dc + 1, rc.y);
                    atomicAdd(dc + 2, rc.z);
                    for (int c = 0; c < n_feat; ++c) atomicAdd(d_feat + (size_t)gs * n_feat + c, r[kG2Base + c]);
                }
                if (sreg != 0.f) {
                    atomicAdd(dsc + 0, sreg);
                    atomicAdd(dsc + 1, sreg);
                    atomicAdd(dsc + 2, sreg);
                }
            }
        }
    }
    if (!(mask & UPS_GRAD_POSE)) return;
    // pose: one reduction per block when the block holds a single view, else
    // per warp (or per lane when a warp straddles two views)
    __shared__ float red[8][6];
    __shared__ int vblock;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v0 = __shfl_sync(full, v, 0);
    bool wsame = __all_sync(full, v == v0);
    if (!wsame) {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (in && pose[i] != 0.f) atomicAdd(d_pose + 6 * v + i, pose[i]);
            pose[i] = 0.f;
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pose[i] += __shfl_xor_sync(full, pose[i], o);
    if (threadIdx.x == 0) vblock = v;
    __syncthreads();
    bool bsame = __syncthreads_and(v == vblock);
    if (bsame) {
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < 6; ++i) red[w][i] = pose[i];
        __syncthreads();
        if (threadIdx.x < 6) {
            float s = 0.f;
            for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) s += red[ww][threadIdx.x];
            atomicAdd(d_pose + 6 * vblock + threadIdx.x, s);
        }
    } else if (lane == 0 && wsame) {
#pragma unroll
        for (int i = 0; i < 6; ++i) atomicAdd(d_pose + 6 * v0 + i, pose[i]);
    }
}

}  // namespace

cudaError_t launch_project(const ViewTable &vt, const BlendParams &bp, int N, int per_view,
                           int total, const ups_gaussians &g, float4 *xyzo, float4 *conic,
                           uint2 *rect, uint32_t *count, uint64_t *dkey, uint32_t *dval,
                           cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    k_project<<<(total + 255) / 256, 256, 0, st>>>(
        vt, bp, N, per_view, total, reinterpret_cast<const float4 *>(g.mean_opacity),
        reinterpret_cast<const float4 *>(g.scale), reinterpret_cast<const float4 *>(g.quat), xyzo,
        conic, rect, count, dkey, dval, nullptr, -1);
    return cudaGetLastError();
}

// Projection writing 32-bit (view, depth) keys (vbits = bits of the view index).
cudaError_t launch_project_k32(const ViewTable &vt, const BlendParams &bp, int N, int per_view,
                               int total, const ups_gaussians &g, float4 *xyzo, float4 *conic,
                               uint2 *rect, uint32_t *count, uint32_t *dkey32, uint32_t *dval,
                               int vbits, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    k_project<<<(total + 255) / 256, 256, 0, st>>>(
        vt, bp, N, per_view, total, reinterpret_cast<const float4 *>(g.mean_opacity),
        reinterpret_cast<const float4 *>(g.scale), reinterpret_cast<const float4 *>(g.quat), xyzo,
        conic, rect, count, nullptr, dval, dkey32, vbits);
    return cudaGetLastError();
}

cudaError_t launch_gather_counts(const uint32_t *sorted_gv, const uint32_t *count, uint32_t *out,
                                 int total, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    k_gather_counts<<<(total + 255) / 256, 256, 0, st>>>(sorted_gv, count, out, total);
    return cudaGetLastError();
}

cudaError_t launch_emit(const ViewTable &vt, const BlendParams &bp, int N, int total, const uint32_t *sorted_gv,
                        const uint64_t *off, const uint2 *rect, const float4 *xyzo, const float4 *conic,
                        uint32_t *ikey, uint32_t *ival, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    k_emit<<<(total + 255) / 256, 256, 0, st>>>(vt, bp, N, total, sorted_gv, off, rect, xyzo, conic, ikey, ival);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t *ikey, uint32_t n, uint2 *ranges, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_ranges<<<(n + 255) / 256, 256, 0, st>>>(ikey, n, ranges);
    return cudaGetLastError();
}

cudaError_t launch_project_bwd(const ViewTable &vt, const BlendParams &bp, int N, int per_view,
                               int total, int n_feat, unsigned mask, float scale_grad,
                               const ups_gaussians &g, const float *g2, const ups_gaussians *grad,
                               float *d_pose, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    float4 *dm = nullptr, *ds = nullptr, *dq = nullptr, *dc = nullptr;
    float *df = nullptr;
    if (grad && (mask & UPS_GRAD_GAUSS)) {
        dm = reinterpret_cast<float4 *>(grad->mean_opacity);
        ds = reinterpret_cast<float4 *>(grad->scale);
        dq = reinterpret_cast<float4 *>(grad->quat);
        dc = reinterpret_cast<float4 *>(grad->color);
        df = grad->feat;
    }
    k_project_bwd<<<(total + 255) / 256, 256, 0, st>>>(
        vt, bp, N, per_view, total, n_feat, mask, scale_grad,
        reinterpret_cast<const float4 *>(g.mean_opacity), reinterpret_cast<const float4 *>(g.scale),
        reinterpret_cast<const float4 *>(g.quat), g2, dm, ds, dq, dc, df, d_pose);
    return cudaGetLastError();
}

}  // namespace ups
