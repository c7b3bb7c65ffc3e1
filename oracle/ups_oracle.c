/*
 * FP64 CPU oracle of the anchor-decoded differentiable Gaussian render path
 * (UP-SLAM, arXiv 2505.22335, Sec. 3.1 and Sec. 3.3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: it is used by the test suite, by the smoke check and by the CPU
 * baseline leg of the benchmark.  It shares no code, header, table or constant
 * generator with the CUDA library; settings (thresholds, sizes) are passed in
 * as plain values.
 *
 * Every function works on ONE view and plain arrays of doubles.  Loops follow
 * the definitions in the paper's order with no blocking or fusion:
 *
 *   orc_decode_view      Eq. 8-9  per-anchor MLP decode into K Gaussians
 *   orc_project_view     Eq. 1-2  covariance R S S^T R^T, EWA projection
 *   orc_render_view      Eq. 3, Eq. 10  front-to-back alpha blending
 *   orc_loss_view        Eq. 4 / Eq. 14 per-pixel weighted image loss
 *   orc_render_bwd_view  derivative of Eq. 3 / Eq. 10 w.r.t. the 2D Gaussians
 *   orc_project_bwd_view derivative of Eq. 1-2 w.r.t. mean, scale, rotation, pose
 *   orc_decode_bwd_view  derivative of Eq. 8-9 w.r.t. MLP weights, anchors, pose
 *
 * Readings of points the paper leaves open (all passed in by the caller):
 *  - alpha_i(p) = min(alpha_max, o_i exp(-1/2 d^T Sigma'^-1 d)), skipped if
 *    below alpha_min; a pixel stops BEFORE the Gaussian that would take its
 *    transmittance below t_min;
 *  - Sigma' gets `dilation` added on its diagonal; pixel (i, j) is sampled at
 *    continuous coordinate (i, j) with u = fx X/Z + cx; background is zero;
 *  - W in Eq. 2 is the rotation of T_cw = T_wc^-1 and J is the Jacobian of the
 *    pinhole projection at the camera-space mean;
 *  - a Gaussian is culled when Z <= near_z, |X/Z| > guard*W/(2 fx) (same in y),
 *    or o < alpha_min;
 *  - the tile rectangle of a Gaussian is the axis-aligned bounding box of the
 *    ellipse where o exp(-q/2) >= alpha_min, clipped to the image; a tile of
 *    the rectangle lists the Gaussian when that ellipse meets the tile's box of
 *    pixel centres (the minimum of q over the box is at most 2 ln(o/alpha_min)),
 *    so the tiled render equals the all-pairs render exactly;
 *  - depth order is ascending (float32(z), Gaussian id).
 *
 * Pose perturbation: T_cw(xi) = Exp(xi) T_cw, xi = (rho, phi), evaluated at
 * xi = 0; gradients are returned as [d rho (3), d phi (3)].
 *
 * The gradients are the analytic derivatives of these definitions; the test
 * suite pins them against central finite differences of the loss.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double fx, fy, cx, cy;
    int width, height;
    double Tcw[16]; /* row-major world-to-camera */
} orc_camera;

typedef struct {
    double alpha_min, alpha_max, t_min, dilation, near_z, guard;
    int tile;  /* tile edge in pixels */
    int brute; /* 1: every valid Gaussian for every pixel (no tile lists) */
} orc_cfg;

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }
static double softplus(double x) { return x > 30.0 ? x : log1p(exp(x)); }

static void camera_centre(const double *T, double *oc)
{
    /* o_c = -R^T t */
    for (int i = 0; i < 3; ++i)
        oc[i] = -(T[0 * 4 + i] * T[3] + T[1 * 4 + i] * T[7] + T[2 * 4 + i] * T[11]);
}

/* rotation of a unit quaternion (w, x, y, z) */
static void quat_to_rot(const double *q, double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z);
    R[0][1] = 2 * (x * y - w * z);
    R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);
    R[1][1] = 1 - 2 * (x * x + z * z);
    R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);
    R[2][1] = 2 * (y * z + w * x);
    R[2][2] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------ */
/* Eq. 8-9: decode                                                          */
/* ------------------------------------------------------------------------ */

/* Row group of output row r: 0 opacity (K rows), 1 covariance (7K), 2 colour
 * (3K), 3 feature (K*NL).  Group g reads hidden units [g*H, (g+1)*H). */
static int out_group(int r, int K)
{
    if (r < K) return 0;
    if (r < 8 * K) return 1;
    if (r < 11 * K) return 2;
    return 3;
}

/* MLP input x = [f_v (F), delta_vc (3), d_vc (1), sin(pi t), cos(pi t)]. */
static void decode_input(int F, const double *pos, const double *feat, const double *oc,
                         double t_norm, double *x, double *delta, double *dist)
{
    double r[3] = {pos[0] - oc[0], pos[1] - oc[1], pos[2] - oc[2]};
    double d = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int i = 0; i < F; ++i) x[i] = feat[i];
    for (int i = 0; i < 3; ++i) {
        delta[i] = r[i] / d;
        x[F + i] = delta[i];
    }
    *dist = d;
    x[F + 3] = d;
    x[F + 4] = sin(M_PI * t_norm);
    x[F + 5] = cos(M_PI * t_norm);
}

/* hidden pre-activations z and activations h (ReLU for groups 0-2, SoftPlus
 * for the feature decoder F_d), then output rows y. */
static void decode_mlp(int K, int F, int H, int NL, const double *W1, const double *b1,
                       const double *W2, const double *b2, const double *x, double *z,
                       double *h, double *y)
{
    int din = F + 6;
    int nout = K * (11 + NL);
    for (int j = 0; j < 4 * H; ++j) {
        double acc = b1[j];
        for (int i = 0; i < din; ++i) acc += W1[j * din + i] * x[i];
        z[j] = acc;
        h[j] = (j < 3 * H) ? (acc > 0 ? acc : 0.0) : softplus(acc);
    }
    for (int r = 0; r < nout; ++r) {
        int g = out_group(r, K);
        double acc = b2[r];
        for (int j = 0; j < H; ++j) acc += W2[r * H + j] * h[g * H + j];
        y[r] = acc;
    }
}

/* Opacity activation: sigmoid, or with op_tanh the Scaffold-GS form o = tanh(y)
 * (the decode the paper cites), whose Gaussians with o <= 0 the projection
 * drops (o < alpha_min is culled there; with alpha_min = 0, o = 0 blends as
 * zero alpha). */
void orc_decode_view(int A, int K, int F, int H, int NL, int op_tanh, const double *anc_pos,
                     const double *anc_feat, const double *anc_off, const double *anc_scale,
                     const double *W1, const double *b1, const double *W2, const double *b2,
                     const orc_camera *cam, double t_norm, double *mean, double *opac,
                     double *scale, double *quat, double *color, double *feat)
{
    double oc[3];
    camera_centre(cam->Tcw, oc);
    int nout = K * (11 + NL);
#pragma omp parallel
    {
        double *x = malloc(sizeof(double) * (F + 6));
        double *z = malloc(sizeof(double) * 4 * H);
        double *h = malloc(sizeof(double) * 4 * H);
        double *y = malloc(sizeof(double) * nout);
#pragma omp for schedule(static)
        for (int a = 0; a < A; ++a) {
            double delta[3], dist;
            decode_input(F, anc_pos + 3 * a, anc_feat + (size_t)F * a, oc, t_norm, x, delta, &dist);
            decode_mlp(K, F, H, NL, W1, b1, W2, b2, x, z, h, y);
            for (int k = 0; k < K; ++k) {
                size_t g = (size_t)a * K + k;
                for (int i = 0; i < 3; ++i)
                    mean[3 * g + i] = anc_pos[3 * a + i] + anc_off[3 * g + i];
                opac[g] = op_tanh ? tanh(y[k]) : sigmoid(y[k]);
                for (int i = 0; i < 3; ++i)
                    scale[3 * g + i] = anc_scale[3 * a + i] * sigmoid(y[K + 7 * k + i]);
                for (int i = 0; i < 4; ++i) quat[4 * g + i] = y[K + 7 * k + 3 + i];
                for (int i = 0; i < 3; ++i) color[3 * g + i] = sigmoid(y[8 * K + 3 * k + i]);
                for (int i = 0; i < NL; ++i) feat[(size_t)NL * g + i] = y[11 * K + NL * k + i];
            }
        }
        free(x);
        free(z);
        free(h);
        free(y);
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 1-2: projection                                                      */
/* ------------------------------------------------------------------------ */

/* Outputs per Gaussian:
 *   valid[g]      1 if not culled
 *   pcam[3g..]    camera-space mean
 *   uv[2g..]      pixel position
 *   cov2d[3g..]   Sigma' (a, b, c) = [[a, b], [b, c]] including the dilation
 *   conic[3g..]   inverse of Sigma'
 *   rect[4g..]    tile rectangle tx0, ty0, tx1, ty1 (inclusive); tx0 > tx1 if empty
 *   extent[4g..]  clipped pixel-space extent xlo, ylo, xhi, yhi of the ellipse box
 */
void orc_project_view(int N, const double *mean, const double *opac, const double *scale,
                      const double *quat, const orc_camera *cam, const orc_cfg *cfg,
                      int *valid, double *pcam, double *uv, double *cov2d, double *conic,
                      int *rect, double *extent)
{
    const double *T = cam->Tcw;
    double W[3][3] = {{T[0], T[1], T[2]}, {T[4], T[5], T[6]}, {T[8], T[9], T[10]}};
    double t[3] = {T[3], T[7], T[11]};
    double limx = cfg->guard * 0.5 * cam->width / cam->fx;
    double limy = cfg->guard * 0.5 * cam->height / cam->fy;
    int ts = cfg->tile;
#pragma omp parallel for schedule(static)
    for (int g = 0; g < N; ++g) {
        const double *mu = mean + 3 * g;
        double p[3];
        for (int i = 0; i < 3; ++i) p[i] = W[i][0] * mu[0] + W[i][1] * mu[1] + W[i][2] * mu[2] + t[i];
        for (int i = 0; i < 3; ++i) pcam[3 * g + i] = p[i];
        rect[4 * g + 0] = 1;
        rect[4 * g + 1] = 1;
        rect[4 * g + 2] = 0;
        rect[4 * g + 3] = 0;
        valid[g] = 0;
        if (!(p[2] > cfg->near_z)) continue;
        if (fabs(p[0] / p[2]) > limx || fabs(p[1] / p[2]) > limy) continue;
        if (opac[g] < cfg->alpha_min) continue;
        valid[g] = 1;

        /* Sigma = R S S^T R^T with R from the normalised quaternion (Eq. 1) */
        double qn[4], qs = 0;
        for (int i = 0; i < 4; ++i) qs += quat[4 * g + i] * quat[4 * g + i];
        qs = sqrt(qs);
        for (int i = 0; i < 4; ++i) qn[i] = quat[4 * g + i] / qs;
        double R[3][3];
        quat_to_rot(qn, R);
        double S[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    acc += R[i][k] * scale[3 * g + k] * scale[3 * g + k] * R[j][k];
                S[i][j] = acc;
            }
        /* camera-frame covariance M = W Sigma W^T */
        double WS[3][3], M[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += W[i][k] * S[k][j];
                WS[i][j] = acc;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += WS[i][k] * W[j][k];
                M[i][j] = acc;
            }
        /* Eq. 2: Sigma' = J M J^T (+ dilation) */
        double z = p[2];
        double J[2][3] = {{cam->fx / z, 0, -cam->fx * p[0] / (z * z)},
                          {0, cam->fy / z, -cam->fy * p[1] / (z * z)}};
        double JM[2][3], C2[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += J[i][k] * M[k][j];
                JM[i][j] = acc;
            }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += JM[i][k] * J[j][k];
                C2[i][j] = acc;
            }
        double a = C2[0][0] + cfg->dilation, b = C2[0][1], c = C2[1][1] + cfg->dilation;
        double det = a * c - b * b;
        cov2d[3 * g + 0] = a;
        cov2d[3 * g + 1] = b;
        cov2d[3 * g + 2] = c;
        conic[3 * g + 0] = c / det;
        conic[3 * g + 1] = -b / det;
        conic[3 * g + 2] = a / det;
        double u = cam->fx * p[0] / z + cam->cx;
        double v = cam->fy * p[1] / z + cam->cy;
        uv[2 * g + 0] = u;
        uv[2 * g + 1] = v;

        /* bounding box of {d : o exp(-d^T Sigma'^-1 d / 2) >= alpha_min} */
        double rx, ry;
        if (cfg->alpha_min > 0) {
            double k2 = 2.0 * log(opac[g] / cfg->alpha_min);
            rx = sqrt(k2 * a);
            ry = sqrt(k2 * c);
        } else {
            rx = ry = INFINITY;
        }
        double xlo = fmax(u - rx, 0.0), xhi = fmin(u + rx, cam->width - 1.0);
        double ylo = fmax(v - ry, 0.0), yhi = fmin(v + ry, cam->height - 1.0);
        extent[4 * g + 0] = u - rx;
        extent[4 * g + 1] = v - ry;
        extent[4 * g + 2] = u + rx;
        extent[4 * g + 3] = v + ry;
        if (xlo > xhi || ylo > yhi) continue; /* empty: rect stays tx0 > tx1 */
        rect[4 * g + 0] = (int)floor(xlo / ts);
        rect[4 * g + 1] = (int)floor(ylo / ts);
        rect[4 * g + 2] = (int)floor(xhi / ts);
        rect[4 * g + 3] = (int)floor(yhi / ts);
    }
}

/* ------------------------------------------------------------------------ */
/* Depth order and tile lists                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    float z;
    int g;
} zkey;

static int zkey_cmp(const void *pa, const void *pb)
{
    const zkey *a = pa, *b = pb;
    if (a->z < b->z) return -1;
    if (a->z > b->z) return 1;
    return (a->g > b->g) - (a->g < b->g);
}

static int rect_ntiles(const int *r)
{
    if (r[0] > r[2] || r[1] > r[3]) return 0;
    return (r[2] - r[0] + 1) * (r[3] - r[1] + 1);
}

/* Minimum of q(d) = a dx^2 + 2 b dx dy + c dy^2 (a positive definite form)
 * over the box [dx0, dx1] x [dy0, dy1]: zero if the box holds the origin,
 * otherwise the smallest of the four edge minima (q restricted to an edge is a
 * 1D convex quadratic, minimised at its vertex clamped to the edge). */
static double box_min_q(double a, double b, double c, double dx0, double dx1, double dy0, double dy1)
{
    if (dx0 <= 0 && 0 <= dx1 && dy0 <= 0 && 0 <= dy1) return 0.0;
    double best = INFINITY;
    const double xs[2] = {dx0, dx1}, ys[2] = {dy0, dy1};
    for (int e = 0; e < 2; ++e) {
        double dx = xs[e];
        double dy = fmin(fmax(-b * dx / c, dy0), dy1);
        best = fmin(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy);
        dy = ys[e];
        dx = fmin(fmax(-b * dy / a, dx0), dx1);
        best = fmin(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy);
    }
    return best;
}

/* Whether tile (tx, ty) lists Gaussian g: the alpha >= alpha_min ellipse meets
 * the tile's box of pixel centres (clipped to the image). */
static int tile_hit(const double *uv, const double *conic, double opac, double alpha_min, int width,
                    int height, int ts, int tx, int ty)
{
    if (!(alpha_min > 0)) return 1;
    double k2 = 2.0 * log(opac / alpha_min);
    double x0 = tx * ts, x1 = fmin(tx * ts + ts - 1.0, width - 1.0);
    double y0 = ty * ts, y1 = fmin(ty * ts + ts - 1.0, height - 1.0);
    double q = box_min_q(conic[0], conic[1], conic[2], x0 - uv[0], x1 - uv[0], y0 - uv[1], y1 - uv[1]);
    return q <= k2;
}

/* Per-view tile lists: for each tile t (row-major), the Gaussians whose rect
 * covers t and whose ellipse meets it (tile_hit), in ascending (float32(z), g).
 * Writes list_g (concatenated over tiles) and ranges [2*t], [2*t+1] =
 * [start, end).  Returns the number of entries; list_g may be NULL to only
 * count. */
long orc_tile_lists(int N, const int *valid, const double *pcam, const int *rect, const double *uv,
                    const double *conic, const double *opac, double alpha_min, int width, int height,
                    int ts, int *list_g, int *ranges)
{
    int tiles_x = (width + ts - 1) / ts, tiles_y = (height + ts - 1) / ts;
    zkey *order = malloc(sizeof(zkey) * (N > 0 ? N : 1));
    int n = 0;
    for (int g = 0; g < N; ++g)
        if (valid[g] && rect_ntiles(rect + 4 * g) > 0) {
            order[n].z = (float)pcam[3 * g + 2];
            order[n].g = g;
            ++n;
        }
    qsort(order, n, sizeof(zkey), zkey_cmp);
    int T = tiles_x * tiles_y;
    long *count = calloc(T + 1, sizeof(long));
    for (int i = 0; i < n; ++i) {
        const int g = order[i].g;
        const int *r = rect + 4 * g;
        for (int ty = r[1]; ty <= r[3]; ++ty)
            for (int tx = r[0]; tx <= r[2]; ++tx)
                if (tile_hit(uv + 2 * g, conic + 3 * g, opac[g], alpha_min, width, height, ts, tx, ty))
                    count[ty * tiles_x + tx]++;
    }
    long total = 0;
    for (int t = 0; t < T; ++t) {
        long c = count[t];
        if (ranges) {
            ranges[2 * t] = (int)total;
            ranges[2 * t + 1] = (int)(total + c);
        }
        count[t] = total;
        total += c;
    }
    if (list_g) {
        for (int i = 0; i < n; ++i) { /* depth order kept within each tile */
            const int g = order[i].g;
            const int *r = rect + 4 * g;
            for (int ty = r[1]; ty <= r[3]; ++ty)
                for (int tx = r[0]; tx <= r[2]; ++tx)
                    if (tile_hit(uv + 2 * g, conic + 3 * g, opac[g], alpha_min, width, height, ts, tx, ty))
                        list_g[count[ty * tiles_x + tx]++] = g;
        }
    }
    free(count);
    free(order);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3 and Eq. 10: front-to-back blending                                 */
/* ------------------------------------------------------------------------ */

/* Per-pixel list of Gaussians to visit: the tile list (tiled mode) or every
 * valid Gaussian in depth order (brute mode). */
typedef struct {
    int *list;
    int *ranges; /* per tile, [start, end) into list */
    int *all;    /* brute: all valid Gaussians in depth order */
    int n_all;
} visit_lists;

static void build_visit(int N, const int *valid, const double *pcam, const int *rect, const double *uv,
                        const double *conic, const double *opac, const orc_camera *cam, const orc_cfg *cfg,
                        visit_lists *vl)
{
    int tiles_x = (cam->width + cfg->tile - 1) / cfg->tile;
    int tiles_y = (cam->height + cfg->tile - 1) / cfg->tile;
    memset(vl, 0, sizeof(*vl));
    if (cfg->brute) {
        zkey *order = malloc(sizeof(zkey) * (N > 0 ? N : 1));
        int n = 0;
        for (int g = 0; g < N; ++g)
            if (valid[g]) {
                order[n].z = (float)pcam[3 * g + 2];
                order[n].g = g;
                ++n;
            }
        qsort(order, n, sizeof(zkey), zkey_cmp);
        vl->all = malloc(sizeof(int) * (n > 0 ? n : 1));
        for (int i = 0; i < n; ++i) vl->all[i] = order[i].g;
        vl->n_all = n;
        free(order);
    } else {
        long total = orc_tile_lists(N, valid, pcam, rect, uv, conic, opac, cfg->alpha_min, cam->width,
                                    cam->height, cfg->tile, NULL, NULL);
        vl->list = malloc(sizeof(int) * (total > 0 ? total : 1));
        vl->ranges = malloc(sizeof(int) * 2 * tiles_x * tiles_y);
        orc_tile_lists(N, valid, pcam, rect, uv, conic, opac, cfg->alpha_min, cam->width, cam->height,
                       cfg->tile, vl->list, vl->ranges);
    }
}

static void pixel_list(const visit_lists *vl, const orc_camera *cam, const orc_cfg *cfg, int px,
                       int py, const int **list, int *n)
{
    if (cfg->brute) {
        *list = vl->all;
        *n = vl->n_all;
    } else {
        int tiles_x = (cam->width + cfg->tile - 1) / cfg->tile;
        int t = (py / cfg->tile) * tiles_x + (px / cfg->tile);
        *list = vl->list + vl->ranges[2 * t];
        *n = vl->ranges[2 * t + 1] - vl->ranges[2 * t];
    }
}

static void free_visit(visit_lists *vl)
{
    free(vl->list);
    free(vl->ranges);
    free(vl->all);
}

static double rel_gap(double a, double b) { return fabs(a - b) / fabs(b); }

/* Outputs (channel planes of one view, HxW each):
 *   out_color[3][H][W], out_depth[H][W], out_feat[NL][H][W], out_T[H][W] (final
 *   transmittance), out_nc[H][W] (list position of the last blended Gaussian
 *   + 1), out_margin[H][W] (smallest relative distance of any visited pair to
 *   the alpha_min / alpha_max / t_min thresholds; the FP32 path may decide such
 *   pairs differently). */
void orc_render_view(int N, int NL, const int *valid, const double *pcam, const double *uv,
                     const double *conic, const double *opac, const double *color,
                     const double *feat, const int *rect, const orc_camera *cam,
                     const orc_cfg *cfg, double *out_color, double *out_depth, double *out_feat,
                     double *out_T, int *out_nc, double *out_margin)
{
    visit_lists vl;
    build_visit(N, valid, pcam, rect, uv, conic, opac, cam, cfg, &vl);
    int Wd = cam->width, Ht = cam->height;
    size_t P = (size_t)Wd * Ht;
#pragma omp parallel for schedule(dynamic, 4)
    for (int py = 0; py < Ht; ++py) {
        double *F = malloc(sizeof(double) * (NL > 0 ? NL : 1));
        for (int px = 0; px < Wd; ++px) {
            const int *list;
            int n;
            pixel_list(&vl, cam, cfg, px, py, &list, &n);
            double T = 1.0, C[3] = {0, 0, 0}, D = 0, margin = INFINITY;
            for (int i = 0; i < NL; ++i) F[i] = 0;
            int last = 0;
            for (int idx = 0; idx < n; ++idx) {
                int g = list[idx];
                double dx = px - uv[2 * g], dy = py - uv[2 * g + 1];
                const double *cn = conic + 3 * g;
                double q = cn[0] * dx * dx + 2.0 * cn[1] * dx * dy + cn[2] * dy * dy;
                double raw = opac[g] * exp(-0.5 * q);
                double alpha = raw < cfg->alpha_max ? raw : cfg->alpha_max;
                if (cfg->alpha_min > 0) margin = fmin(margin, rel_gap(raw, cfg->alpha_min));
                margin = fmin(margin, rel_gap(raw, cfg->alpha_max));
                if (alpha < cfg->alpha_min) continue;
                double Tn = T * (1.0 - alpha);
                if (cfg->t_min > 0) margin = fmin(margin, rel_gap(Tn, cfg->t_min));
                if (Tn < cfg->t_min) break;
                double w = alpha * T;
                for (int ch = 0; ch < 3; ++ch) C[ch] += w * color[3 * g + ch];
                D += w * pcam[3 * g + 2];
                for (int ch = 0; ch < NL; ++ch) F[ch] += w * feat[(size_t)NL * g + ch];
                T = Tn;
                last = idx + 1;
            }
            size_t p = (size_t)py * Wd + px;
            for (int ch = 0; ch < 3; ++ch) out_color[ch * P + p] = C[ch];
            out_depth[p] = D;
            for (int ch = 0; ch < NL; ++ch) out_feat[ch * P + p] = F[ch];
            out_T[p] = T;
            out_nc[p] = last;
            if (out_margin) out_margin[p] = margin;
        }
        free(F);
    }
    free_visit(&vl);
}

/* ------------------------------------------------------------------------ */
/* Eq. 4 / Eq. 14: per-pixel weighted loss (image part)                     */
/* ------------------------------------------------------------------------ */

/* L_view = sum_p w_p [lc sum_ch l(C-Ct) + ld l(D-Dt) + lf sum_ch l(F-Ft)] / norm
 * with l = |.| (l2 = 0) or (.)^2 (l2 = 1).  Returns L_view and writes dL/d
 * of each rendered image (any gradient pointer may be NULL). */
double orc_loss_view(int Wd, int Ht, int NL, const double *color, const double *depth,
                     const double *feat, const double *t_color, const double *t_depth,
                     const double *t_feat, const double *weight, double lc, double ld, double lf,
                     int l2, double norm, double *g_color, double *g_depth, double *g_feat)
{
    size_t P = (size_t)Wd * Ht;
    double total = 0;
    for (size_t p = 0; p < P; ++p) {
        double w = weight ? weight[p] : 1.0;
        for (int k = 0; k < 3 + 1 + NL; ++k) {
            double r, lam;
            if (k < 3) {
                r = color[k * P + p] - t_color[k * P + p];
                lam = lc;
            } else if (k == 3) {
                r = depth[p] - t_depth[p];
                lam = ld;
            } else {
                r = feat[(k - 4) * P + p] - t_feat[(k - 4) * P + p];
                lam = lf;
            }
            double val = l2 ? r * r : fabs(r);
            double der = l2 ? 2.0 * r : (double)((r > 0) - (r < 0));
            total += w * lam * val / norm;
            double gr = w * lam * der / norm;
            if (k < 3) {
                if (g_color) g_color[k * P + p] = gr;
            } else if (k == 3) {
                if (g_depth) g_depth[p] = gr;
            } else if (g_feat) {
                g_feat[(k - 4) * P + p] = gr;
            }
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Backward of Eq. 3 / Eq. 10                                               */
/* ------------------------------------------------------------------------ */

/* Given dL/d(colour, depth, feature, final T) images, accumulate per-Gaussian
 * gradients: g_uv[2], g_conic[3] (a, b, c with q = a dx^2 + 2 b dx dy + c dy^2),
 * g_opac, g_color[3], g_z (depth value), g_feat[NL].  Uses the same visit
 * lists and threshold rules as the forward; per pixel it first replays the
 * forward, storing each blended Gaussian's alpha and transmittance, then walks
 * the stored list back to front. */
void orc_render_bwd_view(int N, int NL, const int *valid, const double *pcam, const double *uv,
                         const double *conic, const double *opac, const double *color,
                         const double *feat, const int *rect, const orc_camera *cam,
                         const orc_cfg *cfg, const double *gC, const double *gD,
                         const double *gF, const double *gT, double *g_uv, double *g_conic,
                         double *g_opac, double *g_color, double *g_z, double *g_feat)
{
    visit_lists vl;
    build_visit(N, valid, pcam, rect, uv, conic, opac, cam, cfg, &vl);
    int Wd = cam->width, Ht = cam->height;
    size_t P = (size_t)Wd * Ht;
    memset(g_uv, 0, sizeof(double) * 2 * N);
    memset(g_conic, 0, sizeof(double) * 3 * N);
    memset(g_opac, 0, sizeof(double) * N);
    memset(g_color, 0, sizeof(double) * 3 * N);
    memset(g_z, 0, sizeof(double) * N);
    if (NL) memset(g_feat, 0, sizeof(double) * NL * (size_t)N);
    int maxn = cfg->brute ? vl.n_all : 0;
    if (!cfg->brute) {
        int nt = ((Wd + cfg->tile - 1) / cfg->tile) * ((Ht + cfg->tile - 1) / cfg->tile);
        for (int t = 0; t < nt; ++t) {
            int c = vl.ranges[2 * t + 1] - vl.ranges[2 * t];
            if (c > maxn) maxn = c;
        }
    }
#pragma omp parallel
    {
        int *sg = malloc(sizeof(int) * (maxn + 1));
        double *sa = malloc(sizeof(double) * (maxn + 1)); /* alpha */
        double *sT = malloc(sizeof(double) * (maxn + 1)); /* T before blending */
        double *sG = malloc(sizeof(double) * (maxn + 1)); /* exp(-q/2) */
        int *sc = malloc(sizeof(int) * (maxn + 1));       /* alpha clamped */
#pragma omp for schedule(dynamic, 4)
        for (int py = 0; py < Ht; ++py) {
            for (int px = 0; px < Wd; ++px) {
                const int *list;
                int n;
                pixel_list(&vl, cam, cfg, px, py, &list, &n);
                size_t p = (size_t)py * Wd + px;
                /* forward replay */
                double T = 1.0;
                int m = 0;
                for (int idx = 0; idx < n; ++idx) {
                    int g = list[idx];
                    double dx = px - uv[2 * g], dy = py - uv[2 * g + 1];
                    const double *cn = conic + 3 * g;
                    double q = cn[0] * dx * dx + 2.0 * cn[1] * dx * dy + cn[2] * dy * dy;
                    double G = exp(-0.5 * q);
                    double raw = opac[g] * G;
                    double alpha = raw < cfg->alpha_max ? raw : cfg->alpha_max;
                    if (alpha < cfg->alpha_min) continue;
                    double Tn = T * (1.0 - alpha);
                    if (Tn < cfg->t_min) break;
                    sg[m] = g;
                    sa[m] = alpha;
                    sT[m] = T;
                    sG[m] = G;
                    sc[m] = !(raw < cfg->alpha_max);
                    ++m;
                    T = Tn;
                }
                double Tfinal = T;
                /* back to front: acc = sum_{k>i} w_k (x_k . g) + gT * T_final */
                double gc[3] = {gC ? gC[p] : 0, gC ? gC[P + p] : 0, gC ? gC[2 * P + p] : 0};
                double gd = gD ? gD[p] : 0;
                double acc = (gT ? gT[p] : 0.0) * Tfinal;
                for (int i = m - 1; i >= 0; --i) {
                    int g = sg[i];
                    double a = sa[i], Ti = sT[i], w = a * Ti;
                    double xg = color[3 * g] * gc[0] + color[3 * g + 1] * gc[1] +
                                color[3 * g + 2] * gc[2] + pcam[3 * g + 2] * gd;
                    for (int ch = 0; ch < NL; ++ch)
                        xg += feat[(size_t)NL * g + ch] * (gF ? gF[ch * P + p] : 0.0);
                    double dalpha = Ti * xg - acc / (1.0 - a);
                    acc += w * xg;
                    double d_opac = 0, d_q = 0;
                    if (!sc[i]) {
                        d_opac = dalpha * sG[i];
                        d_q = dalpha * (-0.5 * a);
                    }
                    double dx = px - uv[2 * g], dy = py - uv[2 * g + 1];
                    const double *cn = conic + 3 * g;
#pragma omp critical(orc_bwd_acc)
                    {
                        for (int ch = 0; ch < 3; ++ch) g_color[3 * g + ch] += w * gc[ch];
                        g_z[g] += w * gd;
                        for (int ch = 0; ch < NL; ++ch)
                            g_feat[(size_t)NL * g + ch] += w * (gF ? gF[ch * P + p] : 0.0);
                        g_opac[g] += d_opac;
                        g_conic[3 * g + 0] += d_q * dx * dx;
                        g_conic[3 * g + 1] += d_q * 2.0 * dx * dy;
                        g_conic[3 * g + 2] += d_q * dy * dy;
                        /* dq/du = -2 (a dx + b dy), dq/dv = -2 (b dx + c dy) */
                        g_uv[2 * g + 0] += d_q * (-2.0) * (cn[0] * dx + cn[1] * dy);
                        g_uv[2 * g + 1] += d_q * (-2.0) * (cn[1] * dx + cn[2] * dy);
                    }
                }
            }
        }
        free(sg);
        free(sa);
        free(sT);
        free(sG);
        free(sc);
    }
    free_visit(&vl);
}

/* ------------------------------------------------------------------------ */
/* Backward of Eq. 1-2                                                      */
/* ------------------------------------------------------------------------ */

/* Inputs: 3D Gaussians of this view, camera, and the 2D gradients from the
 * blending backward.  Outputs (overwritten): g_mean[3], g_scale[3], g_quat[4]
 * per Gaussian; g_pose[6] = dL/d(rho, phi) for T_cw <- Exp(xi) T_cw.
 * scale_reg adds a constant dL/ds (the mean-scale term of Eq. 14). */
void orc_project_bwd_view(int N, const double *mean, const double *scale, const double *quat,
                          const int *valid, const orc_camera *cam, const orc_cfg *cfg,
                          const double *g_uv, const double *g_conic, const double *g_z,
                          double scale_reg, double *g_mean, double *g_scale, double *g_quat,
                          double *g_pose)
{
    const double *T = cam->Tcw;
    double W[3][3] = {{T[0], T[1], T[2]}, {T[4], T[5], T[6]}, {T[8], T[9], T[10]}};
    double t[3] = {T[3], T[7], T[11]};
    double pose[6] = {0, 0, 0, 0, 0, 0};
    for (int g = 0; g < N; ++g) {
        for (int i = 0; i < 3; ++i) {
            g_mean[3 * g + i] = 0;
            g_scale[3 * g + i] = scale_reg;
        }
        for (int i = 0; i < 4; ++i) g_quat[4 * g + i] = 0;
        if (!valid[g]) continue;
        const double *mu = mean + 3 * g;
        double p[3];
        for (int i = 0; i < 3; ++i) p[i] = W[i][0] * mu[0] + W[i][1] * mu[1] + W[i][2] * mu[2] + t[i];
        /* forward recomputation */
        double qn[4], qs = 0;
        for (int i = 0; i < 4; ++i) qs += quat[4 * g + i] * quat[4 * g + i];
        qs = sqrt(qs);
        for (int i = 0; i < 4; ++i) qn[i] = quat[4 * g + i] / qs;
        double R[3][3], s[3] = {scale[3 * g], scale[3 * g + 1], scale[3 * g + 2]};
        quat_to_rot(qn, R);
        double Sg[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += R[i][k] * s[k] * s[k] * R[j][k];
                Sg[i][j] = acc;
            }
        double M[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += W[i][k] * Sg[k][l] * W[j][l];
                M[i][j] = acc;
            }
        double z = p[2], fx = cam->fx, fy = cam->fy;
        double J[2][3] = {{fx / z, 0, -fx * p[0] / (z * z)}, {0, fy / z, -fy * p[1] / (z * z)}};
        double C2[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += J[i][k] * M[k][l] * J[j][l];
                C2[i][j] = acc;
            }
        double A = C2[0][0] + cfg->dilation, B = C2[0][1], Cc = C2[1][1] + cfg->dilation;
        double D = A * Cc - B * B, D2 = D * D;
        /* conic (a, b, c) = (C/D, -B/D, A/D) -> gradient on (A, B, C) */
        double ga = g_conic[3 * g], gb = g_conic[3 * g + 1], gc = g_conic[3 * g + 2];
        double gA = ga * (-Cc * Cc / D2) + gb * (B * Cc / D2) + gc * (-B * B / D2);
        double gB = ga * (2 * B * Cc / D2) + gb * (-(A * Cc + B * B) / D2) + gc * (2 * A * B / D2);
        double gC = ga * (-B * B / D2) + gb * (B * A / D2) + gc * (-A * A / D2);
        /* symmetric 2x2 gradient of Sigma' */
        double G2[2][2] = {{gA, 0.5 * gB}, {0.5 * gB, gC}};
        /* dL/dM = J^T G2 J, dL/dJ = 2 G2 J M */
        double GM[3][3], GJ[2][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 2; ++l) acc += J[k][i] * G2[k][l] * J[l][j];
                GM[i][j] = acc;
            }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 3; ++l) acc += G2[i][k] * J[k][l] * M[l][j];
                GJ[i][j] = 2.0 * acc;
            }
        /* dL/dp from J, from uv and from the depth value */
        double gp[3] = {0, 0, 0};
        gp[0] += GJ[0][2] * (-fx / (z * z));
        gp[1] += GJ[1][2] * (-fy / (z * z));
        gp[2] += GJ[0][0] * (-fx / (z * z)) + GJ[0][2] * (2 * fx * p[0] / (z * z * z)) +
                 GJ[1][1] * (-fy / (z * z)) + GJ[1][2] * (2 * fy * p[1] / (z * z * z));
        double gu = g_uv[2 * g], gv = g_uv[2 * g + 1];
        gp[0] += gu * fx / z;
        gp[1] += gv * fy / z;
        gp[2] += -gu * fx * p[0] / (z * z) - gv * fy * p[1] / (z * z);
        gp[2] += g_z[g];
        /* mean: p = W mu + t */
        for (int i = 0; i < 3; ++i) g_mean[3 * g + i] = W[0][i] * gp[0] + W[1][i] * gp[1] + W[2][i] * gp[2];
        /* Sigma: dL/dSigma = W^T GM W */
        double GS[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += W[k][i] * GM[k][l] * W[l][j];
                GS[i][j] = acc;
            }
        /* Sigma = (R S)(R S)^T : dL/d(RS) = 2 GS (R S) */
        double RS[3][3], GRS[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) RS[i][j] = R[i][j] * s[j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += GS[i][k] * RS[k][j];
                GRS[i][j] = 2.0 * acc;
            }
        double GR[3][3];
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int i = 0; i < 3; ++i) {
                GR[i][j] = GRS[i][j] * s[j];
                acc += GRS[i][j] * R[i][j];
            }
            g_scale[3 * g + j] += acc;
        }
        /* rotation -> unit quaternion */
        double w = qn[0], x = qn[1], y = qn[2], zq = qn[3];
        double dq[4];
        dq[0] = 2 * (-zq * GR[0][1] + y * GR[0][2] + zq * GR[1][0] - x * GR[1][2] - y * GR[2][0] +
                     x * GR[2][1]);
        dq[1] = 2 * (y * GR[0][1] + zq * GR[0][2] + y * GR[1][0] - 2 * x * GR[1][1] -
                     w * GR[1][2] + zq * GR[2][0] + w * GR[2][1] - 2 * x * GR[2][2]);
        dq[2] = 2 * (-2 * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] +
                     zq * GR[1][2] - w * GR[2][0] + zq * GR[2][1] - 2 * y * GR[2][2]);
        dq[3] = 2 * (-2 * zq * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] -
                     2 * zq * GR[1][1] + y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
        /* normalisation q / |q| */
        double dot = qn[0] * dq[0] + qn[1] * dq[1] + qn[2] * dq[2] + qn[3] * dq[3];
        for (int i = 0; i < 4; ++i) g_quat[4 * g + i] = (dq[i] - qn[i] * dot) / qs;
        /* pose: d rho = dL/dp, d phi = p x dL/dp + vee(2 M GM) */
        double A2[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += M[i][k] * GM[k][j];
                A2[i][j] = 2.0 * acc;
            }
        pose[0] += gp[0];
        pose[1] += gp[1];
        pose[2] += gp[2];
        pose[3] += p[1] * gp[2] - p[2] * gp[1] + A2[1][2] - A2[2][1];
        pose[4] += p[2] * gp[0] - p[0] * gp[2] + A2[2][0] - A2[0][2];
        pose[5] += p[0] * gp[1] - p[1] * gp[0] + A2[0][1] - A2[1][0];
    }
    for (int i = 0; i < 6; ++i) g_pose[i] = pose[i];
}

/* ------------------------------------------------------------------------ */
/* Backward of Eq. 8-9                                                      */
/* ------------------------------------------------------------------------ */

/* Given dL/d(mean, opacity, scale, quaternion, colour, feature) of the decoded
 * Gaussians of one view, ACCUMULATE (+=) the gradients of the MLP weights and
 * anchor parameters, and write g_pose[6] (the camera-centre dependence of the
 * decode inputs delta_vc, d_vc). */
void orc_decode_bwd_view(int A, int K, int F, int H, int NL, int op_tanh, const double *anc_pos,
                         const double *anc_feat, const double *anc_off,
                         const double *anc_scale, const double *W1, const double *b1,
                         const double *W2, const double *b2, const orc_camera *cam,
                         double t_norm, const double *g_mean, const double *g_opac,
                         const double *g_scale, const double *g_quat, const double *g_color,
                         const double *g_feat, double *gW1, double *gb1, double *gW2,
                         double *gb2, double *g_pos, double *g_afeat, double *g_off,
                         double *g_ascale, double *g_pose)
{
    double oc[3];
    camera_centre(cam->Tcw, oc);
    const double *T = cam->Tcw;
    int din = F + 6, nout = K * (11 + NL);
    double *x = malloc(sizeof(double) * din), *z = malloc(sizeof(double) * 4 * H);
    double *h = malloc(sizeof(double) * 4 * H), *y = malloc(sizeof(double) * nout);
    double *dy = malloc(sizeof(double) * nout), *dh = malloc(sizeof(double) * 4 * H);
    double *dz = malloc(sizeof(double) * 4 * H), *dx = malloc(sizeof(double) * din);
    double goc[3] = {0, 0, 0};
    for (int a = 0; a < A; ++a) {
        double delta[3], dist;
        decode_input(F, anc_pos + 3 * a, anc_feat + (size_t)F * a, oc, t_norm, x, delta, &dist);
        decode_mlp(K, F, H, NL, W1, b1, W2, b2, x, z, h, y);
        for (int k = 0; k < K; ++k) {
            size_t g = (size_t)a * K + k;
            if (op_tanh) {
                double o = tanh(y[k]);
                dy[k] = g_opac[g] * (1 - o * o);
            } else {
                double o = sigmoid(y[k]);
                dy[k] = g_opac[g] * o * (1 - o);
            }
            for (int i = 0; i < 3; ++i) {
                double sg = sigmoid(y[K + 7 * k + i]);
                dy[K + 7 * k + i] = g_scale[3 * g + i] * anc_scale[3 * a + i] * sg * (1 - sg);
                g_ascale[3 * a + i] += g_scale[3 * g + i] * sg;
            }
            for (int i = 0; i < 4; ++i) dy[K + 7 * k + 3 + i] = g_quat[4 * g + i];
            for (int i = 0; i < 3; ++i) {
                double c = sigmoid(y[8 * K + 3 * k + i]);
                dy[8 * K + 3 * k + i] = g_color[3 * g + i] * c * (1 - c);
            }
            for (int i = 0; i < NL; ++i) dy[11 * K + NL * k + i] = g_feat[(size_t)NL * g + i];
            for (int i = 0; i < 3; ++i) {
                g_pos[3 * a + i] += g_mean[3 * g + i];
                g_off[3 * g + i] += g_mean[3 * g + i];
            }
        }
        for (int j = 0; j < 4 * H; ++j) dh[j] = 0;
        for (int r = 0; r < nout; ++r) {
            int grp = out_group(r, K);
            gb2[r] += dy[r];
            for (int j = 0; j < H; ++j) {
                gW2[r * H + j] += dy[r] * h[grp * H + j];
                dh[grp * H + j] += W2[r * H + j] * dy[r];
            }
        }
        for (int j = 0; j < 4 * H; ++j)
            dz[j] = (j < 3 * H) ? (z[j] > 0 ? dh[j] : 0.0) : dh[j] * sigmoid(z[j]);
        for (int i = 0; i < din; ++i) dx[i] = 0;
        for (int j = 0; j < 4 * H; ++j) {
            gb1[j] += dz[j];
            for (int i = 0; i < din; ++i) {
                gW1[j * din + i] += dz[j] * x[i];
                dx[i] += W1[j * din + i] * dz[j];
            }
        }
        for (int i = 0; i < F; ++i) g_afeat[(size_t)F * a + i] += dx[i];
        /* delta = r/|r|, d = |r|, r = x_v - o_c */
        double dd = dx[F + 3], ddl[3] = {dx[F], dx[F + 1], dx[F + 2]};
        double dot = delta[0] * ddl[0] + delta[1] * ddl[1] + delta[2] * ddl[2];
        for (int i = 0; i < 3; ++i) {
            double dr = (ddl[i] - delta[i] * dot) / dist + dd * delta[i];
            g_pos[3 * a + i] += dr;
            goc[i] -= dr;
        }
    }
    /* o_c(xi) = t_wc - R_wc rho to first order: d rho = -W dL/do_c, d phi = 0 */
    for (int i = 0; i < 3; ++i)
        g_pose[i] = -(T[4 * i + 0] * goc[0] + T[4 * i + 1] * goc[1] + T[4 * i + 2] * goc[2]);
    g_pose[3] = g_pose[4] = g_pose[5] = 0;
    free(x);
    free(z);
    free(h);
    free(y);
    free(dy);
    free(dh);
    free(dz);
    free(dx);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
