/*
 * ups.h — C ABI of the GB300 (sm_103a) differentiable render path of
 * anchor-decoded 3D Gaussians (UP-SLAM, arXiv 2505.22335).
 *
 * Path: decode (Eq. 8-9) -> projection (Eq. 1-2) -> (view, tile, depth) key
 * sort -> tile ranges -> front-to-back blending of colour, depth, an N_l-channel
 * feature map and transmittance (Eq. 3, Eq. 10) -> per-pixel weighted loss
 * (Eq. 4, Eq. 14) -> reverse-order backward into Gaussian, MLP-weight and
 * SE(3) pose gradients.
 *
 * Conventions shared by every entry point
 *  - All tensor arguments are DEVICE pointers to float32 (or uint32 where
 *    stated), owned by the caller, contiguous, 16-byte aligned.
 *  - "float4 [n]" means n records of 4 floats; unused lanes are ignored on
 *    input and written as 0 on output.
 *  - Images of several views are concatenated view after view; inside a view
 *    a C-channel image is C planes of H x W (row-major).  View v starts at
 *    pixel offset P_v = sum_{u<v} H_u W_u, so its channel c of a C-channel
 *    image starts at element C * P_v + c * H_v * W_v.
 *  - Pixel (i, j) is sampled at continuous image coordinate (i, j); a camera
 *    point (X, Y, Z) maps to u = fx X/Z + cx, v = fy Y/Z + cy.  Background 0.
 *  - Poses are world-to-camera T_cw, row-major 4x4 float, on the HOST (copied
 *    into kernel parameters).  Pose gradients are dL/dxi for the left
 *    perturbation T_cw <- Exp(xi) T_cw, xi = (rho[3], phi[3]), at xi = 0.
 *  - Every call is stream-ordered on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream), never aborts and never throws; the return value
 *    is a ups_status and ups_last_error() gives a message.  One ups_ctx must
 *    not be used from two host threads at the same time.
 */
#ifndef UPS_H
#define UPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define UPS_MAX_VIEWS 64

typedef struct ups_ctx ups_ctx;
typedef void *ups_stream; /* cudaStream_t */

typedef enum {
    UPS_OK = 0,
    UPS_PENDING = 1,        /* ups_poll: request not finished yet */
    UPS_ERR_ARG = 2,        /* invalid argument (sizes, NULL, alignment) */
    UPS_ERR_OOM = 3,        /* device or pinned allocation failed */
    UPS_ERR_CUDA = 4,       /* a CUDA runtime call failed */
    UPS_ERR_TIMEOUT = 5,    /* a bounded wait ran out */
    UPS_ERR_CANCELLED = 6,  /* request cancelled before it ran */
    UPS_ERR_NONFINITE = 7,  /* check_finite found NaN/Inf in an input */
    UPS_ERR_CAPACITY = 8,   /* a fixed-size buffer is too small */
    UPS_ERR_STATE = 9       /* call out of order (e.g. backward before forward) */
} ups_status;

/* Readings of the thresholds Eq. 3 leaves open and the model sizes. */
typedef struct {
    float alpha_min;  /* skip a Gaussian whose alpha is below this (1/255) */
    float alpha_max;  /* alpha clamp (0.99) */
    float t_min;      /* stop before the Gaussian that takes T below this (1e-4) */
    float dilation;   /* added to the diagonal of Sigma' in px^2 (0.3) */
    float near_z;     /* cull Z <= near_z (0.2 m) */
    float guard;      /* cull |X/Z| > guard * W / (2 fx), same in y (1.3) */
    int n_feat;       /* N_l, rendered feature channels: 0, 16 or 32 */
    int k;            /* Gaussians per anchor K (1..16) */
    int feat_dim;     /* anchor feature width (32) */
    int hidden;       /* decode MLP hidden width (32) */
    int decode_bf16;  /* 1: decode GEMMs in BF16 on the tensor cores, FP32 accumulate */
    int check_finite; /* 1: scan inputs for NaN/Inf and fail with UPS_ERR_NONFINITE */
    int list_cap;     /* tile lists keep their first list_cap entries in depth order
                         (0: 1024; < 0: no cap; at most 32767).  Blending reads a
                         list only until every pixel of the tile has stopped (Eq. 3
                         with the t_min reading), so a cap changes nothing unless a
                         pixel is still open at the end of a cut list: the forward
                         then sorts that batch again without the cap and blends it
                         again (ups_stats.list_refills).  Views of more than 16383
                         tiles in total are never capped. */
    int opacity_tanh; /* 1: decoded opacity o = tanh(y) (the Scaffold-GS decode the
                         paper cites for Eq. 8-9) instead of sigmoid(y); the
                         projection's cull of o < alpha_min then drops every
                         Gaussian with o <= 0 (alpha_min > 0).  0 (default): sigmoid. */
    int decode_bwd_bf16; /* with decode_bf16: 1 also runs the decode backward's per-row
                         data path with BF16 tensor-core operands; 0 (default) runs it
                         in FP32 on the CUDA cores, which is faster at these sizes and
                         keeps the backward in FP32 (the decode forward stays BF16) */
} ups_config;

/* Fills the defaults listed above (n_feat 16, k 10, feat_dim 32, hidden 32,
 * list_cap 1024, opacity_tanh 0, decode_bwd_bf16 0). */
void ups_config_default(ups_config *cfg);

/* Pinhole camera of one view (Sec. 3.1); t_norm feeds the temporal encoding
 * l_t = (sin pi t, cos pi t) of Sec. 3.3. */
typedef struct {
    float fx, fy, cx, cy;
    int width, height;
    float T_cw[16];
    float t_norm;
} ups_camera;

/* A set of 3D Gaussians G = {(mu, o, c, Sigma = R S S^T R^T)} (Eq. 1).
 *  n         Gaussians per set
 *  per_view  0: one set used by every view (plain 3DGS); 1: one set per view
 *            (decode output, set v belongs to view v)
 *  mean_opacity float4 [sets][n]: mu_x, mu_y, mu_z, o  (o in (0,1))
 *  scale        float4 [sets][n]: s_x, s_y, s_z, -    (s > 0)
 *  quat         float4 [sets][n]: w, x, y, z          (any nonzero norm)
 *  color        float4 [sets][n]: r, g, b, -
 *  feat         float  [sets][n][n_feat]              (NULL if n_feat == 0)
 * The same struct holds gradients dL/d(each field); with per_view == 0 the
 * gradients are summed over views. */
typedef struct {
    int n;
    int per_view;
    float *mean_opacity;
    float *scale;
    float *quat;
    float *color;
    float *feat;
} ups_gaussians;

/* Rendered images (Eq. 3, Eq. 10), layouts as in the header comment.
 *  color [3 planes], depth [1], feat [n_feat planes] (NULL if n_feat == 0),
 *  T     final transmittance prod(1 - alpha_i) [1]; Eq. 3's accumulated T~ is 1 - T
 *  n_contrib uint32 [1]: list position of the last blended Gaussian + 1. */
typedef struct {
    float *color;
    float *depth;
    float *feat;
    float *T;
    uint32_t *n_contrib;
} ups_images;

/* dL/d(rendered images); any pointer may be NULL (zero gradient). */
typedef struct {
    const float *color;
    const float *depth;
    const float *feat;
    const float *T;
} ups_image_grads;

/* Targets of the weighted loss; weight is the per-pixel map w (NULL = 1). */
typedef struct {
    const float *color;
    const float *depth;
    const float *feat;
    const float *weight;
} ups_targets;

/* L = (1/sum_v H_v W_v) sum_p w_p [lc sum l(C-Ct) + ld l(D-Dt) + lf sum l(F-Ft)]
 *     + lambda_scale * mean(s)   (Eq. 4 / Eq. 14; l = |.| or (.)^2) */
typedef struct {
    float lambda_color;
    float lambda_depth;
    float lambda_feat;
    float lambda_scale;
    int l2; /* 0: l1, 1: squared */
} ups_loss_cfg;

/* Anchors (Sec. 3.3 "Adaptively Structured Gaussian").
 *  pos     [n][3] anchor position x_v
 *  feat    [n][feat_dim] anchor feature f_v
 *  offsets [n][k][3] learnable offsets; Gaussian mean mu = x_v + O_{v,k}
 *  scaling [n][3] per-anchor scaling l_v; Gaussian scale s = l_v * sigmoid(.) */
typedef struct {
    int n;
    float *pos;
    float *feat;
    float *offsets;
    float *scaling;
} ups_anchors;

/* The four decode MLPs (Eq. 8-9): opacity, covariance (3 scale + 4 quaternion),
 * colour, feature F_d.  Input x = [f_v (feat_dim), delta_vc (3), d_vc (1),
 * sin(pi t), cos(pi t)] with delta_vc = (x_v - o_c)/|x_v - o_c|, d_vc = |x_v - o_c|.
 *  w1 [4*hidden][feat_dim+6], b1 [4*hidden]: hidden blocks in the order above;
 *     ReLU for the first three, SoftPlus for F_d
 *  w2 [k*(11+n_feat)][hidden], b2 [k*(11+n_feat)]: output rows grouped as
 *     opacity (k), covariance (7k), colour (3k), feature (k*n_feat); group g
 *     reads hidden block g.  Output activations: sigmoid opacity and colour,
 *     s = l_v * sigmoid, raw quaternion, linear feature. */
typedef struct {
    float *w1;
    float *b1;
    float *w2;
    float *b2;
} ups_mlp;

/* Which gradients ups_render_backward / ups_decode_backward produce. */
enum {
    UPS_GRAD_POSE = 1,     /* dL/dxi per view */
    UPS_GRAD_GAUSS = 2,    /* dL/d(Gaussian set) */
    UPS_GRAD_MLP = 4,      /* dL/d(w1, b1, w2, b2) */
    UPS_GRAD_ANCHOR = 8,   /* dL/d(anchor pos, feat, offsets, scaling) */
    UPS_GRAD_ALL = 15
};

/* Counters of the last forward (reading them synchronises the ctx stream). */
typedef struct {
    int n_views;
    long long n_gaussian_views; /* sets used x n over all views */
    long long n_visible;        /* Gaussian-views touching at least one tile */
    long long n_instances;      /* (view, tile, Gaussian) entries sorted */
    long long n_tiles;          /* tiles over all views */
    long long n_pixels;
    int key_bits;               /* significant bits of the (view, tile) key */
    long long n_listed;         /* entries kept in the tile lists (list_cap) */
    int list_refills;           /* 1: a capped list was too short and the lists were rebuilt */
} ups_stats;

/* ---------------------------------------------------------------------- */
/* context                                                                */
/* ---------------------------------------------------------------------- */

/* Creates a context on CUDA device `device` (made current for every call on
 * this ctx).  The ctx owns only scratch memory, grown on demand. */
ups_status ups_create(const ups_config *cfg, int device, ups_ctx **out);
ups_status ups_destroy(ups_ctx *ctx);
/* Message of the last failed call on ctx (or of the last ups_create failure
 * when ctx is NULL).  Valid until the next call on ctx. */
const char *ups_last_error(const ups_ctx *ctx);
const char *ups_version(void);

/* ---------------------------------------------------------------------- */
/* forward                                                                */
/* ---------------------------------------------------------------------- */

/* Eq. 8-9: decode k Gaussians per anchor for each of n_views cameras.
 * out (caller-allocated, per_view must be 1, n == anchors->n * k) receives
 * mean_opacity, scale, quat (unnormalised), color and feat of set v = view v,
 * Gaussian id g = anchor * k + j. */
ups_status ups_decode_anchors(ups_ctx *ctx, const ups_anchors *anchors, const ups_mlp *mlp,
                              const ups_camera *cams, int n_views, ups_gaussians *out,
                              ups_stream stream);

/* Eq. 1-3, Eq. 10: project, bin by (view, tile, depth), blend front to back.
 * g and out must stay alive and unmodified until ups_render_backward on this
 * ctx, which reuses them (T and n_contrib replace per-fragment state).
 * Synchronises `stream` once to size the instance buffers. */
ups_status ups_render_forward(ups_ctx *ctx, const ups_gaussians *g, const ups_camera *cams,
                              int n_views, ups_images *out, ups_stream stream);

/* Weighted loss of the last forward's images against `tgt`.  Writes the
 * scalar loss to loss_dev[0] (device float, overwritten) and dL/d(images) to
 * dL (caller-allocated, same layouts as the images).  If g is not NULL and
 * lcfg->lambda_scale != 0 the mean-scale term of Eq. 14 is added. */
ups_status ups_loss_weighted(ups_ctx *ctx, const ups_images *img, const ups_targets *tgt,
                             const ups_loss_cfg *lcfg, const ups_gaussians *g,
                             float *loss_dev, ups_images *dL, ups_stream stream);

/* Training-free tracking uncertainty (Sec. 3.4 "Tracking", Eq. 6, Eq. 15) of
 * the last forward's images against tgt (color, depth, feat; weight unused),
 * per pixel:
 *   R      = (T < t_mask) (lambda_color |C~ - C|_1 + lambda_depth |D~ - B(D)|
 *                          + lambda_feat min(1, 1 - cos(F, F~)))
 *   sigma2 = 2 R     (Eq. 15 minimises 1/2 (R / sigma^2 + log sigma) per pixel;
 *                     R = 0 gives the limit 0)
 *   motion = 2 sigma2 > 1, i.e. R > 1/4 (1: dynamic)
 * Readings: T is the final transmittance (Eq. 3's T~ read as transmittance, so
 * the mask keeps covered pixels); |.|_1 sums the colour channels; B is the 3x3
 * box filter of the target depth, the mean over the window's pixels inside the
 * view; cos = 0 when either feature vector is zero; n_feat == 0: no feature
 * term.  img needs color, depth, T (and feat); outputs are device arrays of
 * sum_v H_v W_v in the depth layout (R, sigma2 float; motion uint8), each may
 * be NULL.  Defaults (Sec. 4 "Implementation Details"): lambda = (0.25, 0.7,
 * 0.1), t_mask = 0.1. */
typedef struct {
    float lambda_color;
    float lambda_depth;
    float lambda_feat;
    float t_mask;
} ups_residual_cfg;

ups_status ups_tracking_uncertainty(ups_ctx *ctx, const ups_images *img, const ups_targets *tgt,
                                    const ups_residual_cfg *rcfg, float *R, float *sigma2,
                                    unsigned char *motion, ups_stream stream);

/* Feature lifting and distillation (Sec. 3.3, Eq. 11, Eq. 12; App. "MLP
 * Implementation Details"): F^ = F_m(F~) per pixel of the last forward's
 * rendered feature map F~ (n_feat channels), F_m = 1x1 convolution (n_feat ->
 * 128) -> ReLU -> 1x1 convolution (128 -> n_h), and
 *   L_d = (1 / P) sum_p (1 - cos(F_p, F^_p))     (P: pixels of all views)
 * against the DINO features F, given per view on the patch grid (Sec. 3.2:
 * bilinear upsampling to the image): view v's grid is hp x wp = ceil(H/patch)
 * x ceil(W/patch) vectors of n_h floats, row-major [hp][wp][n_h], the views'
 * grids concatenated; pixel (x, y) samples it at ((x + 0.5)/patch - 0.5,
 * (y + 0.5)/patch - 0.5), clamped to the grid.  cos = 0 (and no gradient)
 * where either vector is zero.  Computed without forming F^ (the cosine and
 * the gradients from per-patch products of W2); at n_feat = 16 the per-pixel
 * products run on the tensor cores with FP32 accumulation: the first layer
 * Z = W1 F~ (whose sign decides ReLU') in 3xTF32 (operands split in TF32 hi
 * and lo, FP32-level products), M H, the Gram of b H and dW1 = dZ F~^T in
 * 3xBF16 (about 1e-5 relative per product); dF~ and the per-pixel terms are
 * FP32 on the CUDA cores.  At n_feat = 32 every product is FP32.
 *  feat      rendered F~ in the image layout (n_feat planes per view)
 *  dino      the patch grids (16-byte aligned; UPS_ERR_ARG otherwise)
 *  mlp       w1 [128][n_feat], b1 [128], w2 [n_h][128], b2 [n_h] (b2 16-byte aligned)
 *  weight    per-pixel weight w_p of (1 - cos) in the mean (depth layout; NULL: 1), e.g.
 *            the mask M of Eq. 14 (L = M (L_g + lambda_4 L_d) + ...)
 *  scale     weight of L_d (e.g. lambda_4 of Eq. 14)
 *  loss_dev  device float: overwritten with scale * L_d
 *  d_mlp     if not NULL: scale * dL_d/d(w1, b1, w2, b2) ADDED to its arrays
 *            (each may be NULL)
 *  d_feat    if not NULL: scale * dL_d/dF~ ADDED (image layout), e.g. to the
 *            image loss's feature gradient before ups_render_backward */
typedef struct {
    int n_h;    /* DINO feature width (384): a multiple of 4, at most 4096 */
    int patch;  /* DINO patch size in pixels (14) */
} ups_lift_cfg;

typedef struct {
    float *w1;
    float *b1;
    float *w2;
    float *b2;
} ups_lift_mlp;

ups_status ups_feature_lift(ups_ctx *ctx, const ups_lift_cfg *lcfg, const float *feat, const float *dino,
                            const ups_lift_mlp *mlp, const float *weight, float scale, float *loss_dev,
                            ups_lift_mlp *d_mlp, float *d_feat, ups_stream stream);

/* The D-SSIM term of the geometric loss (Eq. 4):
 *   loss_dev[0] = scale (1 - SSIM(C~, C))   (overwritten)
 * SSIM (Wang et al., cited by the paper) per colour channel of each of the last
 * forward's views: 11 x 11 Gaussian window (sigma 1.5, normalised), C1 =
 * 0.01^2, C2 = 0.03^2 (colours in [0, 1]), zero padding at the border,
 * averaged over the 3 channels and all pixels, each pixel's (1 - S) times
 * weight[p] (depth layout; NULL: 1), e.g. the mask M of Eq. 14.  If d_color is
 * not NULL, scale * d/dC~ is ADDED to it (image layout).  color, t_color:
 * image layout. */
ups_status ups_ssim_loss(ups_ctx *ctx, const float *color, const float *t_color, const float *weight, float scale,
                         float *loss_dev, float *d_color, ups_stream stream);

/* Uncertainty MLP F_u and its loss (Sec. 3.3 "Uncertainty Prediction for
 * Mapping", Eq. 5, Eq. 13; App. "MLP Implementation Details"):
 *   sigma_p = SoftPlus(w2 . ReLU(W1 F_p + b1) + b2)
 * (1x1 conv -> ReLU -> 1x1 conv -> SoftPlus, hidden 128, one output) with F_p
 * the DINO feature of pixel p, bilinear from the patch grids exactly as in
 * ups_feature_lift (lcfg, dino), and
 *   loss_dev[0] = scale * (1/P) sum_p [R_p / (2 sigma_p^2) + lambda log sigma_p]
 * over the last forward's views (overwritten).  R: per-pixel residual in the
 * depth layout (e.g. ups_tracking_uncertainty's R).  The gradient flows only
 * into F_u (the paper keeps the mapping and uncertainty gradient flows apart):
 * if d_mlp is not NULL, scale * dL/d(w1, b1, w2, b2) is ADDED (each may be
 * NULL).  sigma (float) and motion (uint8, M = 2 sigma^2 > 1 of Sec. 3.3) are
 * written per pixel when not NULL.
 *  mlp  w1 [128][n_h], b1 [128], w2 [128], b2 [1] */
ups_status ups_uncertainty_mlp(ups_ctx *ctx, const ups_lift_cfg *lcfg, const float *dino, const float *R,
                               const ups_lift_mlp *mlp, float lambda, float scale, float *loss_dev,
                               ups_lift_mlp *d_mlp, float *sigma, unsigned char *motion, ups_stream stream);

/* Probabilistic anchors (Sec. 3.3 "Adaptively Structured Gaussian", Eq. 7;
 * the probabilistic octree of Sec. 1 read as a voxel grid of edge `voxel`
 * holding the anchors).  One keyframe (cam, its depth map and motion mask):
 *  1. update: each anchor n observed in the keyframe gets
 *       L(n|z_1:t) = clamp(L(n|z_1:t-1) + (L(n|z_t) - L(n)), l_min, l_max),
 *     Eq. 7 in log-odds form L(p) = log(p / (1 - p)), with the garbled last
 *     factor of Eq. 7 read as P(n) / (1 - P(n)) (OctoMap's update, which the
 *     paper cites).  Observation (reading; FP32, one rounding per operation):
 *     the anchor centre x maps to X = R x + t (summed left to right) and to
 *     pixel (floor(fx X/Z + cx + 1/2), floor(fy Y/Z + cy + 1/2)); with D the
 *     depth there, Z <= near_z, a pixel outside the image or D <= near_z is no
 *     observation, Z < D - margin (free space on the ray) a miss, Z <= D +
 *     margin a hit (a miss on a pixel whose motion is nonzero), Z > D + margin
 *     (hidden) no observation.  Unobserved anchors keep their log-odds.
 *  2. prune: anchors whose log-odds is below l_prune are deleted; the others
 *     keep their order (out rows 0 .. n_kept - 1).
 *  3. insert: each pixel with D > near_z and motion 0 is back-projected,
 *     x = R^T ((i - cx) / fx D - t_x, (j - cy) / fy D - t_y, D - t_z), to its
 *     voxel floor(x / voxel) (indices in [-2^20, 2^20) per axis, others are
 *     skipped); every voxel holding no kept anchor (an anchor holds the voxel
 *     floor(pos / voxel)) gets a new anchor at its centre (q + 1/2) voxel, in
 *     the raster order of the first pixel that reached it, while rows remain
 *     below `capacity`: zero feature and offsets, scaling = voxel, log-odds =
 *     clamp(l_prior + (l_hit - l_prior)) (the prior and this one hit).
 *  in, logodds_in   n anchors (ups_anchors layout, feat_dim and k of the ctx)
 *                   and their log-odds float [n]; may be empty (n = 0)
 *  out, logodds_out capacity rows each (capacity >= in->n); must not overlap
 *                   the inputs; out->n is set on return
 *  depth            float [H][W] of the keyframe (metres; <= near_z: none)
 *  motion           uint8 [H][W] (nonzero: dynamic), or NULL: all static
 *  src_index        int [capacity] or NULL: the input row of each output row,
 *                   -1 - p for a row inserted from pixel p = j W + i
 *  res              counts of the call (may be NULL)
 * Synchronises `stream` once to read the counts.  A voxel table that cannot
 * hold the keys (it is sized for twice the anchors plus pixels, so this does
 * not happen) fails with UPS_ERR_CAPACITY. */
typedef struct {
    float l_prior; /* L(P(n)), the prior (P(n) = 0.5) */
    float l_hit;   /* L(P(n|z_t)) of a static surface observation (0.7) */
    float l_miss;  /* L(P(n|z_t)) of free space or a dynamic surface (0.4) */
    float l_min;   /* clamping of the posterior (0.12) */
    float l_max;   /* (0.97) */
    float l_prune; /* delete anchors below this (P = 0.5, i.e. 0) */
    float voxel;   /* anchor voxel edge in metres (0.05) */
    float margin;  /* half-width of the surface band along the ray (0.05) */
    float near_z;  /* depths at or below this are not observations (0.2) */
} ups_anchor_cfg;

/* Fills the defaults listed above (OctoMap's probabilities as log-odds). */
void ups_anchor_cfg_default(ups_anchor_cfg *cfg);

typedef struct {
    int n_kept;     /* input anchors that survived the pruning */
    int n_inserted; /* new anchors written after them */
    int n_dropped;  /* new voxels that found no row below capacity */
    int n_hit;      /* anchors observed as hits / misses */
    int n_miss;
} ups_anchor_result;

ups_status ups_anchor_update(ups_ctx *ctx, const ups_anchor_cfg *acfg, const ups_camera *cam, const float *depth,
                             const unsigned char *motion, const ups_anchors *in, const float *logodds_in,
                             ups_anchors *out, float *logodds_out, int capacity, int *src_index,
                             ups_anchor_result *res, ups_stream stream);

/* ---------------------------------------------------------------------- */
/* backward                                                               */
/* ---------------------------------------------------------------------- */

/* Reverse-order backward of the last ups_render_forward on ctx: the
 * derivative of the blending of Eq. 3 and Eq. 10 (walked back to front from
 * each pixel's last blended Gaussian, transmittance recomputed by division
 * from the stored final T) and of the projection of Eq. 1-2 (conic, camera
 * point, 3D covariance from scale and quaternion), and of the pose T_cw <-
 * Exp(xi) T_cw at xi = 0, xi = (rho, phi).
 *  dL        image gradients (any may be NULL)
 *  grad      UPS_GRAD_GAUSS: dL/d(Gaussian set), same shape as the forward
 *            input; OVERWRITTEN (per_view == 1) or OVERWRITTEN as the sum over
 *            views (per_view == 0).  May be NULL without that flag.
 *  d_pose    UPS_GRAD_POSE: float [n_views][6], OVERWRITTEN
 *  scale_grad  constant added to every dL/ds (the mean-scale term:
 *            lambda_scale / (3 * sets * n)); 0 for none. */
ups_status ups_render_backward(ups_ctx *ctx, const ups_image_grads *dL, unsigned grad_mask,
                               float scale_grad, ups_gaussians *grad, float *d_pose,
                               ups_stream stream);

/* Backward of Eq. 8-9 for the views of the last ups_decode_anchors-shaped
 * call: dG holds dL/d(decoded sets) (per_view == 1).  ACCUMULATES (+=) into
 * d_mlp (UPS_GRAD_MLP), d_anchors (UPS_GRAD_ANCHOR) and d_pose (UPS_GRAD_POSE;
 * the camera-centre dependence of delta_vc and d_vc).  Pointers of a flag that
 * is not set may be NULL. */
ups_status ups_decode_backward(ups_ctx *ctx, const ups_anchors *anchors, const ups_mlp *mlp,
                               const ups_camera *cams, int n_views, const ups_gaussians *dG,
                               unsigned grad_mask, ups_mlp *d_mlp, ups_anchors *d_anchors,
                               float *d_pose, ups_stream stream);

/* ---------------------------------------------------------------------- */
/* inspection (tests and benchmarks)                                      */
/* ---------------------------------------------------------------------- */

ups_status ups_get_stats(ups_ctx *ctx, ups_stats *out);

/* Internal buffers of the last forward, copied to HOST memory `dst` of
 * `bytes` bytes (at most the buffer size; the copy synchronises):
 *   0 sorted instance Gaussian-view ids   uint32 [n_listed] (gv = view*n + g)
 *   1 sorted instance keys                uint32 [n_listed] (tile_base[view] + tile)
 *   2 tile ranges                         uint32 [n_tiles][2]  ([start, end))
 *   3 projected (u, v, z, o)              float4 [n_gaussian_views]
 *   4 conic (a, b, c, -)                  float4 [n_gaussian_views]
 *   5 tile rect (x0 | y0 << 16, x1 | y1 << 16)  uint32 [n_gaussian_views][2]
 *   6 per-Gaussian-view 2D gradients of the last backward
 *     float [n_gaussian_views][12 + n_feat]: du dv dz do dca dcb dcc dr dg db - - df...
 * Returns the buffer size in bytes through *size (dst may be NULL). */
ups_status ups_copy_buffer(ups_ctx *ctx, int which, void *dst, size_t bytes, size_t *size);

/* Stage profiler.  When enabled, every stage (one or more kernels) of the
 * calls above is bracketed by CUDA events recorded on the call's stream.
 * ups_profile_read synchronises on those events and writes a JSON object
 * {"stage": [total_ms, calls], ...} into buf (NUL-terminated; UPS_ERR_ARG if
 * len is too small), stores the number of kernels launched since the last
 * read in *launches (may be NULL; counted whether or not profiling is on), and
 * resets both. */
ups_status ups_profile_enable(ups_ctx *ctx, int on);
ups_status ups_profile_read(ups_ctx *ctx, char *buf, size_t len, long long *launches);

/* ---------------------------------------------------------------------- */
/* serving: request queue with continuous batching                        */
/* ---------------------------------------------------------------------- */

/* UP-SLAM runs tracking and mapping as parallel threads over one map (Sec. 3,
 * Sec. 3.4): tracking renders the map at a pose to form residuals, mapping
 * optimises the map over keyframes.  The server keeps the anchor scene
 * resident and serves both as requests.  Worker threads (one per slot, each
 * with its own context, stream and buffers) pack the requests waiting in the
 * queue, up to max_batch_views views and within the memory budget, into ONE
 * batched decode + forward + backward; slots run concurrently, so requests
 * that arrive while other batches are on the GPU are admitted as slots and
 * memory free up.  Completion is stamped by a stream callback. */

typedef struct ups_server ups_server;

enum { UPS_REQ_TRACK = 0, UPS_REQ_MAP = 1 };

/* One request.  Host fields are copied by ups_submit; device buffers are the
 * caller's and must stay valid until the request is done.
 *  kind      UPS_REQ_TRACK: render `cams[0]` at `levels` pyramid levels (level
 *            l: intrinsics and size divided by 2^l), forward + pose-only
 *            backward.  UPS_REQ_MAP: render n_views keyframes, full backward.
 *  targets   device images of the request's own views (level 0 first for
 *            tracking), layouts as for ups_loss_weighted; weight may be NULL
 *  loss      device float[1]: weighted image loss of the request (Eq. 4/14
 *            image part, normalised by the request's pixels)
 *  d_pose    device float[6 * n_views] (tracking: [6], summed over levels),
 *            OVERWRITTEN
 *  d_mlp, d_anchors  mapping only, optional (NULL pointers = not wanted):
 *            ACCUMULATED (+=) MLP / anchor gradients of the request */
typedef struct {
    int kind;
    int n_views;
    int levels;
    const ups_camera *cams;
    ups_targets targets;
    float *loss;
    float *d_pose;
    ups_mlp d_mlp;
    ups_anchors d_anchors;
} ups_request;

typedef struct {
    int slots;            /* batches in flight at once (worker threads), >= 1 */
    int max_batch_views;  /* views packed into one batch (<= UPS_MAX_VIEWS) */
    int batching;         /* 1: continuous batching; 0: one request per batch */
    double memory_budget_gb; /* admission: estimated scratch of in-flight batches */
    ups_loss_cfg loss;    /* image-loss weights (lambda_scale unused) */
} ups_server_config;

typedef struct {
    int status;          /* UPS_PENDING, UPS_OK, or the error of the request */
    double submit_ms;    /* host steady-clock times, ms since server creation */
    double start_ms;
    double end_ms;       /* stream completion of the request's batch */
    int batch_id;
    int batch_requests;  /* requests packed into that batch */
    int batch_views;
} ups_result;

/* scene: anchors + MLP weights on the device (caller-owned, kept resident;
 * must stay valid and unmodified while requests are in flight). */
ups_status ups_server_create(const ups_config *cfg, const ups_server_config *scfg, int device,
                             const ups_anchors *scene, const ups_mlp *mlp, ups_server **out);
/* Finishes every queued request, then stops the workers and frees buffers. */
ups_status ups_server_destroy(ups_server *srv);
ups_status ups_submit(ups_server *srv, const ups_request *req, uint64_t *ticket);
/* UPS_OK and *out filled when the request is done (its entry is then
 * released), UPS_PENDING while queued or running, UPS_ERR_ARG for an unknown
 * ticket. */
ups_status ups_poll(ups_server *srv, uint64_t ticket, ups_result *out);
/* Removes a request that has not started: UPS_OK (its poll then reports
 * UPS_ERR_CANCELLED), UPS_ERR_STATE if it already started. */
ups_status ups_cancel(ups_server *srv, uint64_t ticket);
/* Blocks until the queue is empty and no batch is in flight, at most
 * timeout_ms (UPS_ERR_TIMEOUT then). */
ups_status ups_server_wait_idle(ups_server *srv, double timeout_ms);
/* Replaces the resident scene (anchors + MLP weights), e.g. after a mapping
 * step or a probabilistic anchor update (ups_anchor_update) changed it.  No new
 * batch starts during the call; it waits, at most timeout_ms (UPS_ERR_TIMEOUT,
 * scene unchanged), until the batches in flight have finished on the GPU, then
 * swaps the pointers.  Requests still queued run on the new scene; a queued
 * mapping request that asked for anchor gradients (d_anchors sized for the old
 * anchor count) fails with UPS_ERR_STATE when the count changed.  The old
 * buffers are the caller's again once the call returns UPS_OK. */
ups_status ups_server_set_scene(ups_server *srv, const ups_anchors *scene, const ups_mlp *mlp,
                                double timeout_ms);
const char *ups_server_last_error(const ups_server *srv);

/* ---------------------------------------------------------------------- */
/* allocation-free forward                                                */
/* ---------------------------------------------------------------------- */

/* The paper has no counterpart to this entry point.
 *
 * Same result as ups_render_forward (same kernels), for callers that cannot
 * allocate GPU memory: a tracking front end running at camera rate inside a
 * fixed memory budget cannot afford cudaMalloc/cudaFree (they synchronise the
 * device and can stall for milliseconds) and may not grow its footprint, so it
 * cannot use a ups_ctx, whose scratch grows on demand.  This call needs no
 * context and allocates nothing: its scratch is one static device array of
 * about 14 MB inside the library, held by every GPU that loads the library
 * until the process exits.
 *  cfg       thresholds and n_feat (k, feat_dim, hidden, decode_bf16 unused)
 *  g, cams, n_views, out   as for ups_render_forward; runs on the CURRENT
 *            device, stream-ordered on `stream`, and synchronises it once
 * Limits (UPS_ERR_CAPACITY, message via ups_last_error(NULL)): n * n_views
 * <= 65536 and <= 8192 16x16 tiles over all views, both checked before any
 * kernel runs; <= 524288 tile instances, known only after the projection and
 * depth sort have run: on that error the static array has been written and
 * the output images have not.  No backward state is kept.
 * The static array is shared by every call on a device and keeps the last
 * call's contents (each call writes or clears what it reads); calls that
 * overlap on the GPU race on it and must be serialised by the caller.  Every
 * call looks up the array's device address on the current device and
 * synchronises `stream` once (to read the instance count). */
ups_status ups_render_forward_static(const ups_config *cfg, const ups_gaussians *g,
                                     const ups_camera *cams, int n_views, ups_images *out,
                                     ups_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* UPS_H */
