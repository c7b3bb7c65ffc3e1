// Host side of the C ABI (include/ups.h): argument checks, scratch memory,
// and the order of kernel launches for decode, forward, loss and backward.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <vector>

#include "common.cuh"
#include "decode_bwd.cuh"

namespace ups {

// launchers implemented in the other translation units
cudaError_t launch_project(const ViewTable &vt, const BlendParams &bp, int N, int per_view,
                           int total, const ups_gaussians &g, float4 *xyzo, float4 *conic,
                           uint2 *rect, uint32_t *count, uint64_t *dkey, uint32_t *dval,
                           cudaStream_t st);
cudaError_t launch_project_k32(const ViewTable &vt, const BlendParams &bp, int N, int per_view,
                               int total, const ups_gaussians &g, float4 *xyzo, float4 *conic,
                               uint2 *rect, uint32_t *count, uint32_t *dkey32, uint32_t *dval,
                               int vbits, cudaStream_t st);
cudaError_t launch_gather_counts(const uint32_t *sorted_gv, const uint32_t *count, uint32_t *out,
                                 int total, cudaStream_t st);
cudaError_t launch_emit(const ViewTable &vt, const BlendParams &bp, int N, int total, const uint32_t *sorted_gv,
                        const uint64_t *off, const uint2 *rect, const float4 *xyzo, const float4 *conic,
                        uint32_t *ikey, uint32_t *ival, cudaStream_t st);
cudaError_t launch_ranges(const uint32_t *ikey, uint32_t n, uint2 *ranges, cudaStream_t st);
cudaError_t launch_project_bwd(const ViewTable &vt, const BlendParams &bp, int N, int per_view,
                               int total, int n_feat, unsigned mask, float scale_grad,
                               const ups_gaussians &g, const float *g2, const ups_gaussians *grad,
                               float *d_pose, cudaStream_t st);
cudaError_t launch_composite_fwd(const ViewTable &vt, const BlendParams &bp, int n_feat, int N,
                                 int per_view, const uint2 *ranges, const uint32_t *ival,
                                 const float4 *xyzo, const float4 *conic, const float4 *color,
                                 const float *feat, const ups_images &out, cudaStream_t st,
                                 const uint32_t *trunc = nullptr, int *trunc_flag = nullptr,
                                 const int *gate = nullptr, int *err = nullptr);
size_t anchor_scratch_bytes(size_t n, size_t P);
cudaError_t anchor_update(const DevView &cam, const float *depth, const uint8_t *motion, int n, const float *pos,
                          const float *feat, const float *offsets, const float *scaling, const float *lin, int F,
                          int K3, float l_prior, float l_hit, float l_miss, float l_min, float l_max, float l_prune,
                          float voxel, float margin, float near_z, long long capacity, float *opos, float *ofeat,
                          float *ooffsets, float *oscaling, float *olog, int *src_index, void *scratch,
                          uint64_t **summary_dev, cudaStream_t st, int *launches);
size_t unc_scratch_floats(int max_patches);
cudaError_t unc_view(int num_sms, cudaStream_t st, int W, int H, int nh, int patch, const float *grid, int wp,
                     int hp, const float *R, const float *w1, const float *b1, const float *w2, const float *b2,
                     float lambda, float g, float *loss, float *d_w1, float *d_b1, float *d_w2, float *d_b2,
                     float *sigma, uint8_t *motion, float *scratch, int *launches);
cudaError_t ssim_set_window();
cudaError_t launch_ssim(const ViewTable &vt, const float *x, const float *y, const float *weight, float *G, float g,
                        float *loss, float *dx, cudaStream_t st);
size_t lift_scratch_floats(size_t np_total);
cudaError_t lift_all(int num_sms, cudaStream_t st, const ViewTable &vt, int nf, int nh, int patch, const float *feat,
                     const float *grid, const float *w1, const float *b1, const float *w2, const float *b2, float g,
                     const float *weight, float *loss, float *d_w1, float *d_b1, float *d_w2, float *d_b2,
                     float *d_feat, float *scratch, int *err, int *launches);
cudaError_t launch_uncertainty(const ViewTable &vt, int n_feat, int max_hw, float lc, float ld, float lf,
                               float t_mask, const ups_images &img, const ups_targets &tgt, float *R, float *sigma2,
                               uint8_t *motion, cudaStream_t st);
cudaError_t launch_loss(const ViewTable &vt, int n_feat, int max_hw, float lc, float ld, float lf,
                        int l2, float inv_norm, const ups_images &img, const ups_targets &tgt,
                        const ups_images &grad, float *loss, cudaStream_t st, int v0 = 0, int v1 = -1);
cudaError_t launch_scale_mean(const float4 *scale, size_t n, float coef, float *loss,
                              cudaStream_t st);
cudaError_t launch_composite_bwd(const ViewTable &vt, const BlendParams &bp, int n_feat, int N,
                                 int per_view, const uint2 *ranges, const uint32_t *ival,
                                 const float4 *xyzo, const float4 *conic, const float4 *color,
                                 const float *feat, const float *T, const uint32_t *nc,
                                 const ups_image_grads &dL, float *g2, cudaStream_t st, int *err);
cudaError_t launch_decode_fwd(const ViewTable &vt, int A, int K, int NF, const ups_anchors &anc,
                              const ups_mlp &mlp, const ups_gaussians &out, int op_tanh, int num_sms,
                              cudaStream_t st);
cudaError_t launch_decode_fwd_tc(const ViewTable &vt, int A, int K, int NF, const ups_anchors &anc,
                                 const ups_mlp &mlp, const ups_gaussians &out, int bf16, int op_tanh, int *err,
                                 int num_sms, cudaStream_t st);
size_t decode_tc_smem_bytes(int NF, int bf16);
cudaError_t launch_decode_bwd(const ViewTable &vt, int A, int K, int NF, const ups_anchors &anc,
                              const ups_mlp &mlp, const ups_gaussians &dG, unsigned mask, const ups_mlp *d_mlp,
                              const ups_anchors *d_anc, float *d_pose, int bf16, int op_tanh, float *scratch,
                              int *err, int num_sms, const dbwd::StageHook &hook, cudaStream_t st);
size_t decode_bwd_scratch_bytes(int A, int V, int K, int NF);
bool decode_bwd_fits(int K, int NF);

cudaError_t DevBuf::reserve(size_t want) {
    if (want <= bytes) return cudaSuccess;
    release();
    size_t b = std::max<size_t>(want + want / 8, 256);
    cudaError_t e = cudaMalloc(&ptr, b);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        return e;
    }
    bytes = b;
    return cudaSuccess;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

}  // namespace ups

using namespace ups;

struct ups_ctx {
    ups_config cfg{};
    int device = 0;
    int num_sms = 1;
    std::string err;
    cudaStream_t last_stream = nullptr;
    // forward state
    bool have_fwd = false;
    ViewTable vt{};
    BlendParams bp{};
    int N = 0, per_view = 0;
    int n_sets = 0;            // Gaussian sets the views read
    bool shared_sets = false;  // some set is read by several views (gradients summed)
    size_t total_gv = 0;
    size_t n_inst = 0, n_visible = 0, n_pix = 0;
    int key_bits = 0, max_hw = 0;
    ups_gaussians g_in{};
    ups_images img{};
    bool have_bwd = false;
    // scratch
    DevBuf xyzo, conic, rect, count, dkey0, dkey1, dval0, dval1, cnt_sorted, off, scan_scr;
    DevBuf ikey0, ikey1, ival0, ival1, ranges, g2;
    DevBuf dec_scratch;  // decode backward: X, H, dL/dY, dL/dZ rows for the weight gradients
    SortScratch sort;
    uint32_t *dval_sorted = nullptr, *ikey_sorted = nullptr, *ival_sorted = nullptr;
    // pinned: [0] instance count, [1] device error / list-cap flag, [2] the
    // last tile range
    uint64_t *h_total = nullptr;
    int *d_err = nullptr;         // set by kernels whose bounded waits ran out
    int *d_trunc_flag = nullptr;  // set by the forward blend: a capped list was too short
    DevBuf trunc;                 // per-tile bit: the list cap cut the tile's list
    bool capped = false;          // the last forward capped its tile lists
    DevBuf lift_scr;              // feature-lifting scratch of one view
    DevBuf ssim_g;                // D-SSIM window-term maps of all colour planes
    DevBuf unc_scr;               // uncertainty-MLP patch scratch of one view
    DevBuf anchor_scr;            // probabilistic-anchor update: flags, scans, voxel table
    uint64_t *h_anchor = nullptr;  // pinned: the anchor update's counts
    bool ssim_window = false;     // the SSIM window is in this device's constant memory
    // stage profiler (CUDA events on the launch stream) and kernel-launch count
    bool prof = false;
    struct Rec {
        const char *name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<double, long long>> acc;
    long long launches = 0;
    const char *cur_name = nullptr;
    cudaEvent_t cur_a = nullptr;
};

namespace {

thread_local std::string g_create_error;

ups_status fail(ups_ctx *c, ups_status s, const std::string &msg) {
    if (c)
        c->err = msg;
    else
        g_create_error = msg;
    return s;
}

ups_status cuda_fail(ups_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? UPS_ERR_OOM : UPS_ERR_CUDA, m);
}

#define UPS_CUDA(c, expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return cuda_fail(c, _e, #expr); \
    } while (0)

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

cudaEvent_t ev_get(ups_ctx *c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Stage timing: begin/end bracket one stage (one or more kernels) on stream st;
// `kernels` is the number of kernel launches of the stage.
void stage_begin(ups_ctx *c, const char *name, cudaStream_t st) {
    if (!c->prof) return;
    c->cur_name = name;
    c->cur_a = ev_get(c);
    cudaEventRecord(c->cur_a, st);
}

void stage_end(ups_ctx *c, cudaStream_t st, long long kernels) {
    c->launches += kernels;
    if (!c->prof || !c->cur_a) return;
    cudaEvent_t b = ev_get(c);
    cudaEventRecord(b, st);
    c->pending.push_back({c->cur_name, c->cur_a, b});
    c->cur_a = nullptr;
}

long long radix_kernels(size_t n, int bits) {
    if (n <= 1 || bits <= 0) return 0;
    return (long long)((bits + 7) / 8) * 5;  // histogram + 3 scan kernels + scatter per pass
}

ups_status build_views(ups_ctx *c, const ups_camera *cams, int n_views, ViewTable &vt,
                       size_t &n_pix, int &max_hw) {
    if (!cams || n_views < 1 || n_views > UPS_MAX_VIEWS)
        return fail(c, UPS_ERR_ARG, "n_views must be in [1, UPS_MAX_VIEWS] and cams non-NULL");
    std::memset(&vt, 0, sizeof(vt));
    vt.n = n_views;
    int tiles = 0;
    size_t pix = 0;
    max_hw = 0;
    for (int v = 0; v < n_views; ++v) {
        const ups_camera &cm = cams[v];
        if (cm.width < 1 || cm.height < 1 || cm.width > 16384 || cm.height > 16384 ||
            !(cm.fx > 0) || !(cm.fy > 0))
            return fail(c, UPS_ERR_ARG, "camera " + std::to_string(v) + ": bad intrinsics or size");
        for (int i = 0; i < 16; ++i)
            if (!std::isfinite(cm.T_cw[i]))
                return fail(c, UPS_ERR_NONFINITE, "camera " + std::to_string(v) + ": non-finite pose");
        DevView &d = vt.v[v];
        d.fx = cm.fx;
        d.fy = cm.fy;
        d.cx = cm.cx;
        d.cy = cm.cy;
        d.W = cm.width;
        d.H = cm.height;
        d.tiles_x = (cm.width + kTile - 1) / kTile;
        d.tiles_y = (cm.height + kTile - 1) / kTile;
        d.tile_base = tiles;
        d.pix_off = (int)pix;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) d.R[3 * i + j] = cm.T_cw[4 * i + j];
            d.t[i] = cm.T_cw[4 * i + 3];
        }
        d.limx = c->cfg.guard * 0.5f * cm.width / cm.fx;
        d.limy = c->cfg.guard * 0.5f * cm.height / cm.fy;
        d.t_norm = cm.t_norm;
        tiles += d.tiles_x * d.tiles_y;
        pix += (size_t)cm.width * cm.height;
        max_hw = std::max(max_hw, cm.width * cm.height);
    }
    if (pix > (size_t)INT32_MAX) return fail(c, UPS_ERR_ARG, "too many pixels in one call");
    vt.total_tiles = tiles;
    n_pix = pix;
    return UPS_OK;
}

ups_status check_gaussians(ups_ctx *c, const ups_gaussians *g, const char *what) {
    if (!g) return fail(c, UPS_ERR_ARG, std::string(what) + " is NULL");
    if (g->n < 1) return fail(c, UPS_ERR_ARG, std::string(what) + ".n must be >= 1");
    const void *ptrs[4] = {g->mean_opacity, g->scale, g->quat, g->color};
    for (const void *p : ptrs)
        if (!p || !aligned16(p))
            return fail(c, UPS_ERR_ARG, std::string(what) + ": NULL or unaligned attribute pointer");
    if (c->cfg.n_feat > 0 && (!g->feat || !aligned16(g->feat)))
        return fail(c, UPS_ERR_ARG, std::string(what) + ".feat NULL or unaligned");
    return UPS_OK;
}

int bits_for(size_t n) {
    int b = 0;
    while (b < 63 && ((size_t)1 << b) < n) ++b;
    return b;
}

ups_status set_device(ups_ctx *c) {
    UPS_CUDA(c, cudaSetDevice(c->device));
    return UPS_OK;
}

}  // namespace

namespace ups {
// Message returned by ups_last_error(NULL) (calls made without a context).
void set_global_error(const std::string &msg) { g_create_error = msg; }

// Loss of views [v0, v1) of the last forward on c, normalised by their pixel
// count; targets and weights are laid out from view v0 (pixel offset 0).
ups_status loss_views(ups_ctx *c, const ups_images *img, const ups_targets *tgt,
                      const ups_loss_cfg *lcfg, int v0, int v1, float *loss_dev, ups_images *dL,
                      cudaStream_t st) {
    if (!c->have_fwd) return fail(c, UPS_ERR_STATE, "loss_views needs a forward first");
    if (v0 < 0 || v1 > c->vt.n || v1 <= v0) return fail(c, UPS_ERR_ARG, "bad view range");
    size_t pix = 0;
    int mhw = 0;
    for (int v = v0; v < v1; ++v) {
        const size_t hw = (size_t)c->vt.v[v].W * c->vt.v[v].H;
        pix += hw;
        mhw = std::max(mhw, (int)hw);
    }
    stage_begin(c, "loss", st);
    UPS_CUDA(c, cudaMemsetAsync(loss_dev, 0, sizeof(float), st));
    UPS_CUDA(c, launch_loss(c->vt, c->cfg.n_feat, mhw, lcfg->lambda_color, lcfg->lambda_depth,
                            lcfg->lambda_feat, lcfg->l2, (float)(1.0 / (double)pix), *img, *tgt, *dL,
                            loss_dev, st, v0, v1));
    stage_end(c, st, 1);
    return UPS_OK;
}
// Entries in the tile lists of the last forward (a capped forward keeps
// fewer than it emitted unless the GPU rebuilt them whole: *refilled).
// Synchronises the ctx stream.
ups_status listed_entries(ups_ctx *c, size_t *listed, int *refilled) {
    *listed = c->n_inst;
    *refilled = 0;
    if (!c->capped) return UPS_OK;
    UPS_CUDA(c, cudaSetDevice(c->device));
    UPS_CUDA(c, cudaStreamSynchronize(c->last_stream));
    uint2 last;
    int flag = 0;
    UPS_CUDA(c, cudaMemcpy(&last, c->ranges.as<uint2>() + c->vt.total_tiles - 1, sizeof(uint2),
                           cudaMemcpyDeviceToHost));
    UPS_CUDA(c, cudaMemcpy(&flag, c->d_trunc_flag, sizeof(int), cudaMemcpyDeviceToHost));
    *listed = last.y;
    *refilled = flag != 0;
    return UPS_OK;
}

}  // namespace ups

extern "C" {

void ups_config_default(ups_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->alpha_min = 1.f / 255.f;
    cfg->alpha_max = 0.99f;
    cfg->t_min = 1e-4f;
    cfg->dilation = 0.3f;
    cfg->near_z = 0.2f;
    cfg->guard = 1.3f;
    cfg->n_feat = 16;
    cfg->k = 10;
    cfg->feat_dim = 32;
    cfg->hidden = 32;
    cfg->decode_bf16 = 0;
    cfg->check_finite = 0;
    cfg->list_cap = 1024;
    cfg->opacity_tanh = 0;
    cfg->decode_bwd_bf16 = 0;
}

void ups_anchor_cfg_default(ups_anchor_cfg *cfg) {
    if (!cfg) return;
    auto L = [](double p) { return (float)std::log(p / (1.0 - p)); };
    cfg->l_prior = L(0.5);
    cfg->l_hit = L(0.7);
    cfg->l_miss = L(0.4);
    cfg->l_min = L(0.12);
    cfg->l_max = L(0.97);
    cfg->l_prune = L(0.5);
    cfg->voxel = 0.05f;
    cfg->margin = 0.05f;
    cfg->near_z = 0.2f;
}

const char *ups_version(void) { return "ups-gb300 0.1 (sm_103a)"; }

ups_status ups_create(const ups_config *cfg, int device, ups_ctx **out) {
    if (!out) return fail(nullptr, UPS_ERR_ARG, "out is NULL");
    *out = nullptr;
    ups_config c{};
    if (cfg)
        c = *cfg;
    else
        ups_config_default(&c);
    if (c.n_feat != 0 && c.n_feat != 16 && c.n_feat != 32)
        return fail(nullptr, UPS_ERR_ARG, "n_feat must be 0, 16 or 32");
    if (c.k < 1 || c.k > 16) return fail(nullptr, UPS_ERR_ARG, "k must be in [1, 16]");
    if (c.feat_dim != 32 || c.hidden != 32)
        return fail(nullptr, UPS_ERR_ARG, "feat_dim and hidden must be 32");
    if (!decode_bwd_fits(c.k, c.n_feat))
        return fail(nullptr, UPS_ERR_ARG, "k * (11 + n_feat) too large for the decode backward tiling");
    if (!(c.alpha_min > 0.f) || !(c.alpha_max >= c.alpha_min) || !(c.alpha_max < 1.f) ||
        !(c.t_min >= 0.f) || !(c.dilation >= 0.f) || !(c.near_z > 0.f) || !(c.guard > 0.f))
        return fail(nullptr, UPS_ERR_ARG, "threshold out of range");
    if (c.list_cap > kMaxListCap) return fail(nullptr, UPS_ERR_ARG, "list_cap must be at most 32767");
    if (c.opacity_tanh != 0 && c.opacity_tanh != 1) return fail(nullptr, UPS_ERR_ARG, "opacity_tanh must be 0 or 1");
    if (c.decode_bwd_bf16 != 0 && c.decode_bwd_bf16 != 1)
        return fail(nullptr, UPS_ERR_ARG, "decode_bwd_bf16 must be 0 or 1");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev)
        return fail(nullptr, UPS_ERR_CUDA, std::string("no CUDA device ") + std::to_string(device) +
                                               (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : ""));
    ups_ctx *ctx = new ups_ctx();
    ctx->cfg = c;
    ctx->device = device;
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_total, 4 * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_trunc_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_trunc_flag, 0, sizeof(int));
    if (e != cudaSuccess) {
        g_create_error = std::string("ups_create: ") + cudaGetErrorString(e);
        delete ctx;
        return UPS_ERR_CUDA;
    }
    ctx->bp = BlendParams{c.alpha_min, c.alpha_max, c.t_min, c.dilation, c.near_z};
    *out = ctx;
    return UPS_OK;
}

ups_status ups_destroy(ups_ctx *c) {
    if (!c) return UPS_OK;
    cudaSetDevice(c->device);
    DevBuf *bufs[] = {&c->xyzo, &c->conic, &c->rect, &c->count, &c->dkey0, &c->dkey1, &c->dval0,
                      &c->dval1, &c->cnt_sorted, &c->off, &c->scan_scr, &c->ikey0, &c->ikey1,
                      &c->ival0, &c->ival1, &c->ranges, &c->g2, &c->dec_scratch, &c->sort.hist, &c->trunc, &c->lift_scr, &c->ssim_g, &c->unc_scr, &c->anchor_scr};
    for (DevBuf *b : bufs) b->release();
    if (c->h_total) cudaFreeHost(c->h_total);
    if (c->h_anchor) cudaFreeHost(c->h_anchor);
    if (c->d_err) cudaFree(c->d_err);
    if (c->d_trunc_flag) cudaFree(c->d_trunc_flag);
    for (auto &r : c->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
    delete c;
    return UPS_OK;
}

const char *ups_last_error(const ups_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

ups_status ups_decode_anchors(ups_ctx *c, const ups_anchors *anc, const ups_mlp *mlp,
                              const ups_camera *cams, int n_views, ups_gaussians *out,
                              ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    if (!anc || !mlp || !out) return fail(c, UPS_ERR_ARG, "NULL argument");
    if (anc->n < 1 || !anc->pos || !anc->feat || !anc->offsets || !anc->scaling)
        return fail(c, UPS_ERR_ARG, "anchors: n < 1 or NULL pointer");
    if (!aligned16(anc->feat)) return fail(c, UPS_ERR_ARG, "anchors.feat must be 16-byte aligned");
    if (!mlp->w1 || !mlp->b1 || !mlp->w2 || !mlp->b2) return fail(c, UPS_ERR_ARG, "mlp: NULL pointer");
    if (!out->per_view || (size_t)out->n != (size_t)anc->n * c->cfg.k)
        return fail(c, UPS_ERR_ARG, "out must be per_view with n == anchors.n * k");
    ups_status s = check_gaussians(c, out, "out");
    if (s != UPS_OK) return s;
    if ((size_t)anc->n * c->cfg.k * n_views >= (size_t)INT32_MAX)
        return fail(c, UPS_ERR_ARG, "anchors * k * views exceeds 2^31");
    ViewTable vt;
    size_t npix;
    int mhw;
    if ((s = build_views(c, cams, n_views, vt, npix, mhw)) != UPS_OK) return s;
    if ((s = set_device(c)) != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    stage_begin(c, "decode_fwd", st);
    // BF16 decode on the tensor cores; the FP32 decode on the CUDA cores (its
    // 3xTF32 tensor-core form needs 223 KB of operands, one CTA per SM, and is
    // slower than the CUDA-core kernel at these sizes)
    const int bf16 = c->cfg.decode_bf16 ? 1 : 0;
    if (bf16 && decode_tc_smem_bytes(c->cfg.n_feat, bf16) + 1024 <= 227 * 1024)
        UPS_CUDA(c, launch_decode_fwd_tc(vt, anc->n, c->cfg.k, c->cfg.n_feat, *anc, *mlp, *out, bf16,
                                         c->cfg.opacity_tanh, c->d_err, c->num_sms, st));
    else
        UPS_CUDA(c, launch_decode_fwd(vt, anc->n, c->cfg.k, c->cfg.n_feat, *anc, *mlp, *out, c->cfg.opacity_tanh,
                                      c->num_sms, st));
    stage_end(c, st, 1);
    return UPS_OK;
}

// (C++ linkage inside this extern "C" block: an internal entry point of the server)
extern "C++" {
namespace ups {
// The render forward of ups_render_forward.  set_of_view (per_view sets only;
// NULL: view v reads set v) names the Gaussian set each view reads, so that
// several views (the pyramid levels of one tracking pose) can share one
// decoded set; sets read by several views get their gradients summed.
ups_status render_forward_sets(ups_ctx *c, const ups_gaussians *g, const ups_camera *cams, int n_views,
                               const int *set_of_view, ups_images *out, ups_stream stream);
}  // namespace ups
}

ups_status ups_render_forward(ups_ctx *c, const ups_gaussians *g, const ups_camera *cams,
                              int n_views, ups_images *out, ups_stream stream) {
    return render_forward_sets(c, g, cams, n_views, nullptr, out, stream);
}

extern "C++" ups_status ups::render_forward_sets(ups_ctx *c, const ups_gaussians *g, const ups_camera *cams,
                                                 int n_views, const int *set_of_view, ups_images *out,
                                                 ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    c->have_fwd = false;
    c->have_bwd = false;
    ups_status s = check_gaussians(c, g, "g");
    if (s != UPS_OK) return s;
    if (!out || !out->color || !out->depth || !out->T || !out->n_contrib ||
        (c->cfg.n_feat > 0 && !out->feat))
        return fail(c, UPS_ERR_ARG, "out: NULL image pointer");
    if (set_of_view && !g->per_view) return fail(c, UPS_ERR_ARG, "a view-to-set map needs per_view sets");
    ViewTable &vt = c->vt;
    if ((s = build_views(c, cams, n_views, vt, c->n_pix, c->max_hw)) != UPS_OK) return s;
    // which set each view reads; whether any set is read by more than one view
    c->n_sets = g->per_view ? (set_of_view ? 0 : n_views) : 1;
    c->shared_sets = !g->per_view;
    for (int v = 0; v < n_views; ++v) {
        const int sv = !g->per_view ? 0 : set_of_view ? set_of_view[v] : v;
        if (sv < 0 || sv >= UPS_MAX_VIEWS) return fail(c, UPS_ERR_ARG, "set index out of range");
        vt.v[v].set = sv;
        vt.v[v].set_first = 1;
        for (int u = 0; u < v; ++u)
            if (vt.v[u].set == sv) {
                vt.v[v].set_first = 0;
                c->shared_sets = true;
            }
        if (set_of_view) c->n_sets = std::max(c->n_sets, sv + 1);
    }
    const size_t total = (size_t)g->n * n_views;
    if (total >= (size_t)INT32_MAX) return fail(c, UPS_ERR_ARG, "n * n_views exceeds 2^31");
    if ((s = set_device(c)) != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    c->N = g->n;
    c->per_view = g->per_view ? 1 : 0;
    c->total_gv = total;
    // per-Gaussian-view scratch
    UPS_CUDA(c, c->xyzo.reserve(total * sizeof(float4)));
    UPS_CUDA(c, c->conic.reserve(total * sizeof(float4)));
    UPS_CUDA(c, c->rect.reserve(total * sizeof(uint2)));
    UPS_CUDA(c, c->count.reserve(total * sizeof(uint32_t)));
    UPS_CUDA(c, c->dkey0.reserve(total * sizeof(uint64_t)));
    UPS_CUDA(c, c->dkey1.reserve(total * sizeof(uint64_t)));
    UPS_CUDA(c, c->dval0.reserve(total * sizeof(uint32_t)));
    UPS_CUDA(c, c->dval1.reserve(total * sizeof(uint32_t)));
    UPS_CUDA(c, c->cnt_sorted.reserve(total * sizeof(uint32_t)));
    UPS_CUDA(c, c->off.reserve((total + 1) * sizeof(uint64_t)));
    UPS_CUDA(c, c->scan_scr.reserve(scan_scratch_bytes(total)));
    UPS_CUDA(c, c->ranges.reserve((size_t)vt.total_tiles * sizeof(uint2)));

    // (view, depth) order of the Gaussian-views: 32-bit keys (view in the top
    // bits, depth bits above 0.125 m below) when the view index fits in 4 bits
    // and the near plane is >= 0.125 m, else 64-bit keys
    int vbits = bits_for((size_t)n_views);
    const bool k32 = vbits <= 4 && c->bp.near_z >= 0.125f;
    uint32_t *dv = c->dval0.as<uint32_t>(), *dv_alt = c->dval1.as<uint32_t>();
    stage_begin(c, "project", st);
    if (k32)
        UPS_CUDA(c, launch_project_k32(vt, c->bp, c->N, c->per_view, (int)total, *g, c->xyzo.as<float4>(),
                                       c->conic.as<float4>(), c->rect.as<uint2>(), c->count.as<uint32_t>(),
                                       c->dkey0.as<uint32_t>(), dv, vbits, st));
    else
        UPS_CUDA(c, launch_project(vt, c->bp, c->N, c->per_view, (int)total, *g, c->xyzo.as<float4>(),
                                   c->conic.as<float4>(), c->rect.as<uint2>(), c->count.as<uint32_t>(),
                                   c->dkey0.as<uint64_t>(), dv, st));
    stage_end(c, st, 1);
    stage_begin(c, "depth_sort", st);
    if (k32) {
        uint32_t *dk = c->dkey0.as<uint32_t>(), *dk_alt = c->dkey1.as<uint32_t>();
        UPS_CUDA(c, radix_sort_u32(&dk, &dk_alt, &dv, &dv_alt, total, 32, c->sort, st));
        stage_end(c, st, radix_kernels(total, 32));
    } else {
        uint64_t *dk = c->dkey0.as<uint64_t>(), *dk_alt = c->dkey1.as<uint64_t>();
        UPS_CUDA(c, radix_sort_u64(&dk, &dk_alt, &dv, &dv_alt, total, 32 + vbits, c->sort, st));
        stage_end(c, st, radix_kernels(total, 32 + vbits));
    }
    c->dval_sorted = dv;
    stage_begin(c, "offsets", st);
    UPS_CUDA(c, launch_gather_counts(dv, c->count.as<uint32_t>(), c->cnt_sorted.as<uint32_t>(), (int)total, st));
    UPS_CUDA(c, exclusive_scan_u32_u64(c->cnt_sorted.as<uint32_t>(), c->off.as<uint64_t>(), total,
                                       c->scan_scr.ptr, st));
    stage_end(c, st, 4);
    UPS_CUDA(c, cudaMemcpyAsync(c->h_total, c->off.as<uint64_t>() + total, sizeof(uint64_t),
                                cudaMemcpyDeviceToHost, st));
    c->h_total[1] = 0;
    UPS_CUDA(c, cudaMemcpyAsync(c->h_total + 1, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    UPS_CUDA(c, cudaStreamSynchronize(st));
    if (c->h_total[1] != 0) {
        cudaMemsetAsync(c->d_err, 0, sizeof(int), st);
        return fail(c, UPS_ERR_TIMEOUT, "a bounded wait of a kernel ran out of polls in an earlier launch");
    }
    const uint64_t n_inst = *c->h_total;
    if (n_inst >= (uint64_t)UINT32_MAX) return fail(c, UPS_ERR_CAPACITY, "more than 2^32 tile instances");
    c->n_inst = (size_t)n_inst;
    UPS_CUDA(c, c->ikey0.reserve(std::max<size_t>(n_inst, 1) * sizeof(uint32_t)));
    UPS_CUDA(c, c->ikey1.reserve(std::max<size_t>(n_inst, 1) * sizeof(uint32_t)));
    UPS_CUDA(c, c->ival0.reserve(std::max<size_t>(n_inst, 1) * sizeof(uint32_t)));
    UPS_CUDA(c, c->ival1.reserve(std::max<size_t>(n_inst, 1) * sizeof(uint32_t)));
    uint32_t *ik = c->ikey0.as<uint32_t>(), *ik_alt = c->ikey1.as<uint32_t>();
    uint32_t *iv = c->ival0.as<uint32_t>(), *iv_alt = c->ival1.as<uint32_t>();
    stage_begin(c, "emit", st);
    UPS_CUDA(c, launch_emit(vt, c->bp, c->N, (int)total, dv, c->off.as<uint64_t>(), c->rect.as<uint2>(),
                            c->xyzo.as<float4>(), c->conic.as<float4>(), ik, iv, st));
    stage_end(c, st, 1);
    // stable bucket by (view, tile): depth order is kept inside each tile
    c->key_bits = bits_for((size_t)vt.total_tiles);
    stage_begin(c, "tile_sort", st);
    const uint32_t cap = c->cfg.list_cap < 0 || vt.total_tiles >= kMaxBucketBins
                             ? kNoListCap
                             : (uint32_t)(c->cfg.list_cap == 0 ? 1024 : c->cfg.list_cap);
    const bool bucket = vt.total_tiles <= kMaxBucketBins;
    if (bucket) {
        // one pass: values in tile order and the tile ranges; the sorted keys
        // are only rebuilt (from the ranges) when inspected
        const size_t need = bucket_sort_scratch_bytes(n_inst, vt.total_tiles, c->num_sms);
        UPS_CUDA(c, c->sort.hist.reserve(std::max<size_t>(need, 256)));
        UPS_CUDA(c, c->trunc.reserve(((size_t)vt.total_tiles + 31) / 32 * 4));
        UPS_CUDA(c, bucket_sort_u32(ik, iv, iv_alt, n_inst, vt.total_tiles, cap, c->ranges.as<uint2>(),
                                    c->trunc.as<uint32_t>(), c->sort.hist.ptr, c->sort.hist.bytes, c->num_sms, st));
        stage_end(c, st, n_inst ? 6 : 0);
        c->ikey_sorted = nullptr;
        c->ival_sorted = iv_alt;
    } else {
        UPS_CUDA(c, radix_sort_u32(&ik, &ik_alt, &iv, &iv_alt, n_inst, c->key_bits, c->sort, st));
        stage_end(c, st, radix_kernels(n_inst, c->key_bits));
        c->ikey_sorted = ik;
        c->ival_sorted = iv;
        stage_begin(c, "ranges", st);
        UPS_CUDA(c, cudaMemsetAsync(c->ranges.ptr, 0, (size_t)vt.total_tiles * sizeof(uint2), st));
        UPS_CUDA(c, launch_ranges(ik, (uint32_t)n_inst, c->ranges.as<uint2>(), st));
        stage_end(c, st, n_inst ? 1 : 0);
    }
    const bool capped = bucket && cap != kNoListCap && n_inst > 0;
    c->capped = capped;
    if (capped) UPS_CUDA(c, cudaMemsetAsync(c->d_trunc_flag, 0, sizeof(int), st));
    stage_begin(c, "composite_fwd", st);
    UPS_CUDA(c, launch_composite_fwd(vt, c->bp, c->cfg.n_feat, c->N, c->per_view, c->ranges.as<uint2>(),
                                     c->ival_sorted, c->xyzo.as<float4>(), c->conic.as<float4>(),
                                     reinterpret_cast<const float4 *>(g->color), g->feat, *out, st,
                                     capped ? c->trunc.as<uint32_t>() : nullptr, capped ? c->d_trunc_flag : nullptr,
                                     nullptr, c->d_err));
    stage_end(c, st, 1);
    if (capped) {
        // a pixel still open at the end of a capped list: the GPU rebuilds the
        // lists without the cap and blends again.  The work is enqueued now
        // and gated on the blend's flag, so the host never waits for it.
        stage_begin(c, "list_refill", st);
        UPS_CUDA(c, bucket_sort_u32(ik, iv, iv_alt, n_inst, vt.total_tiles, kNoListCap, c->ranges.as<uint2>(),
                                    c->trunc.as<uint32_t>(), c->sort.hist.ptr, c->sort.hist.bytes, c->num_sms, st,
                                    c->d_trunc_flag));
        UPS_CUDA(c, launch_composite_fwd(vt, c->bp, c->cfg.n_feat, c->N, c->per_view, c->ranges.as<uint2>(),
                                         c->ival_sorted, c->xyzo.as<float4>(), c->conic.as<float4>(),
                                         reinterpret_cast<const float4 *>(g->color), g->feat, *out, st, nullptr,
                                         nullptr, c->d_trunc_flag, c->d_err));
        stage_end(c, st, 7);
    }
    c->g_in = *g;
    c->img = *out;
    c->have_fwd = true;
    return UPS_OK;
}

ups_status ups_tracking_uncertainty(ups_ctx *c, const ups_images *img, const ups_targets *tgt,
                                    const ups_residual_cfg *rcfg, float *R, float *sigma2,
                                    unsigned char *motion, ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    if (!c->have_fwd) return fail(c, UPS_ERR_STATE, "ups_tracking_uncertainty needs a forward first");
    if (!img || !tgt || !rcfg) return fail(c, UPS_ERR_ARG, "NULL argument");
    const int nf = c->cfg.n_feat;
    if (!img->color || !img->depth || !img->T || !tgt->color || !tgt->depth ||
        (nf > 0 && (!img->feat || !tgt->feat)))
        return fail(c, UPS_ERR_ARG, "NULL image pointer");
    ups_status s = set_device(c);
    if (s != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    stage_begin(c, "uncertainty", st);
    UPS_CUDA(c, launch_uncertainty(c->vt, nf, c->max_hw, rcfg->lambda_color, rcfg->lambda_depth, rcfg->lambda_feat,
                                   rcfg->t_mask, *img, *tgt, R, sigma2, motion, st));
    stage_end(c, st, 1);
    return UPS_OK;
}

ups_status ups_uncertainty_mlp(ups_ctx *c, const ups_lift_cfg *lcfg, const float *dino, const float *R,
                               const ups_lift_mlp *mlp, float lambda, float scale, float *loss_dev,
                               ups_lift_mlp *d_mlp, float *sigma, unsigned char *motion, ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    if (!c->have_fwd) return fail(c, UPS_ERR_STATE, "ups_uncertainty_mlp needs a forward first");
    if (!lcfg || !dino || !R || !mlp || !mlp->w1 || !mlp->b1 || !mlp->w2 || !mlp->b2 || !loss_dev)
        return fail(c, UPS_ERR_ARG, "NULL argument");
    if (lcfg->n_h < 1 || lcfg->n_h > 4096 || lcfg->patch < 1) return fail(c, UPS_ERR_ARG, "n_h or patch out of range");
    ups_status s = set_device(c);
    if (s != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    int max_np = 0;
    for (int v = 0; v < c->vt.n; ++v) {
        const DevView &cam = c->vt.v[v];
        max_np = std::max(max_np, ((cam.H + lcfg->patch - 1) / lcfg->patch) * ((cam.W + lcfg->patch - 1) / lcfg->patch));
    }
    UPS_CUDA(c, c->unc_scr.reserve(unc_scratch_floats(max_np) * sizeof(float)));
    stage_begin(c, "uncertainty_mlp", st);
    UPS_CUDA(c, cudaMemsetAsync(loss_dev, 0, sizeof(float), st));
    const float g = (float)((double)scale / (double)c->n_pix);
    size_t grid_off = 0;
    int launches = 0;
    for (int v = 0; v < c->vt.n; ++v) {
        const DevView &cam = c->vt.v[v];
        const int hp = (cam.H + lcfg->patch - 1) / lcfg->patch, wp = (cam.W + lcfg->patch - 1) / lcfg->patch;
        const size_t P = (size_t)cam.pix_off;
        UPS_CUDA(c, unc_view(c->num_sms, st, cam.W, cam.H, lcfg->n_h, lcfg->patch, dino + grid_off, wp, hp, R + P,
                             mlp->w1, mlp->b1, mlp->w2, mlp->b2, lambda, g, loss_dev, d_mlp ? d_mlp->w1 : nullptr,
                             d_mlp ? d_mlp->b1 : nullptr, d_mlp ? d_mlp->w2 : nullptr, d_mlp ? d_mlp->b2 : nullptr,
                             sigma ? sigma + P : nullptr, motion ? motion + P : nullptr, c->unc_scr.as<float>(),
                             &launches));
        grid_off += (size_t)hp * wp * lcfg->n_h;
    }
    stage_end(c, st, launches);
    return UPS_OK;
}

namespace {
bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}
}  // namespace

ups_status ups_anchor_update(ups_ctx *c, const ups_anchor_cfg *a, const ups_camera *cam, const float *depth,
                             const unsigned char *motion, const ups_anchors *in, const float *logodds_in,
                             ups_anchors *out, float *logodds_out, int capacity, int *src_index,
                             ups_anchor_result *res, ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    if (!a || !cam || !depth || !in || !out || !logodds_out) return fail(c, UPS_ERR_ARG, "NULL argument");
    const int n = in->n;
    if (n < 0 || capacity < n) return fail(c, UPS_ERR_ARG, "need 0 <= in->n <= capacity");
    if (n > 0 && (!in->pos || !in->feat || !in->offsets || !in->scaling || !logodds_in))
        return fail(c, UPS_ERR_ARG, "NULL input anchor array");
    if (capacity > 0 && (!out->pos || !out->feat || !out->offsets || !out->scaling))
        return fail(c, UPS_ERR_ARG, "NULL output anchor array");
    const float lv[6] = {a->l_prior, a->l_hit, a->l_miss, a->l_min, a->l_max, a->l_prune};
    for (float v : lv)
        if (!std::isfinite(v)) return fail(c, UPS_ERR_ARG, "non-finite log-odds in the anchor config");
    if (!(a->l_min <= a->l_max)) return fail(c, UPS_ERR_ARG, "l_min > l_max");
    if (!(a->voxel > 0.f) || !std::isfinite(a->voxel) || !(a->margin >= 0.f) || !std::isfinite(a->margin) ||
        !std::isfinite(a->near_z))
        return fail(c, UPS_ERR_ARG, "voxel must be > 0, margin >= 0, all finite");
    ViewTable vt;
    size_t npix = 0;
    int mhw = 0;
    ups_status s = build_views(c, cam, 1, vt, npix, mhw);
    if (s != UPS_OK) return s;
    if (npix + (size_t)capacity > ((size_t)1 << 29)) return fail(c, UPS_ERR_ARG, "too many anchors plus pixels");
    const int F = c->cfg.feat_dim, K3 = 3 * c->cfg.k;
    const size_t fb = sizeof(float), cn = (size_t)capacity, nn = (size_t)n;
    const void *ins[5] = {in->pos, in->feat, in->offsets, in->scaling, logodds_in};
    const size_t inb[5] = {3 * nn * fb, F * nn * fb, K3 * nn * fb, 3 * nn * fb, nn * fb};
    const void *outs[6] = {out->pos, out->feat, out->offsets, out->scaling, logodds_out, src_index};
    const size_t outb[6] = {3 * cn * fb, F * cn * fb, K3 * cn * fb, 3 * cn * fb, cn * fb, cn * sizeof(int)};
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j < 5; ++j)
            if (overlaps(outs[i], outb[i], ins[j], inb[j]))
                return fail(c, UPS_ERR_ARG, "output anchor arrays overlap the inputs");
        for (int j = 0; j < i; ++j)
            if (overlaps(outs[i], outb[i], outs[j], outb[j]))
                return fail(c, UPS_ERR_ARG, "output anchor arrays overlap each other");
    }
    s = set_device(c);
    if (s != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    UPS_CUDA(c, c->anchor_scr.reserve(anchor_scratch_bytes(nn, npix)));
    if (!c->h_anchor) UPS_CUDA(c, cudaMallocHost(&c->h_anchor, 8 * sizeof(uint64_t)));
    stage_begin(c, "anchor_update", st);
    int launches = 0;
    uint64_t *summary = nullptr;
    UPS_CUDA(c, anchor_update(vt.v[0], depth, motion, n, in->pos, in->feat, in->offsets, in->scaling, logodds_in, F,
                              K3, a->l_prior, a->l_hit, a->l_miss, a->l_min, a->l_max, a->l_prune, a->voxel,
                              a->margin, a->near_z, capacity, out->pos, out->feat, out->offsets, out->scaling,
                              logodds_out, src_index, c->anchor_scr.ptr, &summary, st, &launches));
    stage_end(c, st, launches);
    UPS_CUDA(c, cudaMemcpyAsync(c->h_anchor, summary, 5 * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    UPS_CUDA(c, cudaStreamSynchronize(st));
    const uint64_t *h = c->h_anchor;
    if (h[4] != 0) return fail(c, UPS_ERR_CAPACITY, "voxel table full");
    const long long kept = (long long)h[0], fresh = (long long)h[1];
    const long long ins_n = std::max(0LL, std::min(fresh, (long long)capacity - kept));
    out->n = (int)(kept + ins_n);
    if (res) {
        res->n_kept = (int)kept;
        res->n_inserted = (int)ins_n;
        res->n_dropped = (int)(fresh - ins_n);
        res->n_hit = (int)h[2];
        res->n_miss = (int)h[3];
    }
    return UPS_OK;
}

ups_status ups_ssim_loss(ups_ctx *c, const float *color, const float *t_color, const float *weight, float scale,
                         float *loss_dev, float *d_color, ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    if (!c->have_fwd) return fail(c, UPS_ERR_STATE, "ups_ssim_loss needs a forward first");
    if (!color || !t_color || !loss_dev) return fail(c, UPS_ERR_ARG, "NULL argument");
    ups_status s = set_device(c);
    if (s != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    if (!c->ssim_window) {
        UPS_CUDA(c, ssim_set_window());
        c->ssim_window = true;
    }
    UPS_CUDA(c, c->ssim_g.reserve((size_t)9 * c->n_pix * sizeof(float)));
    stage_begin(c, "ssim", st);
    UPS_CUDA(c, cudaMemsetAsync(loss_dev, 0, sizeof(float), st));
    const float g = (float)((double)scale / (3.0 * (double)c->n_pix));
    UPS_CUDA(c, launch_ssim(c->vt, color, t_color, weight, c->ssim_g.as<float>(), g, loss_dev, d_color, st));
    const int launches = d_color ? 2 : 1;
    stage_end(c, st, launches);
    return UPS_OK;
}

ups_status ups_feature_lift(ups_ctx *c, const ups_lift_cfg *lcfg, const float *feat, const float *dino,
                            const ups_lift_mlp *mlp, const float *weight, float scale, float *loss_dev,
                            ups_lift_mlp *d_mlp, float *d_feat, ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    if (!c->have_fwd) return fail(c, UPS_ERR_STATE, "ups_feature_lift needs a forward first");
    if (!lcfg || !feat || !dino || !mlp || !mlp->w1 || !mlp->b1 || !mlp->w2 || !mlp->b2 || !loss_dev)
        return fail(c, UPS_ERR_ARG, "NULL argument");
    const int nf = c->cfg.n_feat;
    if (nf <= 0) return fail(c, UPS_ERR_ARG, "feature lifting needs n_feat > 0");
    if (lcfg->n_h < 4 || lcfg->n_h > 4096 || lcfg->n_h % 4 != 0 || lcfg->patch < 1 || lcfg->patch > 32)
        return fail(c, UPS_ERR_ARG, "n_h must be a multiple of 4 in [4, 4096] and patch in [1, 32]");
    if (reinterpret_cast<uintptr_t>(dino) % 16 != 0 || reinterpret_cast<uintptr_t>(mlp->b2) % 16 != 0)
        return fail(c, UPS_ERR_ARG, "dino and mlp->b2 must be 16-byte aligned");
    ups_status s = set_device(c);
    if (s != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    size_t np_total = 0;
    for (int v = 0; v < c->vt.n; ++v) {
        const DevView &cam = c->vt.v[v];
        np_total += (size_t)((cam.H + lcfg->patch - 1) / lcfg->patch) * (size_t)((cam.W + lcfg->patch - 1) / lcfg->patch);
    }
    if (np_total >= (size_t)INT32_MAX / 128) return fail(c, UPS_ERR_ARG, "too many DINO patches");
    UPS_CUDA(c, c->lift_scr.reserve(lift_scratch_floats(np_total) * sizeof(float)));
    stage_begin(c, "lift", st);
    UPS_CUDA(c, cudaMemsetAsync(loss_dev, 0, sizeof(float), st));
    const float g = (float)((double)scale / (double)c->n_pix);
    int launches = 0;
    UPS_CUDA(c, lift_all(c->num_sms, st, c->vt, nf, lcfg->n_h, lcfg->patch, feat, dino, mlp->w1, mlp->b1, mlp->w2,
                         mlp->b2, g, weight, loss_dev, d_mlp ? d_mlp->w1 : nullptr, d_mlp ? d_mlp->b1 : nullptr,
                         d_mlp ? d_mlp->w2 : nullptr, d_mlp ? d_mlp->b2 : nullptr, d_feat, c->lift_scr.as<float>(),
                         c->d_err, &launches));
    stage_end(c, st, launches);
    return UPS_OK;
}

ups_status ups_loss_weighted(ups_ctx *c, const ups_images *img, const ups_targets *tgt,
                             const ups_loss_cfg *lcfg, const ups_gaussians *g, float *loss_dev,
                             ups_images *dL, ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    if (!c->have_fwd) return fail(c, UPS_ERR_STATE, "ups_loss_weighted needs a forward first");
    if (!img || !tgt || !lcfg || !loss_dev || !dL) return fail(c, UPS_ERR_ARG, "NULL argument");
    const int nf = c->cfg.n_feat;
    if (!img->color || !img->depth || !tgt->color || !tgt->depth || !dL->color || !dL->depth ||
        (nf > 0 && (!img->feat || !tgt->feat || !dL->feat)))
        return fail(c, UPS_ERR_ARG, "NULL image pointer");
    ups_status s = set_device(c);
    if (s != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    stage_begin(c, "loss", st);
    UPS_CUDA(c, cudaMemsetAsync(loss_dev, 0, sizeof(float), st));
    float inv_norm = (float)(1.0 / (double)c->n_pix);
    UPS_CUDA(c, launch_loss(c->vt, nf, c->max_hw, lcfg->lambda_color, lcfg->lambda_depth,
                            lcfg->lambda_feat, lcfg->l2, inv_norm, *img, *tgt, *dL, loss_dev, st));
    if (g && lcfg->lambda_scale != 0.f) {
        size_t sets = g->per_view ? (size_t)c->n_sets : 1;
        size_t n = sets * (size_t)g->n;
        UPS_CUDA(c, launch_scale_mean(reinterpret_cast<const float4 *>(g->scale), n,
                                      (float)(lcfg->lambda_scale / (3.0 * (double)n)), loss_dev, st));
        c->launches += 1;
    }
    stage_end(c, st, 1);
    return UPS_OK;
}

ups_status ups_render_backward(ups_ctx *c, const ups_image_grads *dL, unsigned mask,
                               float scale_grad, ups_gaussians *grad, float *d_pose,
                               ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    if (!c->have_fwd) return fail(c, UPS_ERR_STATE, "ups_render_backward needs a forward first");
    if (!dL) return fail(c, UPS_ERR_ARG, "dL is NULL");
    if ((mask & UPS_GRAD_POSE) && !d_pose) return fail(c, UPS_ERR_ARG, "d_pose is NULL");
    if (mask & UPS_GRAD_GAUSS) {
        ups_status s = check_gaussians(c, grad, "grad");
        if (s != UPS_OK) return s;
        if (grad->n != c->N || (grad->per_view ? 1 : 0) != c->per_view)
            return fail(c, UPS_ERR_ARG, "grad must have the forward input's n and per_view");
    }
    ups_status s = set_device(c);
    if (s != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    const int nf = c->cfg.n_feat;
    const size_t rec = (size_t)g2_stride(nf);
    UPS_CUDA(c, c->g2.reserve(c->total_gv * rec * sizeof(float)));
    UPS_CUDA(c, cudaMemsetAsync(c->g2.ptr, 0, c->total_gv * rec * sizeof(float), st));
    stage_begin(c, "composite_bwd", st);
    UPS_CUDA(c, launch_composite_bwd(c->vt, c->bp, nf, c->N, c->per_view, c->ranges.as<uint2>(),
                                     c->ival_sorted, c->xyzo.as<float4>(), c->conic.as<float4>(),
                                     reinterpret_cast<const float4 *>(c->g_in.color), c->g_in.feat,
                                     c->img.T, c->img.n_contrib, *dL, c->g2.as<float>(), st, c->d_err));
    stage_end(c, st, 1);
    if (mask & UPS_GRAD_POSE)
        UPS_CUDA(c, cudaMemsetAsync(d_pose, 0, sizeof(float) * 6 * c->vt.n, st));
    if ((mask & UPS_GRAD_GAUSS) && c->shared_sets) {
        size_t n = (size_t)c->N * (size_t)c->n_sets;
        UPS_CUDA(c, cudaMemsetAsync(grad->mean_opacity, 0, n * sizeof(float4), st));
        UPS_CUDA(c, cudaMemsetAsync(grad->scale, 0, n * sizeof(float4), st));
        UPS_CUDA(c, cudaMemsetAsync(grad->quat, 0, n * sizeof(float4), st));
        UPS_CUDA(c, cudaMemsetAsync(grad->color, 0, n * sizeof(float4), st));
        if (nf) UPS_CUDA(c, cudaMemsetAsync(grad->feat, 0, n * nf * sizeof(float), st));
    }
    if (mask & (UPS_GRAD_POSE | UPS_GRAD_GAUSS)) {
        stage_begin(c, "project_bwd", st);
        UPS_CUDA(c, launch_project_bwd(c->vt, c->bp, c->N, c->shared_sets ? 0 : 1, (int)c->total_gv, nf, mask,
                                       scale_grad, c->g_in, c->g2.as<float>(), grad, d_pose, st));
        stage_end(c, st, 1);
    }
    c->have_bwd = true;
    return UPS_OK;
}

ups_status ups_decode_backward(ups_ctx *c, const ups_anchors *anc, const ups_mlp *mlp,
                               const ups_camera *cams, int n_views, const ups_gaussians *dG,
                               unsigned mask, ups_mlp *d_mlp, ups_anchors *d_anc, float *d_pose,
                               ups_stream stream) {
    if (!c) return UPS_ERR_ARG;
    if (!anc || !mlp || !dG) return fail(c, UPS_ERR_ARG, "NULL argument");
    if (anc->n < 1 || !anc->pos || !anc->feat || !anc->offsets || !anc->scaling)
        return fail(c, UPS_ERR_ARG, "anchors: n < 1 or NULL pointer");
    if (!dG->per_view || (size_t)dG->n != (size_t)anc->n * c->cfg.k)
        return fail(c, UPS_ERR_ARG, "dG must be per_view with n == anchors.n * k");
    ups_status s = check_gaussians(c, dG, "dG");
    if (s != UPS_OK) return s;
    if ((mask & UPS_GRAD_MLP) && (!d_mlp || !d_mlp->w1 || !d_mlp->b1 || !d_mlp->w2 || !d_mlp->b2))
        return fail(c, UPS_ERR_ARG, "d_mlp: NULL pointer");
    if ((mask & UPS_GRAD_ANCHOR) &&
        (!d_anc || !d_anc->pos || !d_anc->feat || !d_anc->offsets || !d_anc->scaling))
        return fail(c, UPS_ERR_ARG, "d_anchors: NULL pointer");
    if ((mask & UPS_GRAD_POSE) && !d_pose) return fail(c, UPS_ERR_ARG, "d_pose is NULL");
    ViewTable vt;
    size_t npix;
    int mhw;
    if ((s = build_views(c, cams, n_views, vt, npix, mhw)) != UPS_OK) return s;
    if ((s = set_device(c)) != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    float *scratch = nullptr;
    if ((mask & UPS_GRAD_MLP) && d_mlp) {
        UPS_CUDA(c, c->dec_scratch.reserve(decode_bwd_scratch_bytes(anc->n, n_views, c->cfg.k, c->cfg.n_feat)));
        scratch = c->dec_scratch.as<float>();
    }
    const dbwd::StageHook hook{[](void *u, const char *name, bool begin, cudaStream_t s) {
                                   ups_ctx *cc = static_cast<ups_ctx *>(u);
                                   if (begin)
                                       stage_begin(cc, name, s);
                                   else
                                       stage_end(cc, s, 1);
                               },
                               c};
    UPS_CUDA(c, launch_decode_bwd(vt, anc->n, c->cfg.k, c->cfg.n_feat, *anc, *mlp, *dG, mask, d_mlp, d_anc,
                                  d_pose, c->cfg.decode_bf16 && c->cfg.decode_bwd_bf16 ? 1 : 0,
                                  c->cfg.opacity_tanh, scratch, c->d_err,
                                  c->num_sms, hook, st));
    return UPS_OK;
}

ups_status ups_get_stats(ups_ctx *c, ups_stats *out) {
    if (!c || !out) return UPS_ERR_ARG;
    if (!c->have_fwd) return fail(c, UPS_ERR_STATE, "no forward yet");
    std::memset(out, 0, sizeof(*out));
    out->n_views = c->vt.n;
    out->n_gaussian_views = (long long)c->total_gv;
    out->n_instances = (long long)c->n_inst;
    out->n_tiles = c->vt.total_tiles;
    out->n_pixels = (long long)c->n_pix;
    out->key_bits = c->key_bits;
    size_t listed = 0;
    int refilled = 0;
    const ups_status ls = listed_entries(c, &listed, &refilled);
    if (ls != UPS_OK) return ls;
    out->n_listed = (long long)listed;
    out->list_refills = refilled;
    // visible = Gaussian-views with at least one tile (count > 0)
    std::vector<uint32_t> h(c->total_gv);
    if (c->total_gv) {
        UPS_CUDA(c, cudaSetDevice(c->device));
        UPS_CUDA(c, cudaStreamSynchronize(c->last_stream));
        UPS_CUDA(c, cudaMemcpy(h.data(), c->count.ptr, c->total_gv * 4, cudaMemcpyDeviceToHost));
    }
    long long vis = 0;
    for (uint32_t x : h) vis += x > 0;
    out->n_visible = vis;
    return UPS_OK;
}

ups_status ups_copy_buffer(ups_ctx *c, int which, void *dst, size_t bytes, size_t *size) {
    if (!c) return UPS_ERR_ARG;
    if (!c->have_fwd) return fail(c, UPS_ERR_STATE, "no forward yet");
    size_t listed = 0;
    int refilled = 0;
    if (which <= 1) {
        ups_status s = listed_entries(c, &listed, &refilled);
        if (s != UPS_OK) return s;
    }
    const void *src = nullptr;
    size_t sz = 0;
    switch (which) {
        case 0: src = c->ival_sorted; sz = listed * 4; break;
        case 1:
            sz = listed * 4;
            if (!c->ikey_sorted && sz) {
                UPS_CUDA(c, cudaSetDevice(c->device));
                UPS_CUDA(c, keys_from_ranges(c->ranges.as<uint2>(), c->vt.total_tiles, c->ikey1.as<uint32_t>(),
                                             c->last_stream));
                c->ikey_sorted = c->ikey1.as<uint32_t>();
            }
            src = c->ikey_sorted;
            break;
        case 2: src = c->ranges.ptr; sz = (size_t)c->vt.total_tiles * 8; break;
        case 3: src = c->xyzo.ptr; sz = c->total_gv * 16; break;
        case 4: src = c->conic.ptr; sz = c->total_gv * 16; break;
        case 5: src = c->rect.ptr; sz = c->total_gv * 8; break;
        case 6:
            if (!c->have_bwd) return fail(c, UPS_ERR_STATE, "no backward yet");
            src = c->g2.ptr;
            sz = c->total_gv * g2_stride(c->cfg.n_feat) * 4;
            break;
        default: return fail(c, UPS_ERR_ARG, "unknown buffer id");
    }
    if (size) *size = sz;
    if (!dst) return UPS_OK;
    size_t n = std::min(bytes, sz);
    UPS_CUDA(c, cudaSetDevice(c->device));
    UPS_CUDA(c, cudaStreamSynchronize(c->last_stream));
    if (n) UPS_CUDA(c, cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost));
    return UPS_OK;
}

ups_status ups_profile_enable(ups_ctx *c, int on) {
    if (!c) return UPS_ERR_ARG;
    c->prof = on != 0;
    return UPS_OK;
}

ups_status ups_profile_read(ups_ctx *c, char *buf, size_t len, long long *launches) {
    if (!c) return UPS_ERR_ARG;
    ups_status s = set_device(c);
    if (s != UPS_OK) return s;
    for (auto &r : c->pending) {
        UPS_CUDA(c, cudaEventSynchronize(r.b));
        float ms = 0.f;
        UPS_CUDA(c, cudaEventElapsedTime(&ms, r.a, r.b));
        auto &a = c->acc[r.name];
        a.first += ms;
        a.second += 1;
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->pending.clear();
    std::string js = "{";
    bool first = true;
    for (auto &kv : c->acc) {
        char tmp[160];
        std::snprintf(tmp, sizeof(tmp), "%s\"%s\": [%.6f, %lld]", first ? "" : ", ", kv.first.c_str(),
                      kv.second.first, kv.second.second);
        js += tmp;
        first = false;
    }
    js += "}";
    if (buf && len) {
        std::strncpy(buf, js.c_str(), len - 1);
        buf[len - 1] = 0;
    }
    if (launches) *launches = c->launches;
    c->acc.clear();
    c->launches = 0;
    return js.size() < len ? UPS_OK : fail(c, UPS_ERR_ARG, "profile buffer too small");
}

}  // extern "C"
