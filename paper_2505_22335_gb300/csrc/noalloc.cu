// ups_render_forward_static: the render forward with all of its scratch in one
// file-scope device array, for callers that must not allocate GPU memory.
//
// Who needs it: a real-time tracking front end (or any embedder) that runs
// its frames at camera rate inside a fixed GPU memory budget.  cudaMalloc and
// cudaFree synchronise the device and may block for milliseconds, and some
// embedders hand this library a memory budget it may not grow, so such a
// caller cannot use a context (whose scratch grows with cudaMalloc).  This
// entry point needs no context and calls no allocating routine: its scratch
// is the static array below, fixed in size, which every GPU that loads the
// library keeps until the process exits.
//
// Limits (UPS_ERR_CAPACITY when exceeded):
//   n * n_views            <= 65,536 Gaussian-views  (checked before any launch)
//   tiles over all views   <= 8,192 16x16 tiles      (checked before any launch)
//   tile instances         <= 524,288                (known only after the
//       projection, the depth sort and the count scan have run and the stream
//       has been synchronised: on this error the scratch array has been
//       written and the output images have not)
// Scratch size: about 14 MB.
//
// The array is shared by every call on a device and keeps the last call's
// contents; everything a call reads is written (or cleared) by that call
// first.  Calls that overlap on the GPU (two streams, two host threads) race
// on the array: serialise them.  Every call looks up the array's device
// address (cudaGetSymbolAddress, which allocates nothing) on the caller's
// current device, so a device reset or a new primary context, which may load
// the module at another address, is followed.  Every call synchronises its
// stream once (to read the instance count).
#include <string>

#include "common.cuh"

namespace ups {

cudaError_t launch_project(const ViewTable &vt, const BlendParams &bp, int N, int per_view,
                           int total, const ups_gaussians &g, float4 *xyzo, float4 *conic,
                           uint2 *rect, uint32_t *count, uint64_t *dkey, uint32_t *dval,
                           cudaStream_t st);
cudaError_t launch_gather_counts(const uint32_t *sorted_gv, const uint32_t *count, uint32_t *out,
                                 int total, cudaStream_t st);
cudaError_t launch_emit(const ViewTable &vt, const BlendParams &bp, int N, int total, const uint32_t *sorted_gv,
                        const uint64_t *off, const uint2 *rect, const float4 *xyzo, const float4 *conic,
                        uint32_t *ikey, uint32_t *ival, cudaStream_t st);
cudaError_t launch_ranges(const uint32_t *ikey, uint32_t n, uint2 *ranges, cudaStream_t st);
cudaError_t launch_composite_fwd(const ViewTable &vt, const BlendParams &bp, int n_feat, int N,
                                 int per_view, const uint2 *ranges, const uint32_t *ival,
                                 const float4 *xyzo, const float4 *conic, const float4 *color,
                                 const float *feat, const ups_images &out, cudaStream_t st,
                                 const uint32_t *trunc = nullptr, int *trunc_flag = nullptr,
                                 const int *gate = nullptr, int *err = nullptr);
cudaError_t radix_sort_u32_fixed(uint32_t **key_io, uint32_t **key_alt, uint32_t **val_io,
                                 uint32_t **val_alt, size_t n, int end_bit, void *scratch,
                                 size_t scratch_bytes, cudaStream_t st);
cudaError_t radix_sort_u64_fixed(uint64_t **key_io, uint64_t **key_alt, uint32_t **val_io,
                                 uint32_t **val_alt, size_t n, int end_bit, void *scratch,
                                 size_t scratch_bytes, cudaStream_t st);
void set_global_error(const std::string &msg);

}  // namespace ups

using namespace ups;

namespace {

constexpr size_t kMaxGV = size_t(1) << 16;
constexpr size_t kMaxTiles = size_t(1) << 13;
constexpr size_t kMaxInst = size_t(1) << 19;
constexpr size_t kSortScratch = size_t(512) << 10;  // radix histograms + their scan
constexpr size_t kScanScratch = size_t(4) << 10;    // scan partials of the counts

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// byte offsets of the sub-buffers
constexpr size_t oXyzo = 0;
constexpr size_t oConic = oXyzo + al(kMaxGV * 16);
constexpr size_t oRect = oConic + al(kMaxGV * 16);
constexpr size_t oCount = oRect + al(kMaxGV * 8);
constexpr size_t oDkey0 = oCount + al(kMaxGV * 4);
constexpr size_t oDkey1 = oDkey0 + al(kMaxGV * 8);
constexpr size_t oDval0 = oDkey1 + al(kMaxGV * 8);
constexpr size_t oDval1 = oDval0 + al(kMaxGV * 4);
constexpr size_t oCnt = oDval1 + al(kMaxGV * 4);
constexpr size_t oOff = oCnt + al(kMaxGV * 4);
constexpr size_t oIkey0 = oOff + al((kMaxGV + 1) * 8);
constexpr size_t oIkey1 = oIkey0 + al(kMaxInst * 4);
constexpr size_t oIval0 = oIkey1 + al(kMaxInst * 4);
constexpr size_t oIval1 = oIval0 + al(kMaxInst * 4);
constexpr size_t oRanges = oIval1 + al(kMaxInst * 4);
constexpr size_t oSort = oRanges + al(kMaxTiles * 8);
constexpr size_t oScan = oSort + kSortScratch;
constexpr size_t kScratchBytes = oScan + kScanScratch;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

ups_status fail(ups_status s, const std::string &msg) {
    set_global_error("ups_render_forward_static: " + msg);
    return s;
}

// device address of g_static_scratch on the current device (the host-side
// name of the array is not a device address)
ups_status scratch_address(unsigned char **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
        return fail(UPS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = static_cast<unsigned char *>(p);
    return UPS_OK;
}

#define NA_CUDA(expr)                                                               \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess)                                                      \
            return fail(UPS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int bits_for(size_t n) {
    int b = 0;
    while (b < 63 && ((size_t)1 << b) < n) ++b;
    return b;
}

}  // namespace

extern "C" ups_status ups_render_forward_static(const ups_config *cfg, const ups_gaussians *g,
                                                const ups_camera *cams, int n_views,
                                                ups_images *out, ups_stream stream) {
    if (!cfg || !g || !cams || !out) return fail(UPS_ERR_ARG, "NULL argument");
    const int nf = cfg->n_feat;
    if (nf != 0 && nf != 16 && nf != 32) return fail(UPS_ERR_ARG, "n_feat must be 0, 16 or 32");
    if (!(cfg->alpha_min > 0.f) || !(cfg->alpha_max >= cfg->alpha_min) || !(cfg->alpha_max < 1.f) ||
        !(cfg->t_min >= 0.f) || !(cfg->dilation >= 0.f) || !(cfg->near_z > 0.f) || !(cfg->guard > 0.f))
        return fail(UPS_ERR_ARG, "threshold out of range");
    if (g->n < 1) return fail(UPS_ERR_ARG, "g.n must be >= 1");
    const void *ptrs[4] = {g->mean_opacity, g->scale, g->quat, g->color};
    for (const void *p : ptrs)
        if (!p || !aligned16(p)) return fail(UPS_ERR_ARG, "NULL or unaligned Gaussian attribute");
    if (nf && (!g->feat || !aligned16(g->feat))) return fail(UPS_ERR_ARG, "g.feat NULL or unaligned");
    if (!out->color || !out->depth || !out->T || !out->n_contrib || (nf && !out->feat))
        return fail(UPS_ERR_ARG, "NULL image pointer");
    if (n_views < 1 || n_views > UPS_MAX_VIEWS) return fail(UPS_ERR_ARG, "n_views out of range");
    const size_t total = (size_t)g->n * n_views;
    if (total > kMaxGV)
        return fail(UPS_ERR_CAPACITY, "n * n_views = " + std::to_string(total) + " exceeds 65536");

    ViewTable vt{};
    vt.n = n_views;
    int tiles = 0;
    size_t pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const ups_camera &cm = cams[v];
        if (cm.width < 1 || cm.height < 1 || cm.width > 16384 || cm.height > 16384 ||
            !(cm.fx > 0) || !(cm.fy > 0))
            return fail(UPS_ERR_ARG, "camera " + std::to_string(v) + ": bad intrinsics or size");
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
        d.limx = cfg->guard * 0.5f * cm.width / cm.fx;
        d.limy = cfg->guard * 0.5f * cm.height / cm.fy;
        d.t_norm = cm.t_norm;
        tiles += d.tiles_x * d.tiles_y;
        pix += (size_t)cm.width * cm.height;
        if ((size_t)tiles > kMaxTiles)
            return fail(UPS_ERR_CAPACITY, "more than 8192 tiles over all views");
    }
    vt.total_tiles = tiles;
    const BlendParams bp{cfg->alpha_min, cfg->alpha_max, cfg->t_min, cfg->dilation, cfg->near_z};
    const int N = g->n, per_view = g->per_view ? 1 : 0;
    for (int v = 0; v < n_views; ++v) {
        vt.v[v].set = per_view ? v : 0;
        vt.v[v].set_first = per_view || v == 0;
    }

    unsigned char *base = nullptr;
    ups_status s = scratch_address(&base);
    if (s != UPS_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    float4 *xyzo = reinterpret_cast<float4 *>(base + oXyzo);
    float4 *conic = reinterpret_cast<float4 *>(base + oConic);
    uint2 *rect = reinterpret_cast<uint2 *>(base + oRect);
    uint32_t *count = reinterpret_cast<uint32_t *>(base + oCount);
    uint64_t *dk = reinterpret_cast<uint64_t *>(base + oDkey0);
    uint64_t *dk_alt = reinterpret_cast<uint64_t *>(base + oDkey1);
    uint32_t *dv = reinterpret_cast<uint32_t *>(base + oDval0);
    uint32_t *dv_alt = reinterpret_cast<uint32_t *>(base + oDval1);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(base + oCnt);
    uint64_t *off = reinterpret_cast<uint64_t *>(base + oOff);
    uint32_t *ik = reinterpret_cast<uint32_t *>(base + oIkey0);
    uint32_t *ik_alt = reinterpret_cast<uint32_t *>(base + oIkey1);
    uint32_t *iv = reinterpret_cast<uint32_t *>(base + oIval0);
    uint32_t *iv_alt = reinterpret_cast<uint32_t *>(base + oIval1);
    uint2 *ranges = reinterpret_cast<uint2 *>(base + oRanges);
    void *sort_scr = base + oSort;
    void *scan_scr = base + oScan;

    NA_CUDA(launch_project(vt, bp, N, per_view, (int)total, *g, xyzo, conic, rect, count, dk, dv, st));
    NA_CUDA(radix_sort_u64_fixed(&dk, &dk_alt, &dv, &dv_alt, total, 32 + bits_for((size_t)n_views),
                                 sort_scr, kSortScratch, st));
    NA_CUDA(launch_gather_counts(dv, count, cnt, (int)total, st));
    NA_CUDA(exclusive_scan_u32_u64(cnt, off, total, scan_scr, st));
    uint64_t n_inst = 0;
    NA_CUDA(cudaMemcpyAsync(&n_inst, off + total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (n_inst > kMaxInst)
        return fail(UPS_ERR_CAPACITY, std::to_string(n_inst) + " tile instances exceed 524288");
    NA_CUDA(launch_emit(vt, bp, N, (int)total, dv, off, rect, xyzo, conic, ik, iv, st));
    NA_CUDA(radix_sort_u32_fixed(&ik, &ik_alt, &iv, &iv_alt, (size_t)n_inst,
                                 bits_for((size_t)vt.total_tiles), sort_scr, kSortScratch, st));
    NA_CUDA(cudaMemsetAsync(ranges, 0, (size_t)vt.total_tiles * sizeof(uint2), st));
    NA_CUDA(launch_ranges(ik, (uint32_t)n_inst, ranges, st));
    NA_CUDA(launch_composite_fwd(vt, bp, nf, N, per_view, ranges, iv, xyzo, conic,
                                 reinterpret_cast<const float4 *>(g->color), g->feat, *out, st));
    return UPS_OK;
}
