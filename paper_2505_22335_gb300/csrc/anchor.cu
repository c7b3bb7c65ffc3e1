// Probabilistic anchors (Sec. 3.3 "Adaptively Structured Gaussian", Eq. 7):
// one keyframe updates the occupancy log-odds of every anchor, deletes the
// anchors whose posterior falls below the pruning level and allocates anchors
// in the empty voxels of the keyframe's static surface (the probabilistic
// octree of Sec. 1, read as a voxel grid of edge `voxel`).
//
// Eq. 7 is OctoMap's Bayes update; in log-odds it is an addition,
//   L(n|z_1:t) = L(n|z_1:t-1) + L(n|z_t) - L(n),
// clamped to [l_min, l_max].  Every decision (the pixel of an anchor, its
// observation, the voxel of a pixel) is taken in FP32 with one rounding per
// operation in a fixed order (the __f*_rn intrinsics are never contracted into
// FMAs), so the results do not depend on the compiler.
//
// Launches for n anchors and P keyframe pixels:
//   k_observe       anchor -> pixel -> hit / miss / none, posterior, keep flag
//   scan(keep)      output row of each kept anchor (3 launches)
//   k_compact       kept rows into the output arrays, in input order
//   k_hash_anchors  voxels of the kept anchors into an open-addressing table
//   k_hash_pixels   voxel of every static pixel into the table; the voxel's
//                   owner becomes its lowest pixel index (atomicMin)
//   k_first         flag the pixels that own a voxel no kept anchor holds
//   scan(flags)     raster-order rank of each new voxel (3 launches)
//   k_insert        a new anchor at the centre of each new voxel, to capacity
//   k_summary       the five counts the host reads back
#include <algorithm>

#include "common.cuh"

namespace ups {

namespace {

constexpr int kAThreads = 256;
constexpr int kVoxRange = 1 << 20;                  // voxel indices in [-2^20, 2^20)
constexpr unsigned long long kEmptyKey = ~0ull;      // table slot without a key
constexpr int kNoOwner = 0x7f7f7f7f;                 // memset byte 0x7f: above every pixel index

struct AParams {
    float dh, dm;          // L(hit) - L(n), L(miss) - L(n)
    float l_min, l_max, l_prune;
    float l_new;           // log-odds of a new anchor: the prior plus one hit, clamped
    float voxel, margin, near_z;
};

// voxel (floor(x / voxel) per axis, FP32) packed as three 21-bit fields
// (bits 0..62: never kEmptyKey); false when an index is out of range
__device__ __forceinline__ bool voxel_key(float x, float y, float z, float voxel, unsigned long long &key) {
    const float q0 = floorf(__fdiv_rn(x, voxel)), q1 = floorf(__fdiv_rn(y, voxel)), q2 = floorf(__fdiv_rn(z, voxel));
    const float lo = -(float)kVoxRange, hi = (float)kVoxRange;
    if (!(q0 >= lo && q0 < hi && q1 >= lo && q1 < hi && q2 >= lo && q2 < hi)) return false;
    key = ((unsigned long long)((int)q0 + kVoxRange) << 42) | ((unsigned long long)((int)q1 + kVoxRange) << 21) |
          (unsigned long long)((int)q2 + kVoxRange);
    return true;
}

// 64-bit finaliser of MurmurHash3
__device__ __forceinline__ uint32_t key_hash(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k;
}

// Slot of `key` in the linear-probing table (inserted if absent); -1 if the
// table is full (it is sized for a load of at most 1/2, so this does not happen).
// Keys only ever go from empty to a key, so a stale empty read is settled by
// the CAS and a non-empty read is final.
__device__ __forceinline__ int table_slot(unsigned long long *keys, uint32_t mask, unsigned long long key) {
    uint32_t h = key_hash(key) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        unsigned long long cur = keys[h];
        if (cur == key) return (int)h;
        if (cur == kEmptyKey) {
            cur = atomicCAS(&keys[h], kEmptyKey, key);
            if (cur == kEmptyKey || cur == key) return (int)h;
        }
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ float dot3_rn(float a, float b, float c, float x, float y, float z) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a, x), __fmul_rn(b, y)), __fmul_rn(c, z));
}

// Observation of each anchor (0 none, 1 hit, 2 miss), its posterior and keep flag.
__global__ void __launch_bounds__(kAThreads) k_observe(int n, const float *__restrict__ pos,
                                                       const float *__restrict__ lin, DevView cam,
                                                       const float *__restrict__ depth,
                                                       const uint8_t *__restrict__ motion, AParams ap,
                                                       float *__restrict__ lnew, uint32_t *__restrict__ keep,
                                                       unsigned int *__restrict__ counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int obs = 0;
    if (i < n) {
        const float x = pos[3 * (size_t)i], y = pos[3 * (size_t)i + 1], z = pos[3 * (size_t)i + 2];
        const float X = __fadd_rn(dot3_rn(cam.R[0], cam.R[1], cam.R[2], x, y, z), cam.t[0]);
        const float Y = __fadd_rn(dot3_rn(cam.R[3], cam.R[4], cam.R[5], x, y, z), cam.t[1]);
        const float Z = __fadd_rn(dot3_rn(cam.R[6], cam.R[7], cam.R[8], x, y, z), cam.t[2]);
        if (Z > ap.near_z) {
            const float u = __fadd_rn(__fmul_rn(cam.fx, __fdiv_rn(X, Z)), cam.cx);
            const float v = __fadd_rn(__fmul_rn(cam.fy, __fdiv_rn(Y, Z)), cam.cy);
            const float fu = floorf(__fadd_rn(u, 0.5f)), fv = floorf(__fadd_rn(v, 0.5f));
            if (fu >= 0.f && fu < (float)cam.W && fv >= 0.f && fv < (float)cam.H) {
                const size_t p = (size_t)(int)fv * cam.W + (int)fu;
                const float D = depth[p];
                if (D > ap.near_z) {
                    const float lo = __fsub_rn(D, ap.margin), hi = __fadd_rn(D, ap.margin);
                    if (Z < lo)
                        obs = 2;  // the ray to the surface passed through the anchor
                    else if (Z <= hi)
                        obs = (motion && motion[p]) ? 2 : 1;
                }
            }
        }
        float l = lin[i];
        if (obs) l = fminf(fmaxf(__fadd_rn(l, obs == 1 ? ap.dh : ap.dm), ap.l_min), ap.l_max);
        lnew[i] = l;
        keep[i] = l >= ap.l_prune ? 1u : 0u;
    }
    const unsigned hb = __ballot_sync(0xffffffffu, obs == 1), mb = __ballot_sync(0xffffffffu, obs == 2);
    if ((threadIdx.x & 31) == 0) {
        if (hb) atomicAdd(counts, (unsigned)__popc(hb));
        if (mb) atomicAdd(counts + 1, (unsigned)__popc(mb));
    }
}

// One output array per blockIdx.y: kept row i goes to row off[i].
struct CompactArgs {
    const float *src[5];
    float *dst[5];
    int width[5];
    int *src_index;
};
__global__ void __launch_bounds__(kAThreads) k_compact(int n, const uint32_t *__restrict__ keep,
                                                       const uint64_t *__restrict__ off, CompactArgs a) {
    const int y = blockIdx.y;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    if (y == 5) {
        if (!a.src_index) return;
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n; i += stride)
            if (keep[i]) a.src_index[off[i]] = (int)i;
        return;
    }
    // a switch, not a.src[y]: indexing the parameter arrays would copy them to the stack
    int w;
    const float *s;
    float *d;
    switch (y) {
        case 0: w = a.width[0], s = a.src[0], d = a.dst[0]; break;
        case 1: w = a.width[1], s = a.src[1], d = a.dst[1]; break;
        case 2: w = a.width[2], s = a.src[2], d = a.dst[2]; break;
        case 3: w = a.width[3], s = a.src[3], d = a.dst[3]; break;
        default: w = a.width[4], s = a.src[4], d = a.dst[4]; break;
    }
    const size_t total = (size_t)n * w;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += stride) {
        const size_t i = e / w;
        if (keep[i]) d[off[i] * w + (e - i * w)] = s[e];
    }
}

__global__ void __launch_bounds__(kAThreads) k_hash_anchors(int n, const float *__restrict__ pos,
                                                            const uint32_t *__restrict__ keep, float voxel,
                                                            unsigned long long *keys, int *vals, uint32_t mask,
                                                            int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !keep[i]) return;
    unsigned long long key;
    if (!voxel_key(pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2], voxel, key)) return;
    const int s = table_slot(keys, mask, key);
    if (s < 0)
        atomicExch(err, 1);
    else
        atomicMin(vals + s, -1);
}

// Back-projection of pixel (i, j) at depth D to the world:
// x = R^T ((i - cx) / fx D - t_x, (j - cy) / fy D - t_y, D - t_z).
__global__ void __launch_bounds__(kAThreads) k_hash_pixels(DevView cam, const float *__restrict__ depth,
                                                           const uint8_t *__restrict__ motion, AParams ap,
                                                           unsigned long long *keys, int *vals, uint32_t mask,
                                                           int *__restrict__ slot_of, int *err) {
    const int P = cam.W * cam.H;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    int s = -1;
    const float D = depth[p];
    if (D > ap.near_z && !(motion && motion[p])) {
        const int j = p / cam.W, i = p - j * cam.W;
        const float d0 = __fsub_rn(__fmul_rn(__fdiv_rn(__fsub_rn((float)i, cam.cx), cam.fx), D), cam.t[0]);
        const float d1 = __fsub_rn(__fmul_rn(__fdiv_rn(__fsub_rn((float)j, cam.cy), cam.fy), D), cam.t[1]);
        const float d2 = __fsub_rn(D, cam.t[2]);
        const float x = dot3_rn(cam.R[0], cam.R[3], cam.R[6], d0, d1, d2);
        const float y = dot3_rn(cam.R[1], cam.R[4], cam.R[7], d0, d1, d2);
        const float z = dot3_rn(cam.R[2], cam.R[5], cam.R[8], d0, d1, d2);
        unsigned long long key;
        if (voxel_key(x, y, z, ap.voxel, key)) {
            s = table_slot(keys, mask, key);
            if (s < 0)
                atomicExch(err, 1);
            else
                atomicMin(vals + s, p);
        }
    }
    slot_of[p] = s;
}

__global__ void __launch_bounds__(kAThreads) k_first(int P, const int *__restrict__ slot_of,
                                                     const int *__restrict__ vals, uint32_t *__restrict__ flags) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int s = slot_of[p];
    flags[p] = (s >= 0 && vals[s] == p) ? 1u : 0u;
}

struct InsertArgs {
    float *pos, *feat, *offsets, *scaling, *logodds;
    int *src_index;
    int F, K3;
};
__global__ void __launch_bounds__(kAThreads) k_insert(int P, const uint32_t *__restrict__ flags,
                                                      const uint64_t *__restrict__ off2,
                                                      const uint64_t *__restrict__ n_kept, long long capacity,
                                                      const int *__restrict__ slot_of,
                                                      const unsigned long long *__restrict__ keys, AParams ap,
                                                      InsertArgs o) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !flags[p]) return;
    const unsigned long long r = *n_kept + off2[p];
    if (r >= (unsigned long long)capacity) return;
    const unsigned long long key = keys[slot_of[p]];
    const int q[3] = {(int)(key >> 42) - kVoxRange, (int)((key >> 21) & 0x1fffff) - kVoxRange,
                      (int)(key & 0x1fffff) - kVoxRange};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o.pos[3 * r + a] = __fmul_rn(__fadd_rn((float)q[a], 0.5f), ap.voxel);
        o.scaling[3 * r + a] = ap.voxel;
    }
    for (int c = 0; c < o.F; ++c) o.feat[r * o.F + c] = 0.f;
    for (int c = 0; c < o.K3; ++c) o.offsets[r * o.K3 + c] = 0.f;
    o.logodds[r] = ap.l_new;
    if (o.src_index) o.src_index[r] = -1 - p;
}

__global__ void k_summary(const uint64_t *n_kept, const uint64_t *n_new, const unsigned int *counts,
                          uint64_t *out) {
    if (threadIdx.x == 0) {
        out[0] = *n_kept;
        out[1] = *n_new;
        out[2] = counts[0];
        out[3] = counts[1];
        out[4] = counts[2];
    }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

uint32_t table_size(size_t n, size_t P) {
    uint32_t s = 1024;
    while (s < 2 * (n + P)) s <<= 1;
    return s;
}

struct Layout {
    size_t lnew, keep, off, scan, keys, vals, slot, flags, off2, counts, summary, total;
    uint32_t S;
};

Layout layout(size_t n, size_t P) {
    Layout L{};
    L.S = table_size(n, P);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.lnew = take(n * sizeof(float));
    L.keep = take(n * sizeof(uint32_t));
    L.off = take((n + 1) * sizeof(uint64_t));
    L.scan = take(scan_scratch_bytes(std::max(n, P)));
    L.keys = take((size_t)L.S * sizeof(unsigned long long));
    L.vals = take((size_t)L.S * sizeof(int));
    L.slot = take(P * sizeof(int));
    L.flags = take(P * sizeof(uint32_t));
    L.off2 = take((P + 1) * sizeof(uint64_t));
    L.counts = take(3 * sizeof(unsigned int));
    L.summary = take(5 * sizeof(uint64_t));
    L.total = o;
    return L;
}

}  // namespace

size_t anchor_scratch_bytes(size_t n, size_t P) { return layout(n, P).total; }

// One keyframe (cam: its view, depth / motion: its H x W pixels) on n input
// anchors; writes the output arrays and points *summary_dev at a device
// uint64[5] in the scratch: n_kept, the number of new voxels, hits, misses and
// 1 if the voxel table overflowed (else 0).  F: anchor feature width, K3: 3 k.
cudaError_t anchor_update(const DevView &cam, const float *depth, const uint8_t *motion, int n, const float *pos,
                          const float *feat, const float *offsets, const float *scaling, const float *lin, int F,
                          int K3, float l_prior, float l_hit, float l_miss, float l_min, float l_max, float l_prune,
                          float voxel, float margin, float near_z, long long capacity, float *opos, float *ofeat,
                          float *ooffsets, float *oscaling, float *olog, int *src_index, void *scratch,
                          uint64_t **summary_dev, int num_sms, cudaStream_t st, int *launches) {
    const size_t P = (size_t)cam.W * cam.H;
    const Layout L = layout((size_t)n, P);
    char *base = static_cast<char *>(scratch);
    float *lnew = reinterpret_cast<float *>(base + L.lnew);
    uint32_t *keep = reinterpret_cast<uint32_t *>(base + L.keep);
    uint64_t *off = reinterpret_cast<uint64_t *>(base + L.off);
    void *scan = base + L.scan;
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(base + L.keys);
    int *vals = reinterpret_cast<int *>(base + L.vals);
    int *slot_of = reinterpret_cast<int *>(base + L.slot);
    uint32_t *flags = reinterpret_cast<uint32_t *>(base + L.flags);
    uint64_t *off2 = reinterpret_cast<uint64_t *>(base + L.off2);
    unsigned int *counts = reinterpret_cast<unsigned int *>(base + L.counts);  // hits, misses, table overflow
    int *err = reinterpret_cast<int *>(counts + 2);
    uint64_t *summary = reinterpret_cast<uint64_t *>(base + L.summary);
    *summary_dev = summary;

    AParams ap;
    ap.dh = l_hit - l_prior;
    ap.dm = l_miss - l_prior;
    ap.l_min = l_min;
    ap.l_max = l_max;
    ap.l_prune = l_prune;
    ap.l_new = std::fmin(std::fmax(l_prior + ap.dh, l_min), l_max);
    ap.voxel = voxel;
    ap.margin = margin;
    ap.near_z = near_z;

    cudaError_t e;
    if ((e = cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(keys, 0xff, (size_t)L.S * sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(vals, 0x7f, (size_t)L.S * sizeof(int), st)) != cudaSuccess) return e;
    static_assert(kNoOwner == 0x7f7f7f7f, "memset byte of the owner table");
    const uint32_t mask = L.S - 1;
    const int nb = (n + kAThreads - 1) / kAThreads;
    const int pb = (int)((P + kAThreads - 1) / kAThreads);
    if (n > 0) {
        k_observe<<<nb, kAThreads, 0, st>>>(n, pos, lin, cam, depth, motion, ap, lnew, keep, counts);
        ++*launches;
    }
    if ((e = exclusive_scan_u32_u64(keep, off, (size_t)n, scan, st)) != cudaSuccess) return e;
    if (n > 0) {
        *launches += 3;
        CompactArgs ca{{pos, feat, offsets, scaling, lnew}, {opos, ofeat, ooffsets, oscaling, olog}, {3, F, K3, 3, 1},
                       src_index};
        const int widest = std::max(std::max(F, K3), 3);
        const int gx = (int)std::min<size_t>(((size_t)n * widest + kAThreads - 1) / kAThreads, (size_t)num_sms * 8);
        k_compact<<<dim3(std::max(gx, 1), 6), kAThreads, 0, st>>>(n, keep, off, ca);
        k_hash_anchors<<<nb, kAThreads, 0, st>>>(n, pos, keep, voxel, keys, vals, mask, err);
        *launches += 2;
    }
    if (P > 0) {
        k_hash_pixels<<<pb, kAThreads, 0, st>>>(cam, depth, motion, ap, keys, vals, mask, slot_of, err);
        k_first<<<pb, kAThreads, 0, st>>>((int)P, slot_of, vals, flags);
        *launches += 2;
    }
    if ((e = exclusive_scan_u32_u64(flags, off2, P, scan, st)) != cudaSuccess) return e;
    if (P > 0) {
        *launches += 3;
        InsertArgs ia{opos, ofeat, ooffsets, oscaling, olog, src_index, F, K3};
        k_insert<<<pb, kAThreads, 0, st>>>((int)P, flags, off2, off + n, capacity, slot_of, keys, ap, ia);
        ++*launches;
    }
    k_summary<<<1, 32, 0, st>>>(off + n, off2 + P, counts, summary);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace ups
