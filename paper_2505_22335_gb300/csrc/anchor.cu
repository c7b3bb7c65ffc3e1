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
// Five launches for n anchors and P keyframe pixels, with no separate scan:
// each producer writes per-block counts and each consumer block sums the
// counts of the blocks before it to find its output offset.
//   k_observe      anchor -> pixel -> hit / miss / none, posterior; per block
//                  of 256 anchors the number kept, hits and misses
//   k_compact      kept rows into the output arrays in input order (one block
//                  per row block and array), their voxels into an
//                  open-addressing table (held by an anchor)
//   k_hash_pixels  the voxel of every static pixel into the table; the voxel's
//                  owner becomes its lowest pixel index (atomicMin)
//   k_count_new    per block of 256 pixels, the new voxels they own; totals
//   k_insert       a new anchor at the centre of each new voxel, in the raster
//                  order of the owners, while rows remain below capacity
#include <algorithm>

#include "common.cuh"

namespace ups {

namespace {

constexpr int kAThreads = 256;
constexpr int kVoxRange = 1 << 20;                  // voxel indices in [-2^20, 2^20)
constexpr unsigned long long kEmptyKey = ~0ull;      // table slot without a key
constexpr int kNoOwner = 0x7f7f7f7f;                 // memset byte 0x7f: above every pixel index
constexpr int kCopyUnroll = 4;                       // row-copy loads in flight per thread (k_compact)
constexpr int kPixPerThread = 1;                     // consecutive pixels per thread (k_count_new, k_insert)
constexpr int kPixBlock = kAThreads * kPixPerThread;

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

// ---------------------------------------------------------------------------
// block-wide helpers (kAThreads = 8 warps)
// ---------------------------------------------------------------------------

// Sum of v over the block, returned to every thread.
__device__ __forceinline__ int block_sum(int v, int *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = 0;
#pragma unroll
    for (int w = 0; w < kAThreads / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Exclusive prefix of v over the threads of the block; *total gets the sum.
__device__ __forceinline__ int block_excl_scan(int v, int *red, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) red[w] = x;
    __syncthreads();
    int off = 0, t = 0;
#pragma unroll
    for (int k = 0; k < kAThreads / 32; ++k) {
        off += k < w ? red[k] : 0;
        t += red[k];
    }
    __syncthreads();
    *total = t;
    return off + x - v;
}

// Sum of cnt[0 .. b): the output offset of block b.  Every block reads the
// counts of the blocks before it (a few hundred to a few thousand ints for
// keyframe-sized inputs), which costs less than separate scan launches.
__device__ __forceinline__ int block_prefix(const int *__restrict__ cnt, int b, int *red) {
    int acc = 0;
    for (int j = threadIdx.x; j < b; j += kAThreads) acc += cnt[j];
    return block_sum(acc, red);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Observation of each anchor (0 none, 1 hit, 2 miss) and its posterior; per
// block of kAThreads anchors, the number kept and the hits and misses.
__global__ void __launch_bounds__(kAThreads) k_observe(int n, const float *__restrict__ pos,
                                                       const float *__restrict__ lin, DevView cam,
                                                       const float *__restrict__ depth,
                                                       const uint8_t *__restrict__ motion, AParams ap,
                                                       float *__restrict__ lnew, int *__restrict__ bkept,
                                                       int *__restrict__ bhit, int *__restrict__ bmiss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int obs = 0, kept = 0;
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
        kept = l >= ap.l_prune;
    }
    const int k = __syncthreads_count(kept), h = __syncthreads_count(obs == 1), m = __syncthreads_count(obs == 2);
    if (threadIdx.x == 0) {
        bkept[blockIdx.x] = k;
        bhit[blockIdx.x] = h;
        bmiss[blockIdx.x] = m;
    }
}

// Kept rows (the same kAThreads-row blocks as k_observe) to their output rows in
// input order: blockIdx.y picks the array (pos, feat, offsets, scaling,
// log-odds), so five blocks share a row block and every block recomputes the
// rows' output offsets (a prefix over the block counts and a block scan); the
// pos blocks also write the source index and insert the voxels into the table.
struct RowArrays {
    const float *src[5];  // pos, feat, offsets, scaling, posterior log-odds
    float *dst[5];
    int width[5];
    int *src_index;
};
__global__ void __launch_bounds__(kAThreads) k_compact(int n, const float *__restrict__ lnew,
                                                       const int *__restrict__ bkept, float l_prune, RowArrays a,
                                                       float voxel, unsigned long long *keys, int *vals,
                                                       uint32_t mask, int *err) {
    __shared__ int red[kAThreads / 32];
    __shared__ int s_row[kAThreads];
    const int r0 = blockIdx.x * kAThreads, i = r0 + threadIdx.x;
    const int base = block_prefix(bkept, blockIdx.x, red);
    const int flag = (i < n && lnew[i] >= l_prune) ? 1 : 0;
    int total;
    const int row = base + block_excl_scan(flag, red, &total);
    s_row[threadIdx.x] = flag ? row : -1;
    // a switch, not a.src[blockIdx.y]: indexing the parameter arrays would copy them to the stack
    int w;
    const float *sp;
    float *dp;
    switch (blockIdx.y) {
        case 0: w = a.width[0], sp = a.src[0], dp = a.dst[0]; break;
        case 1: w = a.width[1], sp = a.src[1], dp = a.dst[1]; break;
        case 2: w = a.width[2], sp = a.src[2], dp = a.dst[2]; break;
        case 3: w = a.width[3], sp = a.src[3], dp = a.dst[3]; break;
        default: w = a.width[4], sp = a.src[4], dp = a.dst[4]; break;
    }
    if (blockIdx.y == 0 && flag) {
        if (a.src_index) a.src_index[row] = i;
        const float *x = sp + 3 * (size_t)i;
        unsigned long long key;
        if (voxel_key(x[0], x[1], x[2], voxel, key)) {
            const int s = table_slot(keys, mask, key);
            if (s < 0)
                atomicExch(err, 1);
            else
                atomicMin(vals + s, -1);  // held by an anchor
        }
    }
    __syncthreads();
    // the block's rows are one contiguous run: coalesced reads, kCopyUnroll loads
    // in flight per thread before the (mostly contiguous) stores
    const int nrows = min(kAThreads, n - r0), tot = nrows * w;
    const float *__restrict__ src = sp + (size_t)r0 * w;
    float *__restrict__ dst = dp;
    for (int e0 = threadIdx.x; e0 < tot; e0 += kCopyUnroll * kAThreads) {
        float v[kCopyUnroll];
#pragma unroll
        for (int k = 0; k < kCopyUnroll; ++k) {
            const int e = e0 + k * kAThreads;
            v[k] = e < tot ? src[e] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kCopyUnroll; ++k) {
            const int e = e0 + k * kAThreads;
            if (e >= tot) break;
            const int rl = e / w, r = s_row[rl];
            if (r >= 0) dst[(size_t)r * w + (e - rl * w)] = v[k];
        }
    }
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
                atomicMin(vals + s, p);  // the voxel's owner: its first pixel in raster order
        }
    }
    slot_of[p] = s;
}

// pixel p is the owner of a voxel that no kept anchor holds
__device__ __forceinline__ int owns_new(int P, int p, const int *__restrict__ slot_of, const int *__restrict__ vals) {
    if (p >= P) return 0;
    const int s = slot_of[p];
    return (s >= 0 && vals[s] == p) ? 1 : 0;
}

// Per block of kPixBlock pixels, the number of new voxels it owns; block 0
// also totals the anchor counts (n_kept, hits, misses) into the summary.
__global__ void __launch_bounds__(kAThreads) k_count_new(int P, const int *__restrict__ slot_of,
                                                         const int *__restrict__ vals, int *__restrict__ pnew,
                                                         int nb, const int *__restrict__ bkept,
                                                         const int *__restrict__ bhit, const int *__restrict__ bmiss,
                                                         uint64_t *__restrict__ summary) {
    __shared__ int red[kAThreads / 32];
    const int p0 = blockIdx.x * kPixBlock + kPixPerThread * threadIdx.x;
    int c = 0;
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) c += owns_new(P, p0 + k, slot_of, vals);
    c = block_sum(c, red);
    if (threadIdx.x == 0) pnew[blockIdx.x] = c;
    if (blockIdx.x == 0) {
        int kk = 0, hh = 0, mm = 0;
        for (int j = threadIdx.x; j < nb; j += kAThreads) {
            kk += bkept[j];
            hh += bhit[j];
            mm += bmiss[j];
        }
        kk = block_sum(kk, red);
        hh = block_sum(hh, red);
        mm = block_sum(mm, red);
        if (threadIdx.x == 0) {
            summary[0] = (uint64_t)kk;
            summary[2] = (uint64_t)hh;
            summary[3] = (uint64_t)mm;
        }
    }
}

struct InsertArgs {
    float *pos, *feat, *offsets, *scaling, *logodds;
    int *src_index;
    int F, K3;
};
// A new anchor at the centre of every new voxel, at row n_kept + (its rank in
// the raster order of the owning pixels), while rows remain below capacity.
// The last block writes the number of new voxels and the table-overflow flag.
__global__ void __launch_bounds__(kAThreads) k_insert(int P, const int *__restrict__ slot_of,
                                                      const int *__restrict__ vals, const int *__restrict__ pnew,
                                                      const unsigned long long *__restrict__ keys, AParams ap,
                                                      long long capacity, InsertArgs o, uint64_t *summary,
                                                      const int *err) {
    __shared__ int red[kAThreads / 32];
    const int p0 = blockIdx.x * kPixBlock + kPixPerThread * threadIdx.x;
    const int base = block_prefix(pnew, blockIdx.x, red);
    int f[kPixPerThread], c = 0;
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) c += (f[k] = owns_new(P, p0 + k, slot_of, vals));
    int total;
    int rank = base + block_excl_scan(c, red, &total);
    const long long n_kept = (long long)summary[0];
#pragma unroll
    for (int k = 0; k < kPixPerThread; ++k) {
        if (!f[k]) continue;
        const long long r = n_kept + rank++;
        if (r >= capacity) continue;
        const int p = p0 + k;
        const unsigned long long key = keys[slot_of[p]];
        const int q[3] = {(int)(key >> 42) - kVoxRange, (int)((key >> 21) & 0x1fffff) - kVoxRange,
                          (int)(key & 0x1fffff) - kVoxRange};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o.pos[3 * r + a] = __fmul_rn(__fadd_rn((float)q[a], 0.5f), ap.voxel);
            o.scaling[3 * r + a] = ap.voxel;
        }
        for (int cc = 0; cc < o.F; ++cc) o.feat[r * o.F + cc] = 0.f;
        for (int cc = 0; cc < o.K3; ++cc) o.offsets[r * o.K3 + cc] = 0.f;
        o.logodds[r] = ap.l_new;
        if (o.src_index) o.src_index[r] = -1 - p;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        summary[1] = (uint64_t)(base + total);
        summary[4] = (uint64_t)*err;
    }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

uint32_t table_size(size_t n, size_t P) {
    uint32_t s = 1024;
    while (s < 2 * (n + P)) s <<= 1;
    return s;
}

struct Layout {
    size_t lnew, bkept, bhit, bmiss, keys, vals, slot, pnew, summary, err, total;
    uint32_t S;
};

Layout layout(size_t n, size_t P) {
    Layout L{};
    L.S = table_size(n, P);
    const size_t nb = (n + kAThreads - 1) / kAThreads, npb = (P + kPixBlock - 1) / kPixBlock;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    L.lnew = take(n * sizeof(float));
    L.bkept = take(nb * sizeof(int));
    L.bhit = take(nb * sizeof(int));
    L.bmiss = take(nb * sizeof(int));
    L.keys = take((size_t)L.S * sizeof(unsigned long long));
    L.vals = take((size_t)L.S * sizeof(int));
    L.slot = take(P * sizeof(int));
    L.pnew = take(npb * sizeof(int));
    L.summary = take(5 * sizeof(uint64_t));
    L.err = take(sizeof(int));
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
                          uint64_t **summary_dev, cudaStream_t st, int *launches) {
    const size_t P = (size_t)cam.W * cam.H;
    const Layout L = layout((size_t)n, P);
    char *base = static_cast<char *>(scratch);
    float *lnew = reinterpret_cast<float *>(base + L.lnew);
    int *bkept = reinterpret_cast<int *>(base + L.bkept);
    int *bhit = reinterpret_cast<int *>(base + L.bhit);
    int *bmiss = reinterpret_cast<int *>(base + L.bmiss);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(base + L.keys);
    int *vals = reinterpret_cast<int *>(base + L.vals);
    int *slot_of = reinterpret_cast<int *>(base + L.slot);
    int *pnew = reinterpret_cast<int *>(base + L.pnew);
    uint64_t *summary = reinterpret_cast<uint64_t *>(base + L.summary);
    int *err = reinterpret_cast<int *>(base + L.err);
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
    if ((e = cudaMemsetAsync(err, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(keys, 0xff, (size_t)L.S * sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(vals, 0x7f, (size_t)L.S * sizeof(int), st)) != cudaSuccess) return e;
    static_assert(kNoOwner == 0x7f7f7f7f, "memset byte of the owner table");
    const uint32_t mask = L.S - 1;
    const int nb = (n + kAThreads - 1) / kAThreads;
    const int pb = (int)((P + kAThreads - 1) / kAThreads);
    const int npb = (int)((P + kPixBlock - 1) / kPixBlock);
    if (n > 0) {
        k_observe<<<nb, kAThreads, 0, st>>>(n, pos, lin, cam, depth, motion, ap, lnew, bkept, bhit, bmiss);
        RowArrays ra{{pos, feat, offsets, scaling, lnew}, {opos, ofeat, ooffsets, oscaling, olog}, {3, F, K3, 3, 1},
                     src_index};
        k_compact<<<dim3(nb, 5), kAThreads, 0, st>>>(n, lnew, bkept, l_prune, ra, voxel, keys, vals, mask, err);
        *launches += 2;
    }
    k_hash_pixels<<<pb, kAThreads, 0, st>>>(cam, depth, motion, ap, keys, vals, mask, slot_of, err);
    k_count_new<<<npb, kAThreads, 0, st>>>((int)P, slot_of, vals, pnew, nb, bkept, bhit, bmiss, summary);
    InsertArgs ia{opos, ofeat, ooffsets, oscaling, olog, src_index, F, K3};
    k_insert<<<npb, kAThreads, 0, st>>>((int)P, slot_of, vals, pnew, keys, ap, capacity, ia, summary, err);
    *launches += 3;
    return cudaGetLastError();
}

}  // namespace ups
