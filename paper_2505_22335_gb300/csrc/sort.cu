// Stable LSD radix sort of (key, value) pairs and exclusive scans, written for
// this library (no CUB).  Used twice per forward: once to order Gaussian-views
// by (view, depth) and once to bucket the depth-ordered tile instances by
// (view, tile), which together give the (view, tile, depth, id) order.
//
// One pass = histogram kernel (per-block digit counts, digit-major layout) +
// exclusive scan of the counts + scatter kernel (stable block-local ranking by
// ballots, then a scatter to the scanned offsets).
#include <algorithm>

#include "common.cuh"

namespace ups {

namespace {

constexpr int kThreads = 256;
constexpr int kBins = 256;  // 8-bit digits
constexpr int kWarps = kThreads / 32;

// Items per thread: 8 keeps the scatter kernel near 50 registers (five
// 256-thread blocks per SM hide the latency of its ranking loop) and the
// block tile staged in shared memory under 48 KB.
template <class K> struct Radix {
    static constexpr int items = 8;
    static constexpr int tile = kThreads * items;
};

// 256-wide exclusive scan across the block (one value per thread).
__device__ __forceinline__ uint32_t scan256(uint32_t x, uint32_t *warp_tot) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    uint32_t before = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) before += ww < w ? warp_tot[ww] : 0u;
    return before + incl - x;
}

template <class K>
__global__ void __launch_bounds__(kThreads) k_radix_hist(const K *__restrict__ keys, size_t n,
                                                         int shift, uint32_t *__restrict__ hist,
                                                         int nblocks) {
    constexpr int TILE = Radix<K>::tile;
    __shared__ uint32_t h[kWarps][kBins];
    const int tid = threadIdx.x, w = tid >> 5;
    for (int i = tid; i < kWarps * kBins; i += kThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const size_t base = (size_t)blockIdx.x * TILE;
#pragma unroll 4
    for (int i = tid; i < TILE; i += kThreads) {
        size_t idx = base + i;
        if (idx < n) {
            uint32_t d = (uint32_t)(keys[idx] >> shift) & (kBins - 1);
            atomicAdd(&h[w][d], 1u);
        }
    }
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) s += h[ww][tid];
    hist[(size_t)tid * nblocks + blockIdx.x] = s;
}

// Stable scatter of one block tile: ballot-based ranking inside each warp,
// then the tile is reordered by digit in shared memory and written out in
// order, so consecutive threads store consecutive addresses of a bucket.
template <class K>
__global__ void __launch_bounds__(kThreads) k_radix_scatter(
    const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
    uint32_t *__restrict__ vout, size_t n, int shift, const uint32_t *__restrict__ offs,
    int nblocks) {
    constexpr int ITEMS = Radix<K>::items, TILE = Radix<K>::tile;
    __shared__ uint32_t wcnt[kWarps][kBins];
    __shared__ uint32_t dstart[kBins];
    __shared__ uint32_t gbase[kBins];
    __shared__ uint32_t wtot[kWarps];
    __shared__ K skey[TILE];
    __shared__ uint32_t sval[TILE];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kWarps * kBins; i += kThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    const size_t tile_base = (size_t)blockIdx.x * TILE;
    const size_t base = tile_base + (size_t)w * (32 * ITEMS);
    K key[ITEMS];
    uint32_t val[ITEMS];
    uint32_t rank[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        size_t idx = base + (size_t)j * 32 + lane;
        bool valid = idx < n;
        uint32_t d = kBins;  // sentinel for out-of-range lanes
        if (valid) {
            key[j] = kin[idx];
            val[j] = vin[idx];
            d = (uint32_t)(key[j] >> shift) & (kBins - 1);
        }
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            uint32_t bit = (d >> b) & 1u;
            uint32_t bb = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bb : ~bb;
        }
        uint32_t lt = __popc(peers & lt_mask);
        uint32_t prior = valid ? wcnt[w][d] : 0u;
        __syncwarp();
        if (valid && lt == 0) wcnt[w][d] = prior + __popc(peers);
        __syncwarp();
        rank[j] = prior + lt;
    }
    __syncthreads();
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
        uint32_t c = wcnt[ww][tid];
        wcnt[ww][tid] = run;
        run += c;
    }
    dstart[tid] = scan256(run, wtot);
    gbase[tid] = offs[(size_t)tid * nblocks + blockIdx.x];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        size_t idx = base + (size_t)j * 32 + lane;
        if (idx < n) {
            uint32_t d = (uint32_t)(key[j] >> shift) & (kBins - 1);
            uint32_t lpos = dstart[d] + wcnt[w][d] + rank[j];
            skey[lpos] = key[j];
            sval[lpos] = val[j];
        }
    }
    __syncthreads();
    const int nvalid = (int)min((size_t)TILE, n - tile_base);
    for (int i = tid; i < nvalid; i += kThreads) {
        K k = skey[i];
        uint32_t d = (uint32_t)(k >> shift) & (kBins - 1);
        uint32_t pos = gbase[d] + (uint32_t)i - dstart[d];
        kout[pos] = k;
        vout[pos] = sval[i];
    }
}

// ---------------------------------------------------------------------------
// exclusive scan (3 kernels: block sums, scan of block sums, apply)
// ---------------------------------------------------------------------------

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ T block_exclusive_scan(T x, T *total) {
    __shared__ T warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        T s = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
        T si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = si - s;
        if (lane == kScanThreads / 32 - 1) *total = si;
    }
    __syncthreads();
    T r = warp_sums[w] + incl - x;
    __syncthreads();
    return r;
}

// gate (all scan, histogram, range and scatter kernels): when non-null, the
// kernel does nothing unless *gate != 0 (work enqueued ahead of a decision
// the GPU takes)
template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in,
                                                              size_t n, T *__restrict__ partial,
                                                              const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ T tot;
    const size_t base = (size_t)blockIdx.x * kScanTile;
    T s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        size_t idx = base + i;
        if (idx < n) s += in[idx];
    }
    block_exclusive_scan<T>(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(T *partial, int nb, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ T tot;
    T carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
        int i = b0 + threadIdx.x;
        T x = i < nb ? partial[i] : T(0);
        T ex = block_exclusive_scan<T>(x, &tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t *in, T *out, size_t n,
                                                             const T *__restrict__ partial,
                                                             int write_total, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ uint32_t tile[kScanTile];
    __shared__ T tot;
    const size_t base = (size_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        size_t idx = base + i;
        tile[i] = idx < n ? in[idx] : 0u;
    }
    __syncthreads();
    T loc[kScanItems];
    T s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        loc[j] = s;
        s += tile[threadIdx.x * kScanItems + j];
    }
    T ex = block_exclusive_scan<T>(s, &tot) + partial[blockIdx.x];
    __syncthreads();
    // write back through shared memory for coalesced stores
    T *otile = reinterpret_cast<T *>(tile);  // reuse only when T fits
    if (sizeof(T) == sizeof(uint32_t)) {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) otile[threadIdx.x * kScanItems + j] = ex + loc[j];
        __syncthreads();
        for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
            size_t idx = base + i;
            if (idx < n) out[idx] = otile[i];
        }
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            size_t idx = base + threadIdx.x * kScanItems + j;
            if (idx < n) out[idx] = ex + loc[j];
        }
    }
    if (write_total && base <= n - 1 && n - 1 < base + kScanTile) {
        if (threadIdx.x == (int)((n - 1 - base) / kScanItems)) {
            int j = (int)((n - 1 - base) % kScanItems);
            // total = exclusive prefix of the last element + its value
            out[n] = ex + loc[j] + (T)in[n - 1];
        }
    }
}

template <class T>
cudaError_t scan_impl(const uint32_t *in, T *out, size_t n, void *scratch, int write_total,
                      cudaStream_t st, const int *gate = nullptr) {
    if (n == 0) {
        if (write_total) return cudaMemsetAsync(out, 0, sizeof(T), st);
        return cudaSuccess;
    }
    int nb = (int)((n + kScanTile - 1) / kScanTile);
    T *partial = static_cast<T *>(scratch);
    k_scan_reduce<T><<<nb, kScanThreads, 0, st>>>(in, n, partial, gate);
    k_scan_partials<T><<<1, kScanThreads, 0, st>>>(partial, nb, gate);
    k_scan_apply<T><<<nb, kScanThreads, 0, st>>>(in, out, n, partial, write_total, gate);
    return cudaGetLastError();
}

template <class K>
cudaError_t radix_impl(K **key_io, K **key_alt, uint32_t **val_io, uint32_t **val_alt, size_t n,
                       int end_bit, SortScratch &s, cudaStream_t st) {
    if (n <= 1 || end_bit <= 0) return cudaSuccess;
    int nblocks = (int)((n + Radix<K>::tile - 1) / Radix<K>::tile);
    size_t hist_n = (size_t)kBins * nblocks;
    size_t need = hist_n * sizeof(uint32_t) + scan_scratch_bytes(hist_n);
    cudaError_t e = s.hist.reserve(need);
    if (e != cudaSuccess) return e;
    uint32_t *hist = s.hist.as<uint32_t>();
    void *scr = reinterpret_cast<char *>(s.hist.ptr) + ((hist_n * sizeof(uint32_t) + 255) & ~size_t(255));
    for (int shift = 0; shift < end_bit; shift += 8) {
        k_radix_hist<K><<<nblocks, kThreads, 0, st>>>(*key_io, n, shift, hist, nblocks);
        e = scan_impl<uint32_t>(hist, hist, hist_n, scr, 0, st);
        if (e != cudaSuccess) return e;
        k_radix_scatter<K><<<nblocks, kThreads, 0, st>>>(*key_io, *val_io, *key_alt, *val_alt, n,
                                                         shift, hist, nblocks);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        K *tk = *key_io;
        *key_io = *key_alt;
        *key_alt = tk;
        uint32_t *tv = *val_io;
        *val_io = *val_alt;
        *val_alt = tv;
    }
    return cudaSuccess;
}

// Same passes as radix_impl, with the histogram and scan scratch supplied by
// the caller instead of a growable buffer.
template <class K>
cudaError_t radix_fixed(K **key_io, K **key_alt, uint32_t **val_io, uint32_t **val_alt, size_t n,
                        int end_bit, void *scratch, size_t scratch_bytes, cudaStream_t st) {
    if (n <= 1 || end_bit <= 0) return cudaSuccess;
    int nblocks = (int)((n + Radix<K>::tile - 1) / Radix<K>::tile);
    size_t hist_n = (size_t)kBins * nblocks;
    size_t hist_bytes = (hist_n * sizeof(uint32_t) + 255) & ~size_t(255);
    if (hist_bytes + scan_scratch_bytes(hist_n) > scratch_bytes) return cudaErrorInvalidValue;
    uint32_t *hist = static_cast<uint32_t *>(scratch);
    void *scr = static_cast<char *>(scratch) + hist_bytes;
    for (int shift = 0; shift < end_bit; shift += 8) {
        k_radix_hist<K><<<nblocks, kThreads, 0, st>>>(*key_io, n, shift, hist, nblocks);
        cudaError_t e = scan_impl<uint32_t>(hist, hist, hist_n, scr, 0, st);
        if (e != cudaSuccess) return e;
        k_radix_scatter<K><<<nblocks, kThreads, 0, st>>>(*key_io, *val_io, *key_alt, *val_alt, n,
                                                         shift, hist, nblocks);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        K *tk = *key_io;
        *key_io = *key_alt;
        *key_alt = tk;
        uint32_t *tv = *val_io;
        *val_io = *val_alt;
        *val_alt = tv;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// one-pass stable bucket sort by small keys (tile ids)
// ---------------------------------------------------------------------------
//
// Keys are < nbins <= 2^14.  The input is split into nblocks contiguous runs
// of per_block items (a multiple of the 2048-item sub-tile).  (1) each block
// counts its keys per bucket; (2) an exclusive scan of the counts in
// (bucket, block) order gives every (bucket, block) pair its first output
// slot and every bucket its [start, end) range; (3) each block walks its run
// in sub-tiles: a stable two-pass (7 + 7 bit) sort of the sub-tile in shared
// memory groups equal keys, and item i of a group goes to next[bucket] +
// (i - group start), after which next[bucket] moves past the group.  Only
// the values are written: the sorted keys follow from the ranges.

constexpr int kBkThreads = 256;
constexpr int kBkWarps = kBkThreads / 32;
constexpr int kBkItems = 8;
constexpr int kBkSub = kBkThreads * kBkItems;  // items per sub-tile
constexpr int kBkDigit = 7;                    // bits per in-block pass
constexpr int kBkLocal = 1 << kBkDigit;
constexpr int kBkHistThreads = 512;
constexpr uint32_t kBkPad = kMaxBucketBins - 1;  // digit of the empty slots of a partial sub-tile
constexpr int kBkCapWaves = 4;

__host__ __device__ inline int bk_nbp(int nbins) { return (nbins + 3) & ~3; }
size_t bk_scatter_smem(int nbins) {
    return (size_t)bk_nbp(nbins) * 4 + kBkSub * (2 + 4) + (kBkWarps + 1) * kBkLocal * 4 + 64;
}

__global__ void __launch_bounds__(kBkHistThreads) k_bucket_hist(const uint32_t *__restrict__ keys, size_t n,
                                                                int nbins, size_t per_block,
                                                                uint32_t *__restrict__ hist, int nblocks,
                                                                const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    extern __shared__ uint32_t h[];
    for (int d = threadIdx.x; d < nbins; d += kBkHistThreads) h[d] = 0;
    __syncthreads();
    const size_t beg = (size_t)blockIdx.x * per_block;
    const size_t end = min(n, beg + per_block);
    const uint32_t top = (uint32_t)nbins - 1;
    // beg is a multiple of 2048 items: 16-byte loads up to the last full quad
    const size_t nq = (end - beg) / 4;
    const uint4 *q4 = reinterpret_cast<const uint4 *>(keys + beg);
    for (size_t i = threadIdx.x; i < nq; i += kBkHistThreads) {
        const uint4 k = q4[i];
        atomicAdd(&h[min(k.x, top)], 1u);
        atomicAdd(&h[min(k.y, top)], 1u);
        atomicAdd(&h[min(k.z, top)], 1u);
        atomicAdd(&h[min(k.w, top)], 1u);
    }
    for (size_t i = beg + 4 * nq + threadIdx.x; i < end; i += kBkHistThreads) atomicAdd(&h[min(keys[i], top)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < nbins; d += kBkHistThreads) hist[(size_t)d * nblocks + blockIdx.x] = h[d];
}

// Bucket d keeps its first min(count_d, cap) items: one block scans the kept
// counts into ranges[d] = [start, start + kept) (ostart[d] = start) and sets
// bit d of trunc when count_d > cap.
constexpr int kBkRangeThreads = 1024;
__global__ void __launch_bounds__(kBkRangeThreads) k_bucket_ranges(const uint32_t *__restrict__ offs, int nbins,
                                                                   int nblocks, uint32_t n, uint32_t cap,
                                                                   uint2 *__restrict__ ranges,
                                                                   uint32_t *__restrict__ ostart,
                                                                   uint32_t *__restrict__ trunc,
                                                                   const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    __shared__ uint32_t wsum[kBkRangeThreads / 32];
    __shared__ uint32_t carry_s;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry_s = 0;
    for (int i = tid; i < (nbins + 31) / 32; i += kBkRangeThreads) trunc[i] = 0u;
    __syncthreads();
    for (int d0 = 0; d0 < nbins; d0 += kBkRangeThreads) {
        const int d = d0 + tid;
        uint32_t cnt = 0, kept = 0;
        if (d < nbins) {
            const uint32_t s = offs[(size_t)d * nblocks];
            const uint32_t e = d + 1 < nbins ? offs[(size_t)(d + 1) * nblocks] : n;
            cnt = e - s;
            kept = min(cnt, cap);
        }
        uint32_t incl = kept;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            const uint32_t x = wsum[lane];
            uint32_t wi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            wsum[lane] = wi - x;
        }
        __syncthreads();
        const uint32_t carry = carry_s;
        if (d < nbins) {
            const uint32_t st = carry + wsum[w] + incl - kept;
            ranges[d] = make_uint2(st, st + kept);
            ostart[d] = st;
            if (cnt > cap) atomicOr(trunc + (d >> 5), 1u << (d & 31));
        }
        __syncthreads();
        if (tid == kBkRangeThreads - 1) carry_s = carry + wsum[w] + incl;
        __syncthreads();
    }
}

// One stable counting pass over the 7-bit digit (d >> shift) & 127 of the
// sub-tile's items, held in registers in sub-tile order (item w*256 + j*32 +
// lane); writes them to (od, ov) in digit order.  (od, ov) may be the buffer
// the items were read from: the block syncs before the first write.  Ends
// with the block synced.
__device__ __forceinline__ void bk_local_pass(const uint32_t (&d)[kBkItems], const uint32_t (&v)[kBkItems],
                                              int shift, uint16_t *od, uint32_t *ov, uint32_t *wc,
                                              uint32_t *dstart) {
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t *mine = wc + w * kBkLocal;
#pragma unroll
    for (int b = lane; b < kBkLocal; b += 32) mine[b] = 0u;
    __syncwarp();
    uint32_t rank[kBkItems];
#pragma unroll
    for (int j = 0; j < kBkItems; ++j) {
        const uint32_t b = (d[j] >> shift) & (kBkLocal - 1);
        // lanes holding the same digit, one ballot per bit (a warp match.any
        // costs several times the seven ballots on this GPU)
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int bit = 0; bit < kBkDigit; ++bit) {
            const uint32_t x = (b >> bit) & 1u;
            const uint32_t bb = __ballot_sync(0xffffffffu, x);
            peers &= x ? bb : ~bb;
        }
        const uint32_t lt = __popc(peers & lt_mask);
        const uint32_t prior = mine[b];
        __syncwarp();
        if (lt == 0) mine[b] = prior + __popc(peers);
        __syncwarp();
        rank[j] = prior + lt;
    }
    __syncthreads();
    // exclusive offsets in (digit, warp) order
    if (tid < kBkLocal) {
        uint32_t r = 0;
#pragma unroll
        for (int ww = 0; ww < kBkWarps; ++ww) {
            const uint32_t c = wc[ww * kBkLocal + tid];
            wc[ww * kBkLocal + tid] = r;
            r += c;
        }
        dstart[tid] = r;
    }
    __syncthreads();
    if (w == 0) {
        uint32_t t[kBkLocal / 32], sum = 0;
#pragma unroll
        for (int i = 0; i < kBkLocal / 32; ++i) {
            t[i] = dstart[(kBkLocal / 32) * lane + i];
            sum += t[i];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int i = 0; i < kBkLocal / 32; ++i) {
            dstart[(kBkLocal / 32) * lane + i] = run;
            run += t[i];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kBkItems; ++j) {
        const uint32_t b = (d[j] >> shift) & (kBkLocal - 1);
        const uint32_t pos = dstart[b] + wc[w * kBkLocal + b] + rank[j];
        od[pos] = (uint16_t)d[j];
        ov[pos] = v[j];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBkThreads, 3) k_bucket_scatter(const uint32_t *__restrict__ keys,
                                                                  const uint32_t *__restrict__ vals,
                                                                  uint32_t *__restrict__ vout, size_t n, int nbins,
                                                                  size_t per_block,
                                                                  const uint32_t *__restrict__ offs, int nblocks,
                                                                  const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    extern __shared__ __align__(16) unsigned char bk_smem[];
    const int nbp = bk_nbp(nbins);
    // next[b]: next output slot of bucket b; while a sub-tile is written, the
    // head of b's group rebases it to next[b] - (group start), so that item i
    // of the group goes to next[b] + i
    uint32_t *next = reinterpret_cast<uint32_t *>(bk_smem);
    uint16_t *sd = reinterpret_cast<uint16_t *>(next + nbp);    // [kBkSub] digits
    uint32_t *sv = reinterpret_cast<uint32_t *>(sd + kBkSub);    // [kBkSub] values
    uint32_t *wc = sv + kBkSub;                                 // [kBkWarps][kBkLocal]
    uint32_t *dstart = wc + kBkWarps * kBkLocal;                // [kBkLocal]
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int d = tid; d < nbins; d += kBkThreads) next[d] = offs[(size_t)d * nblocks + blockIdx.x];
    const size_t beg = (size_t)blockIdx.x * per_block;
    const size_t end = min(n, beg + per_block);
    const uint32_t top = (uint32_t)nbins - 1;
    const int slot0 = w * (32 * kBkItems) + lane;  // item j of this thread: slot0 + 32 j
    // raw loads of the next sub-tile stay in flight while this one is sorted
    uint32_t key[kBkItems], val[kBkItems];
    auto load = [&](size_t s0) {
#pragma unroll
        for (int j = 0; j < kBkItems; ++j) {
            const size_t idx = s0 + (size_t)(slot0 + j * 32);
            if (idx < end) {
                key[j] = keys[idx];
                val[j] = vals[idx];
            }
        }
    };
    if (beg < end) load(beg);
    for (size_t s0 = beg; s0 < end; s0 += kBkSub) {
        const int nvalid = (int)min((size_t)kBkSub, end - s0);
        uint32_t d[kBkItems], v[kBkItems];
#pragma unroll
        for (int j = 0; j < kBkItems; ++j) {
            // the empty slots of a partial sub-tile sort behind every key
            const bool ok = slot0 + j * 32 < nvalid;
            d[j] = ok ? min(key[j], top) : kBkPad;
            v[j] = val[j];
        }
        if (s0 + kBkSub < end) load(s0 + kBkSub);
        // low then high 7 bits: the sub-tile ends grouped by key in (sd, sv)
        bk_local_pass(d, v, 0, sd, sv, wc, dstart);
#pragma unroll
        for (int j = 0; j < kBkItems; ++j) {
            d[j] = sd[slot0 + j * 32];
            v[j] = sv[slot0 + j * 32];
        }
        bk_local_pass(d, v, kBkDigit, sd, sv, wc, dstart);
        // group heads rebase the bucket fronts, every item is written, then
        // the group tails move the fronts past their groups
#pragma unroll
        for (int k = 0; k < kBkItems; ++k) {
            const int i = tid + k * kBkThreads;
            if (i < nvalid) {
                const uint32_t dd = sd[i];
                if (i == 0 || sd[i - 1] != dd) next[dd] -= (uint32_t)i;
            }
        }
        __syncthreads();
        uint32_t front[kBkItems];
#pragma unroll
        for (int k = 0; k < kBkItems; ++k) {
            const int i = tid + k * kBkThreads;
            front[k] = 0u;
            if (i < nvalid) {
                const uint32_t dd = sd[i];
                const uint32_t base = next[dd];
                vout[base + (uint32_t)i] = sv[i];
                if (i == nvalid - 1 || sd[i + 1] != dd) front[k] = base + (uint32_t)i + 1u;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kBkItems; ++k) {
            const int i = tid + k * kBkThreads;
            if (i < nvalid && (i == nvalid - 1 || sd[i + 1] != sd[i])) next[sd[i]] = front[k];
        }
        __syncthreads();
    }
}

// Capped variant: bucket d keeps its first cap items.  A bucket whose cap is
// reached takes no more items, so each block first drops, in input order,
// every item whose bucket is already full (most items, once the nearest
// layers of the scene have filled the lists) and packs the others into a
// 2048-item buffer; full buffers are grouped by the two-pass sort and
// written.  The sort carries item indices (relative to the block's run), and
// values are read only for the items that are written.  room[d] (16 bits,
// cap <= kMaxListCap) counts the slots bucket d has left; while a buffer is
// written, the head of d's group rebases next[d] and room[d] by the group
// start, so that item i of the group goes to next[d] + i while i < room[d].
size_t bk_scatter_cap_smem(int nbins) {
    return (size_t)bk_nbp(nbins) * (4 + 2) + 2 * kBkSub * (2 + 4) + (2 * kBkWarps + 1) * kBkLocal * 4 + 64;
}

// Groups and writes the m buffered items of (sd, sv); ends with the block
// synced.
__device__ __forceinline__ void bk_cap_flush(int m, uint16_t *sd, uint32_t *sv, uint32_t *wc, uint32_t *dstart,
                                             uint32_t *next, uint16_t *room, const uint32_t *__restrict__ vals,
                                             size_t beg, uint32_t *__restrict__ vout) {
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int slot0 = w * (32 * kBkItems) + lane;
    uint32_t d[kBkItems], v[kBkItems];
#pragma unroll
    for (int j = 0; j < kBkItems; ++j) {
        const int i = slot0 + j * 32;
        d[j] = i < m ? (uint32_t)sd[i] : kBkPad;
        v[j] = i < m ? sv[i] : 0u;
    }
    bk_local_pass(d, v, 0, sd, sv, wc, dstart);
#pragma unroll
    for (int j = 0; j < kBkItems; ++j) {
        d[j] = sd[slot0 + j * 32];
        v[j] = sv[slot0 + j * 32];
    }
    bk_local_pass(d, v, kBkDigit, sd, sv, wc, dstart);
    // the m items come first (nbins < kMaxBucketBins: no tile id equals the pad)
#pragma unroll
    for (int k = 0; k < kBkItems; ++k) {
        const int i = tid + k * kBkThreads;
        if (i < m) {
            const uint32_t dd = sd[i];
            if (i == 0 || sd[i - 1] != dd) {
                next[dd] -= (uint32_t)i;
                room[dd] = (uint16_t)(room[dd] + i);
            }
        }
    }
    __syncthreads();
    uint32_t front[kBkItems];
    uint16_t left[kBkItems];
#pragma unroll
    for (int k = 0; k < kBkItems; ++k) {
        const int i = tid + k * kBkThreads;
        front[k] = 0xffffffffu;
        left[k] = 0;
        if (i < m) {
            const uint32_t dd = sd[i];
            const uint32_t lim = room[dd];
            const uint32_t base = next[dd];
            if ((uint32_t)i < lim) vout[base + (uint32_t)i] = vals[beg + sv[i]];
            if (i == m - 1 || sd[i + 1] != dd) {
                const uint32_t e = min((uint32_t)i + 1u, lim);
                front[k] = base + e;
                left[k] = (uint16_t)(lim - e);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kBkItems; ++k)
        if (front[k] != 0xffffffffu) {
            const uint32_t dd = sd[tid + k * kBkThreads];
            next[dd] = front[k];
            room[dd] = left[k];
        }
    __syncthreads();
}

__global__ void __launch_bounds__(kBkThreads, 2) k_bucket_scatter_cap(
    const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, uint32_t *__restrict__ vout, size_t n,
    int nbins, size_t per_block, const uint32_t *__restrict__ offs, int nblocks,
    const uint32_t *__restrict__ ostart, uint32_t cap) {
    extern __shared__ __align__(16) unsigned char bk_smem[];
    const int nbp = bk_nbp(nbins);
    uint32_t *next = reinterpret_cast<uint32_t *>(bk_smem);
    uint16_t *room = reinterpret_cast<uint16_t *>(next + nbp);
    uint16_t *sd = room + nbp;                                   // [kBkSub] buffered digits
    uint16_t *cd = sd + kBkSub;                                  // [kBkSub] overflow digits
    uint32_t *sv = reinterpret_cast<uint32_t *>(cd + kBkSub);    // [kBkSub] buffered item indices
    uint32_t *cv = sv + kBkSub;                                  // [kBkSub] overflow item indices
    uint32_t *wc = cv + kBkSub;                                  // [kBkWarps][kBkLocal]
    uint32_t *dstart = wc + kBkWarps * kBkLocal;                 // [kBkLocal]
    uint32_t *wlive = dstart + kBkLocal;                         // [kBkWarps] live items per warp
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int d = tid; d < nbins; d += kBkThreads) {
        const uint32_t before = min(offs[(size_t)d * nblocks + blockIdx.x] - offs[(size_t)d * nblocks], cap);
        next[d] = ostart[d] + before;
        room[d] = (uint16_t)(cap - before);
    }
    __syncthreads();
    const size_t beg = (size_t)blockIdx.x * per_block;
    const size_t end = min(n, beg + per_block);
    const uint32_t top = (uint32_t)nbins - 1;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int slot0 = w * (32 * kBkItems) + lane;
    uint32_t key[kBkItems];
    auto load = [&](size_t s0) {
#pragma unroll
        for (int j = 0; j < kBkItems; ++j) {
            const size_t idx = s0 + (size_t)(slot0 + j * 32);
            if (idx < end) key[j] = keys[idx];
        }
    };
    if (beg < end) load(beg);
    int fill = 0;  // buffered items (the same in every thread)
    for (size_t s0 = beg; s0 < end; s0 += kBkSub) {
        const int nvalid = (int)min((size_t)kBkSub, end - s0);
        uint32_t d[kBkItems];
        bool live[kBkItems];
#pragma unroll
        for (int j = 0; j < kBkItems; ++j) {
            d[j] = min(key[j], top);
            live[j] = slot0 + j * 32 < nvalid && room[d[j]] > 0;
        }
        if (s0 + kBkSub < end) load(s0 + kBkSub);
        // order-preserving compaction of the live items behind the buffered ones
        uint32_t mask[kBkItems], wl = 0;
#pragma unroll
        for (int j = 0; j < kBkItems; ++j) {
            mask[j] = __ballot_sync(0xffffffffu, live[j]);
            wl += __popc(mask[j]);
        }
        if (lane == 0) wlive[w] = wl;
        __syncthreads();
        uint32_t pos = (uint32_t)fill, total = 0;
#pragma unroll
        for (int ww = 0; ww < kBkWarps; ++ww) {
            const uint32_t c = wlive[ww];
            pos += ww < w ? c : 0u;
            total += c;
        }
#pragma unroll
        for (int j = 0; j < kBkItems; ++j) {
            if (live[j]) {
                const uint32_t p = pos + __popc(mask[j] & lt_mask);
                const uint32_t idx = (uint32_t)(s0 - beg) + (uint32_t)(slot0 + j * 32);
                if (p < (uint32_t)kBkSub) {
                    sd[p] = (uint16_t)d[j];
                    sv[p] = idx;
                } else {
                    cd[p - kBkSub] = (uint16_t)d[j];
                    cv[p - kBkSub] = idx;
                }
            }
            pos += __popc(mask[j]);
        }
        fill += (int)total;
        __syncthreads();
        if (fill >= kBkSub) {
            bk_cap_flush(kBkSub, sd, sv, wc, dstart, next, room, vals, beg, vout);
            fill -= kBkSub;
            for (int i = tid; i < fill; i += kBkThreads) {
                sd[i] = cd[i];
                sv[i] = cv[i];
            }
            __syncthreads();
        }
    }
    if (fill > 0) bk_cap_flush(fill, sd, sv, wc, dstart, next, room, vals, beg, vout);
}

}  // namespace

size_t bucket_sort_scratch_bytes(size_t n, int nbins, int num_sms) {
    if (nbins <= 0) return 0;
    const size_t nblocks = std::max<size_t>(
        1, std::min<size_t>((n + kBkSub - 1) / kBkSub, (size_t)std::max(num_sms, 1) * 4 * kBkCapWaves));
    const size_t hist_n = (size_t)nbins * nblocks;
    const size_t aux = ((size_t)nbins * 4 + ((size_t)nbins + 31) / 32 * 4 + 255) & ~size_t(255);
    return ((hist_n * 4 + 255) & ~size_t(255)) + aux + scan_scratch_bytes(hist_n);
}

cudaError_t bucket_sort_u32(const uint32_t *keys, const uint32_t *vals, uint32_t *vals_out, size_t n, int nbins,
                            uint32_t cap, uint2 *ranges, uint32_t *trunc, void *scratch, size_t scratch_bytes,
                            int num_sms, cudaStream_t st, const int *gate) {
    if (gate && cap != kNoListCap) return cudaErrorInvalidValue;
    if (nbins <= 0 || nbins > kMaxBucketBins) return cudaErrorInvalidValue;
    if (cap < kNoListCap && (cap > (uint32_t)kMaxListCap || nbins >= kMaxBucketBins)) return cudaErrorInvalidValue;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(ranges, 0, (size_t)nbins * sizeof(uint2), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(trunc, 0, ((size_t)nbins + 31) / 32 * 4, st);
        return e;
    }
    if (n >= (size_t)UINT32_MAX) return cudaErrorInvalidValue;
    const bool capped = cap < kNoListCap;
    const size_t smem = capped ? bk_scatter_cap_smem(nbins) : bk_scatter_smem(nbins);
    static thread_local int attr_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_dev != dev) {
        e = cudaFuncSetAttribute(k_bucket_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bk_scatter_smem(kMaxBucketBins));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_bucket_scatter_cap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bk_scatter_cap_smem(kMaxBucketBins));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_bucket_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kMaxBucketBins * 4);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    int occ = 1;
    e = capped ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bucket_scatter_cap, kBkThreads, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bucket_scatter, kBkThreads, smem);
    if (e != cudaSuccess) return e;
    occ = std::max(1, std::min(occ, 4));
    // uncapped: one wave of at most num_sms * occupancy blocks, each a run of
    // whole sub-tiles.  Capped: kBkCapWaves times as many shorter runs, since
    // the runs that hold a view's nearest layers (where the lists are still
    // filling) carry nearly all the work
    const size_t subs = (n + kBkSub - 1) / kBkSub;
    size_t nblocks = std::min(subs, (size_t)std::max(num_sms, 1) * occ * (capped ? kBkCapWaves : 1));
    const size_t per_block = ((subs + nblocks - 1) / nblocks) * kBkSub;
    nblocks = (n + per_block - 1) / per_block;
    const size_t hist_n = (size_t)nbins * nblocks;
    const size_t hist_bytes = (hist_n * 4 + 255) & ~size_t(255);
    const size_t aux = ((size_t)nbins * 4 + ((size_t)nbins + 31) / 32 * 4 + 255) & ~size_t(255);
    if (hist_bytes + aux + scan_scratch_bytes(hist_n) > scratch_bytes) return cudaErrorInvalidValue;
    uint32_t *hist = static_cast<uint32_t *>(scratch);
    uint32_t *ostart = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + hist_bytes);
    void *scr = static_cast<char *>(scratch) + hist_bytes + aux;
    k_bucket_hist<<<(int)nblocks, kBkHistThreads, (size_t)nbins * 4, st>>>(keys, n, nbins, per_block, hist,
                                                                           (int)nblocks, gate);
    e = scan_impl<uint32_t>(hist, hist, hist_n, scr, 0, st, gate);
    if (e != cudaSuccess) return e;
    k_bucket_ranges<<<1, kBkRangeThreads, 0, st>>>(hist, nbins, (int)nblocks, (uint32_t)n, cap, ranges, ostart,
                                                   trunc, gate);
    if (capped)
        k_bucket_scatter_cap<<<(int)nblocks, kBkThreads, smem, st>>>(keys, vals, vals_out, n, nbins, per_block,
                                                                     hist, (int)nblocks, ostart, cap);
    else
        k_bucket_scatter<<<(int)nblocks, kBkThreads, smem, st>>>(keys, vals, vals_out, n, nbins, per_block, hist,
                                                                 (int)nblocks, gate);
    return cudaGetLastError();
}

namespace {
__global__ void k_keys_from_ranges(const uint2 *__restrict__ ranges, uint32_t *__restrict__ keys) {
    const uint2 r = ranges[blockIdx.x];
    for (uint32_t i = r.x + threadIdx.x; i < r.y; i += blockDim.x) keys[i] = blockIdx.x;
}
}  // namespace

cudaError_t keys_from_ranges(const uint2 *ranges, int nbins, uint32_t *keys, cudaStream_t st) {
    if (nbins <= 0) return cudaSuccess;
    k_keys_from_ranges<<<nbins, 256, 0, st>>>(ranges, keys);
    return cudaGetLastError();
}

cudaError_t radix_sort_u32_fixed(uint32_t **key_io, uint32_t **key_alt, uint32_t **val_io,
                                 uint32_t **val_alt, size_t n, int end_bit, void *scratch,
                                 size_t scratch_bytes, cudaStream_t st) {
    return radix_fixed<uint32_t>(key_io, key_alt, val_io, val_alt, n, end_bit, scratch,
                                 scratch_bytes, st);
}

cudaError_t radix_sort_u64_fixed(uint64_t **key_io, uint64_t **key_alt, uint32_t **val_io,
                                 uint32_t **val_alt, size_t n, int end_bit, void *scratch,
                                 size_t scratch_bytes, cudaStream_t st) {
    return radix_fixed<uint64_t>(key_io, key_alt, val_io, val_alt, n, end_bit, scratch,
                                 scratch_bytes, st);
}

size_t scan_scratch_bytes(size_t n) {
    size_t nb = (n + kScanTile - 1) / kScanTile + 1;
    return 256 + nb * sizeof(uint64_t);
}

size_t radix_hist_bytes(size_t n) {
    size_t nblocks = (n + Radix<uint64_t>::tile - 1) / Radix<uint64_t>::tile;
    size_t hist_n = (size_t)kBins * nblocks;
    return hist_n * 4 + 256 + scan_scratch_bytes(hist_n);
}

cudaError_t radix_sort_u32(uint32_t **key_io, uint32_t **key_alt, uint32_t **val_io,
                           uint32_t **val_alt, size_t n, int end_bit, SortScratch &s,
                           cudaStream_t st) {
    return radix_impl<uint32_t>(key_io, key_alt, val_io, val_alt, n, end_bit, s, st);
}

cudaError_t radix_sort_u64(uint64_t **key_io, uint64_t **key_alt, uint32_t **val_io,
                           uint32_t **val_alt, size_t n, int end_bit, SortScratch &s,
                           cudaStream_t st) {
    return radix_impl<uint64_t>(key_io, key_alt, val_io, val_alt, n, end_bit, s, st);
}

cudaError_t exclusive_scan_u32_u64(const uint32_t *in, uint64_t *out, size_t n, void *scratch,
                                   cudaStream_t st) {
    return scan_impl<uint64_t>(in, out, n, scratch, 1, st);
}

}  // namespace ups
