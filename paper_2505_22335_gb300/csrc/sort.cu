// Stable LSD radix sort of (key, value) pairs and exclusive scans, written for
// this library (no CUB).  Used twice per forward: once to order Gaussian-views
// by (view, depth) and once to bucket the depth-ordered tile instances by
// (view, tile), which together give the (view, tile, depth, id) order.
//
// One pass = histogram kernel (per-block digit counts, digit-major layout) +
// exclusive scan of the counts + scatter kernel (stable block-local ranking by
// ballots, then a scatter to the scanned offsets).
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

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in,
                                                              size_t n, T *__restrict__ partial) {
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
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(T *partial, int nb) {
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
                                                             int write_total) {
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
                      cudaStream_t st) {
    if (n == 0) {
        if (write_total) return cudaMemsetAsync(out, 0, sizeof(T), st);
        return cudaSuccess;
    }
    int nb = (int)((n + kScanTile - 1) / kScanTile);
    T *partial = static_cast<T *>(scratch);
    k_scan_reduce<T><<<nb, kScanThreads, 0, st>>>(in, n, partial);
    k_scan_partials<T><<<1, kScanThreads, 0, st>>>(partial, nb);
    k_scan_apply<T><<<nb, kScanThreads, 0, st>>>(in, out, n, partial, write_total);
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

}  // namespace

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
