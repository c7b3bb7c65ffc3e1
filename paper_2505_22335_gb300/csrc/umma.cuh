// Minimal tcgen05 (5th-generation tensor core) helpers for sm_100a/sm_103a:
// shared-memory matrix descriptors for canonical K-major, no-swizzle operands,
// instruction descriptors for kind::f16 (BF16) and kind::tf32 with FP32
// accumulation, TMEM allocation, MMA issue/commit, bounded mbarrier waits and
// TMEM loads.  Written from the PTX ISA description of these instructions.
//
// Canonical K-major layout (no swizzle): an M x K operand is a grid of "core
// matrices" of 8 rows x 16 bytes (8 BF16 or 4 TF32 elements per row); the 8
// rows of a core matrix are 16 bytes apart, core matrices adjacent along K are
// LBO = 128 bytes apart, 8-row groups are SBO = (K bytes / 16) * 128 apart.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace ups {
namespace umma {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) of a canonical K-major operand whose rows
// hold `kbytes` bytes (a multiple of 16), element size `esize`.
__device__ __forceinline__ uint32_t kmajor_offset(int row, int k, int kbytes, int esize) {
    const int per_core = 16 / esize;
    return (uint32_t)(((row >> 3) * (kbytes >> 4) + k / per_core) * 128 + (row & 7) * 16 +
                      (k % per_core) * esize);
}

__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t kbytes) {
    const uint32_t lbo = 128, sbo = (kbytes >> 4) * 128;
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;
}

// K-major operand in the 64-byte swizzle layout, as a tiled TMA load with
// 64-byte swizzle writes it: rows of 64 bytes (16 TF32 values of K), 8-row
// groups 512 bytes apart (SBO), the 16-byte chunks of row r permuted by XOR
// with (r / 2) % 4 (bits 4-5 of the address XOR bits 7-8).  Operand bases are
// 512-byte aligned; a K step inside the 64-byte row advances the start
// address by its byte offset.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                // LBO: unused for a swizzled K-major operand one atom wide
    d |= (uint64_t)((512 >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                // descriptor version
    d |= (uint64_t)4 << 61;                // layout: 64-byte swizzle
    return d;
}

enum Kind { kBF16 = 0, kTF32 = 1 };

__host__ __device__ constexpr uint32_t idesc(Kind kind, int M, int N) {
    return (1u << 4)                                   // D: FP32
           | ((kind == kBF16 ? 1u : 2u) << 7)           // A format
           | ((kind == kBF16 ? 1u : 2u) << 10)          // B format
           | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <Kind K>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    if (K == kBF16)
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
                     "l"(a), "l"(b), "r"(id), "r"(acc));
    else
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
                     "l"(a), "l"(b), "r"(id), "r"(acc));
}

// kind::f16 MMA with A in tensor memory (rows in lanes, K along columns, two
// 16-bit elements per 32-bit column, the lower K index in the low half) and B
// from a shared-memory descriptor
__device__ __forceinline__ void mma_f16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(tmem_d),
                 "r"(tmem_a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_addr(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// Waits for the phase with parity `parity`; gives up after `limit` polls and
// returns false (the caller records the failure and skips the TMEM reads).
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, int limit) {
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(smem_addr(mbar)), "r"(parity));
    return done != 0;
}

// bulk copy (TMA, untiled) global -> shared, completing `bytes` of the
// transaction count of *mbar; both addresses 16-byte aligned, bytes a multiple
// of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}

// arrive on *mbar (one of its expected arrivals) and add `bytes` to the
// transaction count of the current phase
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// tiled TMA load of the box at (x, y) of a 2D tensor map (a kernel parameter
// declared __grid_constant__) into shared memory, completing on *mbar
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_addr(mbar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_addr(mbar)) : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }

// one warp: allocate `ncols` TMEM columns (power of two >= 32), address to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive 32-bit columns of this thread's TMEM lane from registers
// (complete once tmem_st_wait returns)
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::
            "r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// TF32 split: x = hi + lo with hi a TF32 value (round to nearest) and lo the
// FP32 remainder; hi*b_hi + hi*b_lo + lo*b_hi recovers FP32-level products.
__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace umma
}  // namespace ups
