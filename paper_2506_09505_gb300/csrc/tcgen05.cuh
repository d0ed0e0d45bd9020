// Building blocks of the tensor-core kernels (tcgen05, sm_103a): shared-
// memory matrix descriptors, one-thread MMA issue and commit to an
// mbarrier, bounded mbarrier waits, tensor-memory loads and stores, and the
// exact byte-limb arithmetic around a contraction: a 64-bit word split into
// its 8 bytes as fp16 subnormals (bits = byte) for an A operand, and the
// combination of eight fp32 column sums (bits 0x3E800000 + offset + Z, see
// TcTables) back into a word mod p.
//
// Every contraction here is D[128 x N] (+)= A[128 x K] B[N x K]^T with fp16
// A and B in K-major, unswizzled 8 x 8 core matrices of 128 contiguous
// bytes, and fp32 accumulators in tensor memory, row = lane.
#pragma once
#include <cstdint>

#include "field.cuh"

namespace pg12 {
namespace dev {

// instruction descriptor: fp16 A and B, fp32 D, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t tc_idesc(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// a wait that has not seen the tensor cores finish after this many SM clocks gives up
constexpr long long kTcWaitClocks = 4ll << 30;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: no swizzle, K-major; lbo = byte distance
// between core matrices along K, sbo = along M (or N); bit 46 is the
// descriptor version of this architecture.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void group_sync(int id, int threads = 128) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Barrier of a group of threads that also ORs a flag over them (the same
// answer in every thread).
__device__ __forceinline__ uint32_t group_sync_or(int id, uint32_t flag, int threads = 128) {
    uint32_t any;
    asm volatile("{\n\t.reg .pred q, p;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, %3, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(any)
                 : "r"(flag), "r"(id), "r"(threads)
                 : "memory");
    return any;
}

// Waits for phase `parity` of the mbarrier; false if it has not completed
// within kTcWaitClocks (the clock is read only after a first test failed).
__device__ __forceinline__ uint32_t mbar_try(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(a), "r"(parity)
                 : "memory");
    return done;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
    const uint32_t a = smem_addr(mbar);
    if (mbar_try(a, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(a, parity)) return true;
        if (clock64() - t0 > kTcWaitClocks) return false;
    }
}

// Consecutive 32-bit columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ uint64_t tmem_ld_word(uint32_t taddr) {
    uint32_t lo, hi;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(lo), "=r"(hi) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ void tmem_st_words(uint32_t taddr, uint64_t a, uint64_t b) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(lo32(a)), "r"(hi32(a)),
                 "r"(lo32(b)), "r"(hi32(b))
                 : "memory");
}

// y = sum_b 2^(8b) w[b] + x mod p for eight column words w[b] < 2^31 and a
// 64-bit x: two 56-bit sums lo = sum_(b<4), hi = sum_(b>=4) (IMAD.WIDE with
// the running sum as addend), V = lo + hi 2^32 + x < 2^89 = lo' + h 2^64 with
// lo' = lo + x + hi.lo 2^32 and h = hi.hi + carries, then the fold
// (2^64 = 2^32 - 1).
__device__ __forceinline__ uint64_t tc_combine(const uint32_t *w, uint64_t x = 0) {
    uint64_t lo = madw(w[1], 1u << 8, (uint64_t)w[0]);
    lo = madw(w[2], 1u << 16, lo);
    lo = madw(w[3], 1u << 24, lo);
    uint64_t hi = madw(w[5], 1u << 8, (uint64_t)w[4]);
    hi = madw(w[6], 1u << 16, hi);
    hi = madw(w[7], 1u << 24, hi);
    uint32_t l0, l1, h;
    asm("add.cc.u32 %0, %3, %5;\n\t"
        "addc.cc.u32 %1, %4, %6;\n\t"
        "addc.u32 %2, %8, 0;\n\t"
        "add.cc.u32 %1, %1, %7;\n\t"
        "addc.u32 %2, %2, 0;"
        : "=r"(l0), "=r"(l1), "=r"(h)
        : "r"(lo32(lo)), "r"(hi32(lo)), "r"(lo32(x)), "r"(hi32(x)), "r"(lo32(hi)), "r"(hi32(hi)));
    return fold(((uint64_t)l1 << 32) | l0, (uint64_t)h, 0);
}

// The 8 bytes of y as fp16 subnormals whose bit patterns are the bytes
// (one 16-byte row of a K chunk), and the word back from such a row.
__device__ __forceinline__ uint4 tc_bytes(uint64_t y) {
    const uint32_t lo = lo32(y), hi = hi32(y);
    uint4 v;
    v.x = __byte_perm(lo, 0u, 0x4140);
    v.y = __byte_perm(lo, 0u, 0x4342);
    v.z = __byte_perm(hi, 0u, 0x4140);
    v.w = __byte_perm(hi, 0u, 0x4342);
    return v;
}
__device__ __forceinline__ uint64_t tc_word(uint4 v) {
    return ((uint64_t)__byte_perm(v.z, v.w, 0x6420) << 32) | __byte_perm(v.x, v.y, 0x6420);
}

}  // namespace dev
}  // namespace pg12
