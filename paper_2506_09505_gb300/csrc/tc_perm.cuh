// Poseidon-12 permutation with the full rounds' dense layers on the tensor
// cores (tcgen05, sm_103a), 128 states per group of 128 threads.
//
// Alg. 1's full rounds are x <- M S(x + c_r).  The S-boxes and the partial
// rounds stay on the integer pipes (one thread per state, as in
// poseidon.cuh); the 12x12 products M y of a whole group are one tensor-core
// contraction of byte limbs (the digit scheme of TcTables in
// pg12_internal.h):
//
//   thread t: y_j = S(x_j + c_rj), its 8 bytes -> row t of A (fp16
//             subnormals, bits = byte), in shared memory
//   leader  : D[128 x 96] = A[128 x 96] * B_m^T + bias   (7 tcgen05.mma, K = 16
//             each, fp32 accumulators in tensor memory), commit -> mbarrier
//   thread t: reads row t of D (tcgen05.ld), y_i = sum_b 2^(8b) bits(D[t][8i+b])
//             folded mod p
//
// Every fp32 sum is an exact integer below 2^24, so the result is the exact
// residue: the same function as the integer-pipe form, bit for bit after
// canonicalisation.  A group's threads meet at one named barrier per round
// (A written, D of the previous round read) and wait on the group's
// mbarrier for the tensor cores; every wait is bounded.
#pragma once
#include "poseidon.cuh"

namespace pg12 {
namespace dev {

constexpr int kTcGroup = 128;                 // states (threads) per group
constexpr int kTcAChunk = 128;                // bytes of one 8 x 8 fp16 core matrix
constexpr int kTcAChunks = kTcK / 8;           // core-matrix columns of A (12)
constexpr int kTcABytes = kTcGroup * kTcK * 2;  // A operand of a group: 24 KiB
constexpr int kTcSlotBytes = kTcGroup * kT * 8;
constexpr int kTcDCols = kTcN;                // columns of one group's D (96, a multiple of 32)
// tensor-memory columns one CTA of `groups` groups allocates: a power of two
// (at least 32) that holds every group's D
constexpr int tc_tmem_alloc(int groups) {
    return groups * kTcDCols <= 128 ? 128 : groups * kTcDCols <= 256 ? 256 : 512;
}
// instruction descriptor: fp16 A and B, fp32 D, both K-major, N = 96, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcGroup >> 4) << 24);
// a wait that has not seen the tensor cores finish after this many SM clocks gives up
constexpr long long kTcWaitClocks = 4ll << 30;

__device__ __align__(16) TcTables g_tc;  // uploaded with the other constant tables

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: no swizzle, K-major; lbo = byte distance
// between core matrices along K, sbo = along M (or N); bit 46 is the
// descriptor version of this architecture.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                 "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kTcGroup) : "memory"); }

// Barrier of a group's 128 threads that also ORs a flag over them (the
// same answer in every thread).
__device__ __forceinline__ uint32_t group_sync_or(int id, uint32_t flag) {
    uint32_t any;
    asm volatile("{\n\t.reg .pred q, p;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, %3, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(any)
                 : "r"(flag), "r"(id), "r"(kTcGroup)
                 : "memory");
    return any;
}

// Waits for phase `parity` of the mbarrier; false if it has not completed
// within kTcWaitClocks.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
    const uint32_t a = smem_addr(mbar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if (clock64() - t0 > kTcWaitClocks) return false;
    }
}

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// y = sum_b 2^(8b) w[b] mod p for eight column words w[b] < 2^31: two 56-bit
// sums lo = sum_(b<4), hi = sum_(b>=4) (IMAD.WIDE with the running sum as
// addend), V = lo + hi 2^32 < 2^88 = lo' + h 2^64 with lo' = lo + hi.lo 2^32
// and h = hi.hi + carry, then the fold (2^64 = 2^32 - 1).
__device__ __forceinline__ uint64_t tc_combine(const uint32_t *w) {
    uint64_t lo = madw(w[1], 1u << 8, (uint64_t)w[0]);
    lo = madw(w[2], 1u << 16, lo);
    lo = madw(w[3], 1u << 24, lo);
    uint64_t hi = madw(w[5], 1u << 8, (uint64_t)w[4]);
    hi = madw(w[6], 1u << 16, hi);
    hi = madw(w[7], 1u << 24, hi);
    uint32_t l1, h;
    asm("add.cc.u32 %0, %2, %3;\n\t"
        "addc.u32 %1, %4, 0;"
        : "=r"(l1), "=r"(h)
        : "r"(hi32(lo)), "r"(lo32(hi)), "r"(hi32(hi)));
    return fold(((uint64_t)l1 << 32) | lo32(lo), (uint64_t)h, 0);
}

// One group's share of the CTA's shared memory and tensor memory.
struct TcGroup {
    uint8_t *a;           // A operand, kTcABytes
    uint64_t *slot;       // states: cell i of thread t at slot[i * kTcGroup + t]
    uint64_t *mbar;       // tensor-core completion barrier
    uint32_t tmem;        // D: lanes 0..127, kTcDCols columns
    uint32_t phase;       // parity of the mbarrier's next completion
    int bar;              // named barrier of the group's 128 threads
    int t;                // thread index within the group
    uint32_t failed;      // this thread saw a tensor-core wait run out
    volatile uint32_t *bcast;  // one word through which thread 0 hands the group a value
    uint32_t a_addr, b_addr, bias_addr, zcap_addr;  // shared addresses for the descriptors
};

// Row t's chunk j of A (K columns 8j..8j+7) <- the 8 bytes of y as fp16 subnormals.
__device__ __forceinline__ void tc_put(const TcGroup &G, int j, uint64_t y) {
    const uint32_t lo = lo32(y), hi = hi32(y);
    uint4 v;
    v.x = __byte_perm(lo, 0u, 0x4140);
    v.y = __byte_perm(lo, 0u, 0x4342);
    v.z = __byte_perm(hi, 0u, 0x4140);
    v.w = __byte_perm(hi, 0u, 0x4342);
    *reinterpret_cast<uint4 *>(G.a + ((G.t >> 3) * kTcAChunks + j) * kTcAChunk + (G.t & 7) * 16) = v;
}


// Dense layer of round r (matrix m: 0 = M, 1 = transition) on the states
// whose S-box outputs are in A; writes rows 0..rows-1 of the result to the
// slots.  z: round 0 of states whose capacity entered as zero (A holds
// cells 0..7; cells 8..11 come from the constant zcap pattern).  Returns
// false, in every thread of the group, once a wait of the group has run out.
__device__ __forceinline__ bool tc_dense(TcGroup &G, int m, bool z, int rows) {
    fence_async_smem();   // this thread's A stores -> the tensor cores' proxy
    tc_fence_before();    // its tensor-memory reads of the previous round are complete
    if (group_sync_or(G.bar, G.failed)) return false;
    if (G.t == 0) {
        tc_fence_after();
        const uint32_t bm = G.b_addr + (uint32_t)m * (uint32_t)sizeof(TcTables::b[0]);
        constexpr uint32_t sbo_b = kTcKC * kTcAChunk, sbo_a = kTcAChunks * kTcAChunk;
        tc_mma(G.tmem, tc_desc(G.bias_addr, kTcAChunk, 0), tc_desc(bm + 12 * kTcAChunk, kTcAChunk, sbo_b), 0);
#pragma unroll
        for (int kb = 0; kb < 6; ++kb) {
            const uint64_t a = (z && kb >= 4) ? tc_desc(G.zcap_addr + (kb - 4) * 2 * kTcAChunk, kTcAChunk, 0)
                                              : tc_desc(G.a_addr + kb * 2 * kTcAChunk, kTcAChunk, sbo_a);
            tc_mma(G.tmem, a, tc_desc(bm + kb * 2 * kTcAChunk, kTcAChunk, sbo_b), 1);
        }
        tc_commit(G.mbar);
    }
    const bool ok = mbar_wait(G.mbar, G.phase);
    G.phase ^= 1u;
    if (!ok) G.failed = 1;
    tc_fence_after();
    const uint32_t lane_base = G.tmem + ((uint32_t)(G.t & ~31) << 16);
    uint64_t *slot = G.slot + G.t;
#pragma unroll 1
    for (int i = 0; i < rows; i += 2) {
        uint32_t w[16];
        tmem_ld16(lane_base + 8 * i, w);
        slot[i * kTcGroup] = tc_combine(w);
        slot[(i + 1) * kTcGroup] = tc_combine(w + 8);
    }
    return true;
}

// Code shape of the tensor-core path (measured on the 2^22 x 8 tree, 4
// groups): S-boxes four cells per loop iteration and the partial rounds'
// eleven cells unrolled in registers, 10.25 ms; two cells per iteration and
// the cells walked in the slots (the integer-pipe kernels' shape), 10.67 ms.
#ifndef PG12_TC_SBOX_CELLS
#define PG12_TC_SBOX_CELLS 4  // 1, 2 or 4 (divides 8 and 12)
#endif
#ifndef PG12_TC_PARTIAL_LOOP
#define PG12_TC_PARTIAL_LOOP 0
#endif

// The permutation on the group's slots (weak words in, weak words out),
// with the same zcap / digest shortcuts as permute_slot.
__device__ __forceinline__ bool tc_permute(TcGroup &G, bool zcap, bool digest) {
    uint64_t *slot = G.slot + G.t;
#pragma unroll 1
    for (int r = 0; r < kRF; ++r) {
        const bool z = zcap && r == 0;
        const int cells = z ? kRate : kT;
#pragma unroll 1
        for (int j = 0; j < cells; j += PG12_TC_SBOX_CELLS) {
            uint64_t a[PG12_TC_SBOX_CELLS];
#pragma unroll
            for (int k = 0; k < PG12_TC_SBOX_CELLS; ++k) a[k] = add_canon(slot[(j + k) * kTcGroup], c_dev.full_rc[r][j + k]);
#pragma unroll
            for (int k = 0; k < PG12_TC_SBOX_CELLS; ++k) tc_put(G, j + k, sbox(a[k]));
        }
        if (!tc_dense(G, r == kRF / 2 - 1 ? 1 : 0, z, digest && r == kRF - 1 ? kDigest : kT)) return false;
        if (r == kRF / 2 - 1) partial_phase<kTcGroup, PG12_TC_PARTIAL_LOOP>(slot);
    }
    return true;
}

// Shared-memory layout of a CTA of GROUPS groups: the tables, then each
// group's A operand, then each group's state slots, then the barriers.
template <int GROUPS>
struct TcLayout {
    static_assert(GROUPS * kTcDCols <= 512, "the groups' accumulators exceed tensor memory");
    static constexpr int kTmemCols = tc_tmem_alloc(GROUPS);
    static constexpr size_t kTables = 0;
    static constexpr size_t kA = (sizeof(TcTables) + 127) & ~(size_t)127;
    static constexpr size_t kSlot = kA + (size_t)GROUPS * kTcABytes;
    static constexpr size_t kBar = kSlot + (size_t)GROUPS * kTcSlotBytes;
    static constexpr size_t kBcast = kBar + 8 * GROUPS + 16;
    static constexpr size_t kBytes = kBcast + 4 * GROUPS;
};

__device__ int g_tc_fault;  // set when a tensor-core wait ran out (read by pg_device_flags)

// Prologue of a tensor-core kernel: tables into shared memory, the groups'
// barriers, one tensor-memory allocation for all groups.
template <int GROUPS>
__device__ __forceinline__ TcGroup tc_setup(uint8_t *sm) {
    using L = TcLayout<GROUPS>;
    const uint4 *src = reinterpret_cast<const uint4 *>(&g_tc);
    uint4 *dst = reinterpret_cast<uint4 *>(sm + L::kTables);
    for (unsigned i = threadIdx.x; i < sizeof(TcTables) / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::kBar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + GROUPS);
    if (threadIdx.x == 0) {
        for (int g = 0; g < GROUPS; ++g) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bars + g)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(L::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int g = threadIdx.x / kTcGroup;
    TcGroup G;
    G.t = threadIdx.x % kTcGroup;
    G.failed = 0;
    G.a = sm + L::kA + (size_t)g * kTcABytes;
    G.slot = reinterpret_cast<uint64_t *>(sm + L::kSlot + (size_t)g * kTcSlotBytes);
    G.mbar = bars + g;
    G.tmem = *tslot + (uint32_t)(g * kTcDCols);
    G.phase = 0;
    G.bar = 1 + g;
    G.bcast = reinterpret_cast<volatile uint32_t *>(sm + L::kBcast) + g;
    const TcTables *T = reinterpret_cast<const TcTables *>(sm + L::kTables);
    G.a_addr = smem_addr(G.a);
    G.b_addr = smem_addr(T->b[0]);
    G.bias_addr = smem_addr(T->a_bias);
    G.zcap_addr = smem_addr(T->a_zcap);
    return G;
}

// Thread 0 adds one to *counter; every thread of the group gets the old
// value.  The first barrier orders the group's earlier stores (each thread
// fences its own first) before the atomic and keeps thread 0 from
// overwriting a value others have not read yet.
__device__ __forceinline__ uint32_t group_fetch_add(TcGroup &G, uint32_t *counter) {
    group_sync(G.bar);
    if (G.t == 0) *G.bcast = atomicAdd(counter, 1u);
    group_sync(G.bar);
    return *G.bcast;
}

// Epilogue: every group is done with tensor memory; the allocating warp
// frees it.  A group whose wait ran out records the fault and gives its
// last contraction one more bounded wait before the memory is freed.
template <int GROUPS>
__device__ __forceinline__ void tc_teardown(uint8_t *sm, TcGroup &G) {
    using L = TcLayout<GROUPS>;
    if (G.failed) {
        atomicExch(&g_tc_fault, 1);
        if (G.t == 0) mbar_wait(G.mbar, G.phase ^ 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        const uint32_t base = *reinterpret_cast<uint32_t *>(sm + L::kBar + 8 * GROUPS);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(L::kTmemCols));
    }
}

}  // namespace dev
}  // namespace pg12
