// Poseidon-12 permutation with its dense contractions on the tensor cores
// (tcgen05, sm_103a), 128 states per group of 128 threads.
//
// Alg. 1's full rounds are x <- M S(x + c_r); the 12x12 products M y of a
// whole group are one tensor-core contraction of byte limbs (the digit scheme
// of TcTables in pg12_internal.h):
//
//   thread t: y_j = S(x_j + c_rj), its 8 bytes -> row t of A (fp16
//             subnormals, bits = byte), in shared memory
//   leader  : D[128 x 96] = A[128 x 96] * B^T + bias   (7 tcgen05.mma, K = 16
//             each, fp32 accumulators in tensor memory), commit -> mbarrier
//   thread t: reads row t of D (tcgen05.ld), y_i = sum_b 2^(8b) bits(D[t][8i+b])
//             folded mod p
//
// The 22 partial rounds (Alg. 1, MDSPartial) run in their unrolled form
// (ChainParams): the dot products U_q with the partial rounds' input and the
// deferred cell updates W s are contractions of round 3's S-box bytes and of
// the 22 partial S-box outputs; only the chain c_q -> s_q = S(c_q + k_q) ->
// c_(q+1) = U_q + sum_(r<=q) beta[q][r] s_r runs on the integer pipes, one
// thread per state, in two halves: the first half's terms in the second
// half's chain values are one more contraction, so each thread forms 110 of
// the 231 products beta[q][r] s_r.
//
// Every fp32 sum is an exact integer below 2^24 (times 2^-24), so each result
// is the exact residue: the same function as the integer-pipe form, bit for
// bit after canonicalisation.  A group's threads meet at one named barrier
// per contraction (operands written, the previous accumulators read) and
// wait on the group's mbarrier for the tensor cores; every wait is bounded.
#pragma once
#include <cstddef>

#include "poseidon.cuh"
#include "tcgen05.cuh"

namespace pg12 {
namespace dev {

constexpr int kTcGroup = 128;                   // states (threads) per group
constexpr int kTcAChunk = 128;                  // bytes of one 8 x 8 fp16 core matrix
constexpr int kTcAChunks = kTcK / 8;            // core-matrix columns of A (12 input words)
constexpr int kTcABytes = kTcGroup * kTcK * 2;  // A operand of a group: 24 KiB
constexpr int kTcRegion = 128;                  // tensor-memory columns of one group
constexpr int kTcUStore = kTcN;                 // columns 96..119 of a region hold chain values as words
// tensor-memory columns one CTA of `groups` groups allocates (a power of two)
constexpr int tc_tmem_alloc(int groups) { return groups <= 1 ? 128 : groups <= 2 ? 256 : 512; }

// byte offsets of the tables inside TcTables (and inside its shared-memory copy)
constexpr uint32_t kTabM = offsetof(TcTables, m), kTabPre = offsetof(TcTables, pre);
constexpr uint32_t kTabBBias = offsetof(TcTables, b_bias), kTabABias = offsetof(TcTables, a_bias);
constexpr uint32_t kTabZcap = offsetof(TcTables, a_zcap);
constexpr uint32_t kTabVpa = offsetof(TcTables, vpa), kTabVpb = offsetof(TcTables, vpb), kTabBs = offsetof(TcTables, bs);
constexpr uint32_t kTabW1 = offsetof(TcTables, w1), kTabW2 = offsetof(TcTables, w2);
constexpr size_t kTabCore = offsetof(TcTables, vpa);  // what kernels without the chain copy
static_assert(kTabVpa % 128 == 0 && kTabVpb % 128 == 0 && kTabBs % 128 == 0 && kTabW1 % 128 == 0 &&
                  kTabW2 % 128 == 0 &&
                  kTabBBias % 128 == 0 && kTabZcap % 128 == 0,
              "tables are 128-byte aligned");

__device__ __align__(16) TcTables g_tc;     // uploaded with the other constant tables
__constant__ uint64_t c_beta[kRP][kRP];     // ChainParams::beta

// One group's share of the CTA's shared memory and tensor memory.
struct TcGroup {
    uint8_t *a;           // A operand, kTcABytes
    uint64_t *mbar;       // tensor-core completion barrier
    uint32_t tmem;        // the group's kTcRegion columns, lanes 0..127
    uint32_t phase;       // parity of the mbarrier's next completion
    int bar;              // named barrier of the group's 128 threads
    int t;                // thread index within the group
    uint32_t failed;      // this thread saw a tensor-core wait run out
    volatile uint32_t *bcast;  // one word through which thread 0 hands the group a value
    uint32_t a_addr, tab;      // shared addresses of A and of the tables
};

// Row t's chunk j of A (K columns 8j..8j+7) <- the 8 bytes of y as fp16 subnormals.
__device__ __forceinline__ void tc_put(const TcGroup &G, int j, uint64_t y) {
    *reinterpret_cast<uint4 *>(G.a + ((G.t >> 3) * kTcAChunks + j) * kTcAChunk + (G.t & 7) * 16) = tc_bytes(y);
}

// The word y that tc_put wrote to row t's chunk j (the low byte of each fp16).
__device__ __forceinline__ uint64_t tc_get(const TcGroup &G, int j) {
    return tc_word(*reinterpret_cast<const uint4 *>(G.a + ((G.t >> 3) * kTcAChunks + j) * kTcAChunk + (G.t & 7) * 16));
}

// One contraction into the group's D (columns 0 .. n-1): the group meets
// (its A stores visible to the tensor cores, its earlier tensor-memory
// accesses done), thread 0 issues the bias block (when `bias`: D starts at
// the bias; else D accumulates) and kblocks K = 16 blocks of A (cells 8..11
// from the zero-capacity block when z) against the table at byte offset
// b_off with b_chunks input words per row group, and commits; every thread
// waits.  Returns false, in every thread of the group, once a wait of the
// group has run out.
__device__ __forceinline__ bool tc_contract(TcGroup &G, uint32_t b_off, uint32_t b_chunks, int n, int kblocks,
                                            bool bias, bool z) {
    fence_async_smem();   // this thread's A stores -> the tensor cores' proxy
    tc_fence_before();    // its tensor-memory accesses are complete
    if (group_sync_or(G.bar, G.failed)) return false;
    if (G.t == 0) {
        tc_fence_after();
        const uint32_t idesc = tc_idesc(n);
        const uint32_t sbo_b = b_chunks * kTcAChunk, sbo_a = kTcAChunks * kTcAChunk;
        if (bias)
            tc_mma(G.tmem, tc_desc(G.tab + kTabABias, kTcAChunk, 0), tc_desc(G.tab + kTabBBias, kTcAChunk, 0), idesc,
                   0);
        for (int kb = 0; kb < kblocks; ++kb) {
            const uint64_t a = (z && kb >= 4) ? tc_desc(G.tab + kTabZcap + (kb - 4) * 2 * kTcAChunk, kTcAChunk, 0)
                                              : tc_desc(G.a_addr + kb * 2 * kTcAChunk, kTcAChunk, sbo_a);
            tc_mma(G.tmem, a, tc_desc(G.tab + b_off + kb * 2 * kTcAChunk, kTcAChunk, sbo_b), idesc, 1);
        }
        tc_commit(G.mbar);
    }
    const bool ok = mbar_wait(G.mbar, G.phase);
    G.phase ^= 1u;
    if (!ok) G.failed = 1;
    tc_fence_after();
    return true;
}

// Dense layer of a full round (table at m_off) on the S-box outputs in A;
// rows 0..rows-1 of the result go to x.  z: round 0 of states whose
// capacity entered as zero (A holds cells 0..7; cells 8..11 come from the
// constant zcap block).
__device__ __forceinline__ bool tc_dense(TcGroup &G, uint32_t m_off, bool z, int rows, uint64_t (&x)[kT]) {
    if (!tc_contract(G, m_off, kTcAChunks, kTcN, 6, true, z)) return false;
    const uint32_t lane_base = G.tmem + ((uint32_t)(G.t & ~31) << 16);
#pragma unroll
    for (int i = 0; i < kT; i += 2) {
        if (i < rows) {
            uint32_t w[16];
            tmem_ld16(lane_base + 8 * i, w);
            x[i] = tc_combine(w);
            x[i + 1] = tc_combine(w + 8);
        }
    }
    return true;
}

#ifndef PG12_TC_MAC_UNROLL
#define PG12_TC_MAC_UNROLL 2  // 1: measured 0.5% slower
#endif
constexpr int kTcMacUnroll = PG12_TC_MAC_UNROLL;
// One half of the chain: s_q = S(c + k_q) for q = q0 .. q1 - 1, each into
// A's chunk q - q0; between them c = U_q + sum_(r = q0 .. q) beta[q][r] s_r,
// U_q the word in tensor-memory column kTcUStore + 2 (q - u0).
__device__ __forceinline__ void chain_half(const TcGroup &G, uint32_t lane_base, uint64_t c, int q0, int q1, int u0) {
#pragma unroll 1
    for (int q = q0;; ++q) {
        tc_put(G, q - q0, sbox(add_canon(c, c_dev.part_rc[q])));
        if (q == q1 - 1) break;
        Acc A;
        acc_init(A, tmem_ld_word(lane_base + kTcUStore + 2 * (q - u0)));
#pragma unroll kTcMacUnroll
        for (int r = q0; r <= q; ++r) acc_mac(A, tc_get(G, r - q0), c_beta[q][r]);
        c = acc_reduce(A);
    }
}

// Rows 0 .. rows-1 of D combined into words, stored at tensor-memory columns
// kTcUStore + 2 i.
template <int ROWS>
__device__ __forceinline__ void tc_store_rows(uint32_t lane_base) {
#pragma unroll
    for (int i = 0; i < ROWS; i += 2) {
        uint32_t w[16];
        tmem_ld16(lane_base + 8 * i, w);
        tmem_st_words(lane_base + kTcUStore + 2 * i, tc_combine(w), tc_combine(w + 8));
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// The 22 partial rounds in their unrolled form, after round 3's dense layer
// (A still holds round 3's S-box bytes y3, x holds x^(0) = P y3).
__device__ __forceinline__ bool tc_partial(TcGroup &G, uint64_t (&x)[kT]) {
    const uint32_t lane_base = G.tmem + ((uint32_t)(G.t & ~31) << 16);
    // U_0 .. U_9 as words
    if (!tc_contract(G, kTabVpa, kTcAChunks, kTcUa * 8, 6, true, false)) return false;
    tc_store_rows<kTcUa>(lane_base);
    // U_10 .. U_21 as column sums in D (A still holds y3)
    if (!tc_contract(G, kTabVpb, kTcAChunks, kTcN, 6, true, false)) return false;
    // first half: s_0 .. s_10 into A's chunks 0..10
    chain_half(G, lane_base, x[0], 0, kTcSplit, 0);
    // D += their terms in c_11 .. c_21: the second half's U'_q (q = 10 .. 20) and U_21, as words
    if (!tc_contract(G, kTabBs, kTcAChunks, kTcN, 6, false, false)) return false;
    tc_store_rows<kT>(lane_base);
    // the deferred updates W s, from s_0 .. s_10 now, s_11 .. s_21 after the second half
    if (!tc_contract(G, kTabW1, kTcAChunks, kTcN, 6, true, false)) return false;
    chain_half(G, lane_base, tmem_ld_word(lane_base + kTcUStore), kTcSplit, kRP, kTcUa);
    if (!tc_contract(G, kTabW2, kTcAChunks, kTcN, 6, false, false)) return false;
    // cell 0 = c_22 = U_21 + (W s)_0, cell i = x_i^(0) + (W s)_i
    const uint64_t u21 = tmem_ld_word(lane_base + kTcUStore + 2 * (kRP - 1 - kTcUa));
#pragma unroll
    for (int i = 0; i < kT; i += 2) {
        uint32_t w[16];
        tmem_ld16(lane_base + 8 * i, w);
        x[i] = tc_combine(w, i == 0 ? u21 : x[i]);
        x[i + 1] = tc_combine(w + 8, x[i + 1]);
    }
    return true;
}

// The 22 partial rounds on the integer pipes, state in registers (the
// MDSPartial form of Alg. 1: 12 products for cell 0, 11 multiply-adds).
__device__ __forceinline__ void partial_regs(uint64_t (&x)[kT]) {
#pragma unroll 1
    for (int q = 0; q < kRP; ++q) {
        const uint64_t x0 = sbox(add_canon(x[0], c_dev.part_rc[q]));
        Acc A;
        acc_zero(A);
        acc_mac(A, x0, c_dev.part_v[q][0]);
#pragma unroll
        for (int j = 1; j < kT; ++j) acc_mac(A, x[j], c_dev.part_v[q][j]);
#pragma unroll
        for (int i = 1; i < kT; ++i) x[i] = mul_add(c_dev.part_w[q][i], x0, x[i]);
        x[0] = acc_reduce(A);
    }
}

// The permutation on x, the thread's state in registers (weak words in,
// weak words out), with the same zcap / digest shortcuts as permute_slot.
// Each round's twelve S-boxes and twelve output folds are unrolled (the
// state never leaves registers).  CHAIN: the partial rounds in their
// unrolled form on the tensor cores (tc_partial); else on the integer pipes
// (partial_regs).
template <bool CHAIN>
__device__ __forceinline__ bool tc_permute(TcGroup &G, uint64_t (&x)[kT], bool zcap, bool digest) {
#pragma unroll 1
    for (int r = 0; r < kRF; ++r) {
        const bool z = zcap && r == 0;
#pragma unroll
        for (int j = 0; j < kRate; ++j) tc_put(G, j, sbox(add_canon(x[j], c_dev.full_rc[r][j])));
        if (!z) {
#pragma unroll
            for (int j = kRate; j < kT; ++j) tc_put(G, j, sbox(add_canon(x[j], c_dev.full_rc[r][j])));
        }
        const bool mid = r == kRF / 2 - 1;
        if (!tc_dense(G, mid ? kTabPre : kTabM, z, digest && r == kRF - 1 ? kDigest : kT, x)) return false;
        if (mid) {
            if (CHAIN) {
                if (!tc_partial(G, x)) return false;
            } else {
                partial_regs(x);
            }
        }
    }
    return true;
}

// Shared-memory layout of a CTA of GROUPS groups: the tables (all of them
// with CHAIN, else the full rounds' part), then each group's A operand, then
// the barriers.
template <int GROUPS, bool CHAIN>
struct TcLayout {
    static_assert(GROUPS * kTcRegion <= 512, "the groups' tensor memory exceeds the SM's");
    static constexpr int kTmemCols = tc_tmem_alloc(GROUPS);
    static constexpr size_t kTableBytes = CHAIN ? sizeof(TcTables) : kTabCore;
    static constexpr size_t kTables = 0;
    static constexpr size_t kA = (kTableBytes + 127) & ~(size_t)127;
    static constexpr size_t kBar = kA + (size_t)GROUPS * kTcABytes;
    static constexpr size_t kBcast = kBar + 8 * GROUPS + 16;
    static constexpr size_t kBytes = kBcast + 4 * GROUPS;
};

__device__ int g_tc_fault;  // set when a tensor-core wait ran out (read by pg_device_faults)

// Prologue of a tensor-core kernel: tables into shared memory, the groups'
// barriers, one tensor-memory allocation for all groups.
template <int GROUPS, bool CHAIN>
__device__ __forceinline__ TcGroup tc_setup(uint8_t *sm) {
    using L = TcLayout<GROUPS, CHAIN>;
    const uint4 *src = reinterpret_cast<const uint4 *>(&g_tc);
    uint4 *dst = reinterpret_cast<uint4 *>(sm + L::kTables);
    for (unsigned i = threadIdx.x; i < L::kTableBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
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
    G.mbar = bars + g;
    G.tmem = *tslot + (uint32_t)(g * kTcRegion);
    G.phase = 0;
    G.bar = 1 + g;
    G.bcast = reinterpret_cast<volatile uint32_t *>(sm + L::kBcast) + g;
    G.a_addr = smem_addr(G.a);
    G.tab = smem_addr(sm + L::kTables);
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
template <int GROUPS, bool CHAIN>
__device__ __forceinline__ void tc_teardown(uint8_t *sm, TcGroup &G) {
    using L = TcLayout<GROUPS, CHAIN>;
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
