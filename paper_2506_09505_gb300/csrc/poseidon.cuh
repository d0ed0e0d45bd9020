// Device Poseidon-12 permutation, one thread per state (Alg. 1).
//
// Round structure (Alg. 1, HALF_FULL_ROUNDS = 4, PARTIAL_ROUNDS = 22) in the
// optimised form whose constants the host derives from (C, M):
//   full rounds 0..3   : x += c_r; x = x^7 (all cells); x = M x  (round 3 uses
//                        the transition matrix instead of M)
//   partial rounds     : x_0 += k_q; x_0 = x_0^7; MDSPartial:
//                        new_0 = <v_q, x>, new_i = x_i + w_q[i-1] * x_0
//   full rounds 26..29 : x += c_r; x = x^7; x = M x
//
// Code shape.  The fully unrolled permutation is ~100 KB of SASS; when the
// warps of an SM sit in different rounds it no longer fits the instruction
// caches.  So every phase is a short loop: the twelve state words live in
// the thread's own shared-memory slot (element i at slot[i * STRIDE], so a
// warp's accesses are consecutive words) between phases, the S-box phase
// walks the slot two cells at a time, and the dense phase keeps the twelve
// inputs in registers while it loops over output rows, fetching each row's
// constants with uniform loads and storing each output straight back to
// the slot.  Dense rows are accumulated lazily (twelve 128-bit products,
// one reduction per output cell).  Where the caller knows more about the
// state (its capacity cells enter as zero, or only the digest cells of the
// result are read) the first and last rounds skip the work that knowledge
// makes constant or unused (permute_slot).
#pragma once
#include "field.cuh"
#include "pg12_internal.h"

namespace pg12 {
namespace dev {

// Device copy of the optimised constants, laid out for uniform loads.
struct DevConsts {
    uint64_t full_rc[kRF][kT];
    uint64_t mat[2][kT][kT];  // [0] = M, [1] = transition matrix of round 3
    uint64_t part_rc[kRP];
    uint64_t part_v[kRP][kT];
    uint64_t part_w[kRP][kT];  // entry 0 unused (keeps rows 16-byte aligned)
    uint32_t small_mat[kT][kT];  // M again when its entries fit 8 bits
    uint32_t small;              // 1: full rounds other than round 3 use small_mat
    uint32_t pad[3];
    // Round 0 of a state whose capacity cells 8..11 enter as zero (every
    // node compression, the first chunk of every sponge): those cells become
    // the constants (c_0[j])^7, so their share of row i of M is the constant
    // zcap_k[i] = sum_{j >= 8} M_ij (c_0[j])^7.
    uint64_t zcap_k[kT];
};

// One copy per translation unit that includes this header; filled by
// upload_constants() via cudaMemcpyToSymbol.
__constant__ __align__(16) DevConsts c_dev;

inline void make_dev_consts(const OptParams &op, DevConsts &dc) {
    bool small = true;
    for (int i = 0; i < kT; ++i)
        for (int j = 0; j < kT; ++j) {
            small = small && op.mds[i][j] < 256;
            dc.small_mat[i][j] = (uint32_t)(op.mds[i][j] & 0xFFu);
        }
    dc.small = small ? 1u : 0u;
    dc.pad[0] = dc.pad[1] = dc.pad[2] = 0;
    for (int r = 0; r < kRF; ++r)
        for (int i = 0; i < kT; ++i) dc.full_rc[r][i] = op.full_rc[r][i];
    for (int i = 0; i < kT; ++i)
        for (int j = 0; j < kT; ++j) {
            dc.mat[0][i][j] = op.mds[i][j];
            dc.mat[1][i][j] = op.pre[i][j];
        }
    const auto mulmod = [](uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) % P); };
    for (int i = 0; i < kT; ++i) {
        uint64_t k = 0;
        for (int j = kRate; j < kT; ++j) {
            const uint64_t c = op.full_rc[0][j] % P;
            const uint64_t c2 = mulmod(c, c), c4 = mulmod(c2, c2), c7 = mulmod(mulmod(c4, c2), c);
            k = (uint64_t)(((unsigned __int128)k + mulmod(op.mds[i][j] % P, c7)) % P);
        }
        dc.zcap_k[i] = k;
    }
    for (int q = 0; q < kRP; ++q) {
        dc.part_rc[q] = op.part_rc[q];
        for (int j = 0; j < kT; ++j) dc.part_v[q][j] = op.part_v[q][j];
        dc.part_w[q][0] = 0;
        for (int i = 1; i < kT; ++i) dc.part_w[q][i] = op.part_w[q][i - 1];
    }
}

// Cells 0 .. cells-1 of round r: constant, then the S-box, PG12_SBOX_CELLS
// cells per loop iteration (independent chains in flight).
#ifndef PG12_SBOX_CELLS
#define PG12_SBOX_CELLS 2  // 2 or 4 (both divide 8 and 12); 4 measured the same (14.81 ms a tree)
#endif
template <int S>
__device__ __forceinline__ void sbox_phase(uint64_t *slot, int r, int cells) {
#pragma unroll 1
    for (int i = 0; i < cells; i += PG12_SBOX_CELLS) {
        uint64_t a[PG12_SBOX_CELLS];
#pragma unroll
        for (int k = 0; k < PG12_SBOX_CELLS; ++k) a[k] = add_canon(slot[(i + k) * S], c_dev.full_rc[r][i + k]);
#pragma unroll
        for (int k = 0; k < PG12_SBOX_CELLS; ++k) slot[(i + k) * S] = sbox(a[k]);
    }
}

#ifndef PG12_DENSE_ROWS
#define PG12_DENSE_ROWS 1  // output rows per iteration of the dense loop (1 or 2)
#endif

// Dense layer x = mat[m] x over the first NT cells of the slot; with
// NT = kRate (round 0, capacity cells entered as zero) each row starts from
// zcap_k instead of the products of cells 8..11.
template <int S, int NT = kT>
__device__ __forceinline__ void dense_phase(uint64_t *slot, int m, int rows = kT) {
    uint64_t x[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) x[j] = slot[j * S];
#pragma unroll 1
    for (int i = 0; i < rows; i += PG12_DENSE_ROWS) {
        Acc A[PG12_DENSE_ROWS];
#pragma unroll
        for (int k = 0; k < PG12_DENSE_ROWS; ++k) {
            if (NT < kT) acc_init(A[k], c_dev.zcap_k[i + k]);
            else acc_zero(A[k]);
        }
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int k = 0; k < PG12_DENSE_ROWS; ++k) acc_mac(A[k], x[j], c_dev.mat[m][i + k][j]);
#pragma unroll
        for (int k = 0; k < PG12_DENSE_ROWS; ++k) slot[(i + k) * S] = acc_reduce(A[k]);
    }
}

// Dense layer of an MDS matrix with 8-bit entries (Table 1's mmult_4x12_8):
// x_j * m for m < 2^8 is two 32x8-bit products; twelve of them fit 64 bits,
// so both halves accumulate through the IMAD.WIDE addend with no carries and
// one fold per output.

template <int S, int NT = kT>
__device__ __forceinline__ void dense_small_phase(uint64_t *slot, int rows = kT) {
    uint64_t x[NT];
#pragma unroll
    for (int j = 0; j < NT; ++j) x[j] = slot[j * S];
#pragma unroll 1
    for (int i = 0; i < rows; ++i) {
        uint64_t lo = 0, hi = 0;  // sums of x_j.lo * m_ij and x_j.hi * m_ij (< 2^44 each)
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const uint32_t m = c_dev.small_mat[i][j];
            lo = madw(lo32(x[j]), m, lo);
            hi = madw(hi32(x[j]), m, hi);
        }
        // value = lo + hi * 2^32 (+ zcap_k[i] < p) < 2^78
        u128 v = (u128)lo + ((u128)hi << 32);
        if (NT < kT) v += c_dev.zcap_k[i];
        slot[i * S] = reduce128(v);
    }
}

// 1 (default): partial rounds walk cells 1..11 in the slot, one cell per
// loop iteration; 0: the eleven cells stay in registers, fully unrolled.
// The loop form executes about 2% more instructions but its code is a
// fraction of the size, and with a dozen warps per SM in different phases
// the unrolled form stalls on instruction fetch (measured: 2^22 x 8 tree
// 17.8 ms against 19.1 ms).
#ifndef PG12_PARTIAL_LOOP
#define PG12_PARTIAL_LOOP 1
#endif
// In the loop form: 1 (default) walks the cells two per iteration after
// cell 1 (two independent products in flight; with PG12_MERKLE_MIN_BLOCKS=4 a
// 2^22 x 8 tree 15.86 ms against 15.98 ms one cell per iteration).
#ifndef PG12_PARTIAL_PAIRS
#define PG12_PARTIAL_PAIRS 1
#endif

// In the pairs form: 1 sums the dot product's even and odd cells in two
// accumulators (two independent carry chains), joined before the one
// reduction; 0 (default): one accumulator.
#ifndef PG12_PARTIAL_ACC2
#define PG12_PARTIAL_ACC2 0
#endif

// Sum of two lazy accumulators (A += B), each below 2^150.
__device__ __forceinline__ void acc_join(Acc &A, const Acc &B) {
    asm("add.cc.u32 %0, %0, %5;\n\t"
        "addc.cc.u32 %1, %1, %6;\n\t"
        "addc.cc.u32 %2, %2, %7;\n\t"
        "addc.cc.u32 %3, %3, %8;\n\t"
        "addc.u32 %4, %4, %9;"
        : "+r"(A.a0), "+r"(A.a1), "+r"(A.a2), "+r"(A.a3), "+r"(A.a4)
        : "r"(B.a0), "r"(B.a1), "r"(B.a2), "r"(B.a3), "r"(B.a4));
#if PG12_ACC_MID64
    A.mlo += B.mlo;
    A.mhi += B.mhi;
#else
    asm("add.cc.u32 %0, %0, %3;\n\t"
        "addc.cc.u32 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, %5;"
        : "+r"(A.m0), "+r"(A.m1), "+r"(A.m2)
        : "r"(B.m0), "r"(B.m1), "r"(B.m2));
#endif
}

template <int S, int LOOP = PG12_PARTIAL_LOOP>
__device__ __forceinline__ void partial_phase(uint64_t *slot) {
    if (LOOP) {
        // Cells 1..11 stay in the slot; each round walks them once, so the loop
        // body is one cell's product and update instead of all eleven.
#pragma unroll 1
        for (int q = 0; q < kRP; ++q) {
            const uint64_t x0 = sbox(add_canon(slot[0], c_dev.part_rc[q]));
            Acc A;
            acc_zero(A);
            acc_mac(A, x0, c_dev.part_v[q][0]);
#if PG12_PARTIAL_PAIRS
            // cell 1, then cells (2,3) ... (10,11) two per iteration
            {
                const uint64_t x1 = slot[S];
                acc_mac(A, x1, c_dev.part_v[q][1]);
                slot[S] = mul_add(c_dev.part_w[q][1], x0, x1);
            }
#if PG12_PARTIAL_ACC2
            Acc B;
            acc_zero(B);
#pragma unroll 1
            for (int j = 2; j < kT; j += 2) {
                const uint64_t xa = slot[j * S], xb = slot[(j + 1) * S];
                acc_mac(A, xa, c_dev.part_v[q][j]);
                acc_mac(B, xb, c_dev.part_v[q][j + 1]);
                slot[j * S] = mul_add(c_dev.part_w[q][j], x0, xa);
                slot[(j + 1) * S] = mul_add(c_dev.part_w[q][j + 1], x0, xb);
            }
            acc_join(A, B);
#else
#pragma unroll 1
            for (int j = 2; j < kT; j += 2) {
                const uint64_t xa = slot[j * S], xb = slot[(j + 1) * S];
                acc_mac(A, xa, c_dev.part_v[q][j]);
                acc_mac(A, xb, c_dev.part_v[q][j + 1]);
                slot[j * S] = mul_add(c_dev.part_w[q][j], x0, xa);
                slot[(j + 1) * S] = mul_add(c_dev.part_w[q][j + 1], x0, xb);
            }
#endif
#else
#pragma unroll 1
            for (int j = 1; j < kT; ++j) {
                const uint64_t xj = slot[j * S];
                acc_mac(A, xj, c_dev.part_v[q][j]);
                slot[j * S] = mul_add(c_dev.part_w[q][j], x0, xj);
            }
#endif
            slot[0] = acc_reduce(A);
        }
    } else {
        uint64_t x[kT];
#pragma unroll
        for (int j = 0; j < kT; ++j) x[j] = slot[j * S];
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
#pragma unroll
        for (int j = 0; j < kT; ++j) slot[j * S] = x[j];
    }
}

// Matrix kinds the kernels are compiled for: the full-width Cauchy matrix
// of pg12_v1 and the 8-bit circulant of pg12_small (chosen on the host from
// the active parameter set, so each kernel carries only its own code).
enum MdsKind { kMdsFull = 0, kMdsSmall = 1 };

// The permutation on the state in `slot` (weak words in, weak words out).
// zcap: cells 8..11 hold zero (a node compression or a sponge's first
// chunk); round 0 then skips their S-boxes and products (zcap_k), which is
// the same function with 4 of 118 S-boxes and 48 of 1,416 dense products
// fewer.  digest: only cells 0..3 of the result are read (a node, or a
// sponge's last chunk); the last dense layer then computes rows 0..3 only
// (96 products fewer) and leaves cells 4..11 holding S-box outputs.
#ifndef PG12_ZCAP
#define PG12_ZCAP 1  // 0: every permutation takes the general round 0
#endif
#ifndef PG12_DIGEST_ROWS
#define PG12_DIGEST_ROWS 1  // 0: the last dense layer always computes all rows
#endif
template <int S, int MDS = kMdsFull>
__device__ __forceinline__ void permute_slot(uint64_t *slot, bool zcap = false, bool digest = false) {
#pragma unroll 1
    for (int r = 0; r < kRF; ++r) {
        const bool z = PG12_ZCAP && zcap && r == 0;
        const int rows = PG12_DIGEST_ROWS && digest && r == kRF - 1 ? kDigest : kT;
        sbox_phase<S>(slot, r, z ? kRate : kT);
        if (z) {
            if (MDS == kMdsSmall) dense_small_phase<S, kRate>(slot);
            else dense_phase<S, kRate>(slot, 0);
        } else if (MDS == kMdsSmall && r != kRF / 2 - 1) {
            dense_small_phase<S>(slot, rows);
        } else {
            dense_phase<S>(slot, r == kRF / 2 - 1 ? 1 : 0, rows);
        }
        if (r == kRF / 2 - 1) partial_phase<S>(slot);
    }
}


// ------------------------------------------------------------ wide form
// Sixteen lanes share one state: lane e < 12 holds cell x_e (lanes 12..15
// carry zeros).  Used where few permutations are in flight (the top levels
// of a tree), because its latency is about a tenth of the one-thread form.
// Lanes index the constants by their own cell, so the kernels stage a copy
// of the tables in shared memory (load_consts) and pass it in as K.
__device__ __align__(16) DevConsts g_dev;
static_assert(sizeof(DevConsts) % 16 == 0, "constant tables are copied in 16-byte pieces");

// Block-wide copy of the constant tables into shared memory (16-byte loads).
__device__ __forceinline__ void load_consts(DevConsts &dst) {
    const uint4 *src = reinterpret_cast<const uint4 *>(&g_dev);
    uint4 *d = reinterpret_cast<uint4 *>(&dst);
    for (unsigned i = threadIdx.x; i < sizeof(DevConsts) / sizeof(uint4); i += blockDim.x) d[i] = __ldg(src + i);
    __syncthreads();
}

__device__ __forceinline__ uint64_t add_weak(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    if (s < b) {
        s += EPS;
        if (s < EPS) s += EPS;  // second wrap (only when both inputs are >= p)
    }
    return s;
}

// `lane16` = lane index within its 16-lane group, `gmask` = the warp's active
// mask; every lane of the group must execute this.  Latency is what matters
// here, so the critical path is kept short: in a partial round the products
// v_e x_e (e >= 1) and their butterfly sum do not wait for the S-box; only
// v_0 x_0^7 is added after it.  Dense rows use two accumulators.  There are
// no lane-dependent branches (a divergent warp would run the two sides one
// after the other): every lane computes and operands are selected.  Lanes 12
// to 15 carry values nobody reads (dense rows gather lanes 0-11, x_0 comes
// from lane 0, and their products are masked out of the sum).
__device__ __forceinline__ uint64_t permute_wide(uint64_t x, int lane16, unsigned gmask, const DevConsts &K) {
    const int e = lane16 < kT ? lane16 : 0;
    const uint64_t pmask = (lane16 >= 1 && lane16 < kT) ? ~0ull : 0ull;
    const bool lane0 = lane16 == 0;
    const int base = (threadIdx.x & 31) & ~15;
#pragma unroll 1
    for (int r = 0; r < kRF; ++r) {
        x = sbox(add_canon(x, K.full_rc[r][e]));
        const int m = r == kRF / 2 - 1 ? 1 : 0;
        Acc A, B;
        acc_zero(A);
        acc_zero(B);
#pragma unroll
        for (int j = 0; j < kT; j += 2) {
            const uint64_t xa = __shfl_sync(gmask, x, base + j);
            const uint64_t xb = __shfl_sync(gmask, x, base + j + 1);
            acc_mac(A, xa, K.mat[m][e][j]);
            acc_mac(B, xb, K.mat[m][e][j + 1]);
        }
        x = add_weak(acc_reduce(A), acc_reduce(B));
        if (r == kRF / 2 - 1) {
#pragma unroll 1
            for (int q = 0; q < kRP; ++q) {
                const uint64_t x0 = __shfl_sync(gmask, x, base);
                const uint64_t y = sbox(add_canon(x0, K.part_rc[q]));
                // sum of v_e x_e over e = 1..11 (independent of the S-box)
                uint64_t t = mul(x, K.part_v[q][e]) & pmask;
#pragma unroll
                for (int d = 8; d >= 1; d >>= 1) t = add_weak(t, __shfl_xor_sync(gmask, t, d));
                // lane 0: v_0 y + t; lane e: x_e + w_e y
                const uint64_t coef = lane0 ? K.part_v[q][0] : K.part_w[q][e];
                x = mul_add(coef, y, lane0 ? t : x);
            }
        }
    }
    return x;
}

}  // namespace dev
}  // namespace pg12
