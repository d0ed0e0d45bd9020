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
// one reduction per output cell).
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
};

// One copy per translation unit that includes this header; filled by
// upload_constants() via cudaMemcpyToSymbol.
__constant__ __align__(16) DevConsts c_dev;

inline void make_dev_consts(const OptParams &op, DevConsts &dc) {
    for (int r = 0; r < kRF; ++r)
        for (int i = 0; i < kT; ++i) dc.full_rc[r][i] = op.full_rc[r][i];
    for (int i = 0; i < kT; ++i)
        for (int j = 0; j < kT; ++j) {
            dc.mat[0][i][j] = op.mds[i][j];
            dc.mat[1][i][j] = op.pre[i][j];
        }
    for (int q = 0; q < kRP; ++q) {
        dc.part_rc[q] = op.part_rc[q];
        for (int j = 0; j < kT; ++j) dc.part_v[q][j] = op.part_v[q][j];
        dc.part_w[q][0] = 0;
        for (int i = 1; i < kT; ++i) dc.part_w[q][i] = op.part_w[q][i - 1];
    }
}

template <int S>
__device__ __forceinline__ void sbox_phase(uint64_t *slot, int r) {
#pragma unroll 1
    for (int i = 0; i < kT; i += 2) {
        const uint64_t a = add_canon(slot[i * S], c_dev.full_rc[r][i]);
        const uint64_t b = add_canon(slot[(i + 1) * S], c_dev.full_rc[r][i + 1]);
        slot[i * S] = sbox(a);
        slot[(i + 1) * S] = sbox(b);
    }
}

template <int S>
__device__ __forceinline__ void dense_phase(uint64_t *slot, int m) {
    uint64_t x[kT];
#pragma unroll
    for (int j = 0; j < kT; ++j) x[j] = slot[j * S];
#pragma unroll 1
    for (int i = 0; i < kT; ++i) {
        Acc A;
        acc_zero(A);
#pragma unroll
        for (int j = 0; j < kT; ++j) acc_mac(A, x[j], c_dev.mat[m][i][j]);
        slot[i * S] = acc_reduce(A);
    }
}

template <int S>
__device__ __forceinline__ void partial_phase(uint64_t *slot) {
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

// The permutation on the state in `slot` (weak words in, weak words out).
template <int S>
__device__ __forceinline__ void permute_slot(uint64_t *slot) {
#pragma unroll 1
    for (int r = 0; r < kRF; ++r) {
        sbox_phase<S>(slot, r);
        dense_phase<S>(slot, r == kRF / 2 - 1 ? 1 : 0);
        if (r == kRF / 2 - 1) partial_phase<S>(slot);
    }
}

}  // namespace dev
}  // namespace pg12
