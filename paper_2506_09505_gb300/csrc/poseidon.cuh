// Device Poseidon-12 permutation, one thread per state (Alg. 1).
//
// The state lives in twelve 64-bit registers.  Round structure (Alg. 1,
// HALF_FULL_ROUNDS = 4, PARTIAL_ROUNDS = 22) in the optimised form whose
// constants the host derives from (C, M):
//   full rounds 0..3   : x += c_r; x = x^7 (all cells); x = M x  (round 3 uses
//                        the transition matrix instead of M)
//   partial rounds     : x_0 += k_q; x_0 = x_0^7; MDSPartial:
//                        new_0 = <v_q, x>, new_i = x_i + w_q[i-1] * x_0
//   full rounds 26..29 : x += c_r; x = x^7; x = M x
// Dense matrix rows are accumulated lazily: twelve 128-bit products summed
// in 160 bits and reduced once per output cell.
#pragma once
#include "field.cuh"
#include "pg12_internal.h"

namespace pg12 {
namespace dev {

// Constants of the optimised form (one copy per translation unit that
// includes this header; filled by pg_init via cudaMemcpyToSymbol).
__constant__ OptParams c_opt;

// y = N x for a dense 12x12 matrix held in constant memory.
__device__ __forceinline__ void dense_layer(uint64_t (&x)[kT], const uint64_t (&n)[kT][kT]) {
    uint64_t y[kT];
#pragma unroll
    for (int i = 0; i < kT; ++i) {
        Acc a;
        acc_zero(a);
#pragma unroll
        for (int j = 0; j < kT; ++j) acc_mac(a, x[j], n[i][j]);
        y[i] = acc_reduce(a);
    }
#pragma unroll
    for (int i = 0; i < kT; ++i) x[i] = y[i];
}

__device__ __forceinline__ void full_round(uint64_t (&x)[kT], const uint64_t (&rc)[kT],
                                           const uint64_t (&n)[kT][kT]) {
#pragma unroll
    for (int i = 0; i < kT; ++i) x[i] = sbox(add_canon(x[i], rc[i]));
    dense_layer(x, n);
}

__device__ __forceinline__ void partial_round(uint64_t (&x)[kT], int q) {
    const uint64_t x0 = sbox(add_canon(x[0], c_opt.part_rc[q]));
    Acc a;
    acc_zero(a);
    acc_mac(a, x0, c_opt.part_v[q][0]);
#pragma unroll
    for (int j = 1; j < kT; ++j) acc_mac(a, x[j], c_opt.part_v[q][j]);
#pragma unroll
    for (int i = 1; i < kT; ++i) {
        uint64_t lo, hi;
        mul_full(x0, c_opt.part_w[q][i - 1], lo, hi);
        // add x_i into the 128-bit product before the single reduction
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(lo), "+l"(hi) : "l"(x[i]));
        x[i] = reduce128(lo, hi);
    }
    x[0] = acc_reduce(a);
}

// y = N x for a dense matrix addressed at run time (entries fetched with
// uniform constant loads instead of constant-bank operands).
__device__ __forceinline__ void dense_layer_rt(uint64_t (&x)[kT], const uint64_t *n) {
    uint64_t y[kT];
#pragma unroll
    for (int i = 0; i < kT; ++i) {
        Acc a;
        acc_zero(a);
#pragma unroll
        for (int j = 0; j < kT; ++j) acc_mac(a, x[j], n[i * kT + j]);
        y[i] = acc_reduce(a);
    }
#pragma unroll
    for (int i = 0; i < kT; ++i) x[i] = y[i];
}

// Code shapes of the permutation (all compute the same map):
//   kShapeCbank  one loop over the 8 full rounds; the dense layer is
//                instantiated twice (M and the transition matrix) so that
//                every matrix entry is a constant-bank operand;
//   kShapeRt     one loop, one dense layer whose matrix is picked per round
//                (fewer registers, extra constant loads).
// A separate inlined copy per round group makes ptxas hoist constants
// across the copies and spill, so the rounds are always one loop.
enum PermShape { kShapeCbank = 0, kShapeRt = 1 };

template <int SHAPE = kShapeCbank>
__device__ __forceinline__ void permute(uint64_t (&x)[kT]) {
#pragma unroll 1
    for (int r = 0; r < kRF; ++r) {
#pragma unroll
        for (int i = 0; i < kT; ++i) x[i] = sbox(add_canon(x[i], c_opt.full_rc[r][i]));
        if (SHAPE == kShapeRt) {
            dense_layer_rt(x, r == kRF / 2 - 1 ? &c_opt.pre[0][0] : &c_opt.mds[0][0]);
            if (r == kRF / 2 - 1) {
#pragma unroll 1
                for (int q = 0; q < kRP; ++q) partial_round(x, q);
            }
        } else {
            if (r == kRF / 2 - 1) {
                dense_layer(x, c_opt.pre);
#pragma unroll 1
                for (int q = 0; q < kRP; ++q) partial_round(x, q);
            } else {
                dense_layer(x, c_opt.mds);
            }
        }
    }
}

}  // namespace dev
}  // namespace pg12
