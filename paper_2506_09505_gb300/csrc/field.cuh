// Device arithmetic in the Goldilocks field, Eq. 1: p = 2^64 - 2^32 + 1.
//
// Values travel between operations as 64-bit "weak" representatives: any
// word in [0, 2^64) standing for its residue mod p.  Only stored results are
// made canonical (0 <= e < p, Sec. 2.4).  Products are formed from four
// 32x32->64 partial products (IMAD.WIDE.U32) and folded with the identities
// 2^64 = 2^32 - 1 and 2^96 = -1 (mod p) -- the special-prime reduction of
// Alg. 2 and Eqs. 2-4, rewritten for 32-bit limbs so that no 64-bit
// multiply is needed.
#pragma once
#include <cstdint>

namespace pg12 {
namespace dev {

constexpr uint64_t P = 0xFFFFFFFF00000001ull;
constexpr uint64_t EPS = 0xFFFFFFFFull;  // 2^64 mod p

__device__ __forceinline__ uint32_t lo32(uint64_t x) { return (uint32_t)x; }
__device__ __forceinline__ uint32_t hi32(uint64_t x) { return (uint32_t)(x >> 32); }

// Full 128-bit product a*b = (hi, lo) from four IMAD.WIDE.U32.
__device__ __forceinline__ void mul_full(uint64_t a, uint64_t b, uint64_t &lo, uint64_t &hi) {
    const uint32_t a0 = lo32(a), a1 = hi32(a), b0 = lo32(b), b1 = hi32(b);
    const uint64_t ll = (uint64_t)a0 * b0;
    const uint64_t lh = (uint64_t)a0 * b1 + (ll >> 32);       // < 2^64
    const uint64_t hl = (uint64_t)a1 * b0 + (uint64_t)lo32(lh); // < 2^64
    hi = (uint64_t)a1 * b1 + (lh >> 32) + (hl >> 32);          // < 2^64
    lo = (hl << 32) | (uint64_t)lo32(ll);
}

// a^2 from three partial products (the cross term is doubled).
__device__ __forceinline__ void sqr_full(uint64_t a, uint64_t &lo, uint64_t &hi) {
    const uint32_t a0 = lo32(a), a1 = hi32(a);
    const uint64_t ll = (uint64_t)a0 * a0;
    const uint64_t lh = (uint64_t)a0 * a1;
    const uint64_t mid1 = lh + (ll >> 32);  // < 2^64
    const uint64_t mid = mid1 + lh;         // 65-bit sum: keep the carry
    const uint64_t carry = (mid < lh) ? (1ull << 32) : 0ull;
    hi = (uint64_t)a1 * a1 + (mid >> 32) + carry;
    lo = (mid << 32) | (uint64_t)lo32(ll);
}

// 128-bit (hi, lo) -> weak 64-bit residue.
// With hi = hh*2^32 + hl:  value = lo - hh + hl*(2^32 - 1)  (mod p).
// A borrow out of lo - hh is worth -2^64 = -(2^32 - 1); a carry out of the
// final sum is worth +(2^32 - 1); neither correction can wrap again.
__device__ __forceinline__ uint64_t reduce128(uint64_t lo, uint64_t hi) {
    const uint64_t hh = hi >> 32;
    const uint64_t hl = hi & EPS;
    uint64_t t0 = lo - hh;
    if (lo < hh) t0 -= EPS;
    const uint64_t t1 = (hl << 32) - hl;
    uint64_t r = t0 + t1;
    if (r < t1) r += EPS;
    return r;
}

__device__ __forceinline__ uint64_t canon(uint64_t x) { return x >= P ? x - P : x; }

__device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) {
    uint64_t lo, hi;
    mul_full(a, b, lo, hi);
    return reduce128(lo, hi);
}

__device__ __forceinline__ uint64_t sqr(uint64_t a) {
    uint64_t lo, hi;
    sqr_full(a, lo, hi);
    return reduce128(lo, hi);
}

// weak a + canonical c (c < p): at most one wrap, folded as +(2^32 - 1).
__device__ __forceinline__ uint64_t add_canon(uint64_t a, uint64_t c) {
    uint64_t s = a + c;
    if (s < c) s += EPS;
    return s;
}

// S-box of Alg. 1: x^7 = (x^2)^2 * (x^2 * x).
__device__ __forceinline__ uint64_t sbox(uint64_t x) {
    const uint64_t x2 = sqr(x);
    const uint64_t x3 = mul(x2, x);
    const uint64_t x4 = sqr(x2);
    return mul(x4, x3);
}

// 160-bit accumulator for lazily reduced dot products: sum of up to 2^32
// 128-bit products.
struct Acc {
    uint64_t lo, hi;
    uint32_t top;
};

__device__ __forceinline__ void acc_zero(Acc &a) { a.lo = 0; a.hi = 0; a.top = 0; }

__device__ __forceinline__ void acc_add128(Acc &a, uint64_t plo, uint64_t phi) {
    asm volatile("add.cc.u64 %0, %0, %3;\n\t"
        "addc.cc.u64 %1, %1, %4;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+l"(a.lo), "+l"(a.hi), "+r"(a.top)
        : "l"(plo), "l"(phi));
}

__device__ __forceinline__ void acc_mac(Acc &a, uint64_t x, uint64_t m) {
    uint64_t plo, phi;
    mul_full(x, m, plo, phi);
    acc_add128(a, plo, phi);
}

// 160-bit -> weak 64-bit: top * 2^128 = -top * 2^32 (mod p) since 2^96 = -1.
__device__ __forceinline__ uint64_t acc_reduce(const Acc &a) {
    const uint64_t r = reduce128(a.lo, a.hi);
    const uint64_t t = (uint64_t)a.top << 32;
    uint64_t u = r - t;
    if (r < t) u -= EPS;  // the wrap added 2^64 = 2^32 - 1
    return u;
}

}  // namespace dev
}  // namespace pg12
