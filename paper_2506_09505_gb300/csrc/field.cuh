// Device arithmetic in the Goldilocks field, Eq. 1: p = 2^64 - 2^32 + 1.
//
// Values travel between operations as 64-bit "weak" representatives: any
// word in [0, 2^64) standing for its residue mod p.  Only stored results are
// made canonical (0 <= e < p, Sec. 2.4).  Products are formed from four
// 32x32->64 partial products (IMAD.WIDE.U32 with a zero addend, so no
// register pair has to be built for the addend) and summed column by column
// in carry chains.  The 128-bit (or 160-bit) result is folded with
// 2^64 = 2^32 - 1, 2^96 = -1 and 2^128 = -2^32 (mod p): the special-prime
// reduction of Alg. 2 and Eqs. 2-4 on 32-bit limbs, with no 64-bit multiply.
#pragma once
#include <cstdint>

namespace pg12 {
namespace dev {

constexpr uint64_t P = 0xFFFFFFFF00000001ull;
constexpr uint64_t EPS = 0xFFFFFFFFull;  // 2^64 mod p

typedef unsigned __int128 u128;
typedef __int128 s128;

__device__ __forceinline__ uint32_t lo32(uint64_t x) { return (uint32_t)x; }
__device__ __forceinline__ uint32_t hi32(uint64_t x) { return (uint32_t)(x >> 32); }

// The four partial products of a*b (each < 2^64).
struct Partial {
    uint64_t ll, lh, hl, hh;
};

__device__ __forceinline__ Partial partials(uint64_t a, uint64_t b) {
    const uint32_t a0 = lo32(a), a1 = hi32(a), b0 = lo32(b), b1 = hi32(b);
    Partial q;
    q.ll = (uint64_t)a0 * b0;
    q.lh = (uint64_t)a0 * b1;
    q.hl = (uint64_t)a1 * b0;
    q.hh = (uint64_t)a1 * b1;
    return q;
}

// (r3:r2:r1:r0) = ll + (lh + hl) * 2^32 + hh * 2^64, two carry chains.
// (Running the second chain as multiply-adds by a 1 held in constant memory,
// to move its adds from the ALU pipe to the FMA pipe, measured 1% slower.)
__device__ __forceinline__ u128 join(const Partial &q) {
    uint32_t r0 = lo32(q.ll), r1, r2, r3;
    asm("add.cc.u32 %0, %3, %4;\n\t"
        "addc.cc.u32 %1, %5, %6;\n\t"
        "addc.u32 %2, %7, 0;\n\t"
        "add.cc.u32 %0, %0, %8;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.u32 %2, %2, 0;"
        : "=r"(r1), "=r"(r2), "=r"(r3)
        : "r"(hi32(q.ll)), "r"(lo32(q.lh)), "r"(hi32(q.lh)), "r"(lo32(q.hh)), "r"(hi32(q.hh)),
          "r"(lo32(q.hl)), "r"(hi32(q.hl)));
    return ((u128)(((uint64_t)r3 << 32) | r2) << 64) | (((uint64_t)r1 << 32) | r0);
}

// a^2 = ll + 2 lh 2^32 + hh 2^64 from three partial products.
__device__ __forceinline__ u128 sqr_full(uint64_t a) {
    const uint32_t a0 = lo32(a), a1 = hi32(a);
    const uint64_t ll = (uint64_t)a0 * a0, lh = (uint64_t)a0 * a1, hh = (uint64_t)a1 * a1;
    uint32_t r1, r2, r3;
    asm("add.cc.u32 %0, %3, %4;\n\t"
        "addc.cc.u32 %1, %5, %6;\n\t"
        "addc.u32 %2, %7, 0;\n\t"
        "add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.u32 %2, %2, 0;"
        : "=r"(r1), "=r"(r2), "=r"(r3)
        : "r"(hi32(ll)), "r"(lo32(lh)), "r"(hi32(lh)), "r"(lo32(hh)), "r"(hi32(hh)));
    return ((u128)(((uint64_t)r3 << 32) | r2) << 64) | (((uint64_t)r1 << 32) | lo32(ll));
}

// value = lo + hl 2^32 - hl - hh - k 2^32 (mod p) for hi = hh:hl and a small
// extra k (the 2^128 limb of a lazy sum, 2^128 = -2^32).  The exact signed
// value t lies in (-(k + 2) 2^32, 2^65 - 2^33]; its top word tp is -1, 0 or 1
// and is folded back as tp (2^32 - 1) (2^64 = 2^32 - 1).  That add cannot wrap
// again: for tp = 1 the low word is at most 2^64 - 2^33, for tp = -1 at least
// 2^64 - (k + 2) 2^32.
//
// 1 (default): the words of t come from one borrow/carry chain on 32-bit
// limbs; 0: the same value through signed 128-bit C arithmetic (measured: a
// 2^22 x 8 tree 3% slower, S-box 10% slower).
#ifndef PG12_FOLD_PTX
#define PG12_FOLD_PTX 1
#endif
__device__ __forceinline__ uint64_t fold(uint64_t lo, uint64_t hi, uint32_t k) {
#if PG12_FOLD_PTX
    // t = l0 + (l1 + hl - k) 2^32 - hl - hh as a 96-bit two's-complement value (w0, w1, tp)
    uint32_t w0, w1, tp;
    asm("sub.cc.u32 %0, %3, %5;\n\t"
        "subc.cc.u32 %1, %4, %7;\n\t"
        "subc.u32 %2, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, %6;\n\t"
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.u32 %2, %2, 0;\n\t"
        "add.cc.u32 %1, %1, %5;\n\t"
        "addc.u32 %2, %2, 0;"
        : "=r"(w0), "=r"(w1), "=r"(tp)
        : "r"(lo32(lo)), "r"(hi32(lo)), "r"(lo32(hi)), "r"(hi32(hi)), "r"(k));
    // + tp (2^32 - 1): minus tp sign-extended, plus tp at 2^32 (the same
    // correction as 64-bit C arithmetic on the sign-extended tp measured 2%
    // slower in the tensor-core kernels)
    uint32_t r0, r1;
    asm("{\n\t.reg .u32 sh;\n\t"
        "shr.s32 sh, %4, 31;\n\t"
        "sub.cc.u32 %0, %2, %4;\n\t"
        "subc.u32 %1, %3, sh;\n\t"
        "add.u32 %1, %1, %4;\n\t}"
        : "=r"(r0), "=r"(r1)
        : "r"(w0), "r"(w1), "r"(tp));
    return ((uint64_t)r1 << 32) | r0;
#else
    const uint64_t hl = hi & EPS, hh = hi >> 32;
    const s128 t = (s128)lo + (s128)(hl << 32) - (s128)(hl + hh) - (s128)((uint64_t)k << 32);
    const uint64_t top = (uint64_t)(t >> 64);
    return (uint64_t)t + ((top << 32) - top);
#endif
}

__device__ __forceinline__ uint64_t reduce128(u128 r) { return fold((uint64_t)r, (uint64_t)(r >> 64), 0); }

// a * b + c for 32-bit a, b and a 64-bit c (one IMAD.WIDE; the caller keeps
// the sum below 2^64)
__device__ __forceinline__ uint64_t madw(uint32_t a, uint32_t b, uint64_t c) {
    uint64_t d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

__device__ __forceinline__ uint64_t canon(uint64_t x) { return x >= P ? x - P : x; }

// (Summing the columns inside chained 32x32+64-bit multiply-adds instead of
// carry chains measured 0.5% slower in the tensor-core kernels.)
__device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) { return reduce128(join(partials(a, b))); }

__device__ __forceinline__ uint64_t sqr(uint64_t a) { return reduce128(sqr_full(a)); }

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

// x + w*y as one 128-bit value (x added into the product), reduced once.
__device__ __forceinline__ uint64_t mul_add(uint64_t w, uint64_t y, uint64_t x) {
    u128 r = join(partials(w, y));
    r += x;  // < 2^128: the product is below p * 2^64
    return reduce128(r);
}

// Lazy dot-product accumulator.  The outer partial products (ll, hh) of a
// term are one contiguous 128-bit value and go into a 160-bit sum; the two
// middle products go into a separate sum that is shifted in once at the end.
// Holds up to 2^30 terms.
#ifndef PG12_ACC_MID64
#define PG12_ACC_MID64 1  // 0: middle products in a 96-bit carry chain (measured 2% slower)
#endif
struct Acc {
    uint32_t a0, a1, a2, a3, a4;
#if PG12_ACC_MID64
    uint64_t mlo, mhi;  // sums of the low / high halves of lh and hl (weights 2^32, 2^64)
#else
    uint32_t m0, m1, m2;
#endif
};

__device__ __forceinline__ void acc_zero(Acc &A) {
    A.a0 = A.a1 = A.a2 = A.a3 = A.a4 = 0;
#if PG12_ACC_MID64
    A.mlo = A.mhi = 0;
#else
    A.m0 = A.m1 = A.m2 = 0;
#endif
}

// Sum that starts from one 64-bit value v (as if a first term were v * 1).
__device__ __forceinline__ void acc_init(Acc &A, uint64_t v) {
    acc_zero(A);
    A.a0 = lo32(v);
    A.a1 = hi32(v);
}

__device__ __forceinline__ void acc_mac(Acc &A, uint64_t x, uint64_t m) {
    const Partial q = partials(x, m);
#if PG12_ACC_MID64
    asm("add.cc.u32 %0, %0, %5;\n\t"
        "addc.cc.u32 %1, %1, %6;\n\t"
        "addc.cc.u32 %2, %2, %7;\n\t"
        "addc.cc.u32 %3, %3, %8;\n\t"
        "addc.u32 %4, %4, 0;"
        : "+r"(A.a0), "+r"(A.a1), "+r"(A.a2), "+r"(A.a3), "+r"(A.a4)
        : "r"(lo32(q.ll)), "r"(hi32(q.ll)), "r"(lo32(q.hh)), "r"(hi32(q.hh)));
    // three-input adds into 64-bit words: no carry leaves them
    A.mlo += (uint64_t)lo32(q.lh) + lo32(q.hl);
    A.mhi += (uint64_t)hi32(q.lh) + hi32(q.hl);
#else
    asm("add.cc.u32 %0, %0, %8;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.cc.u32 %2, %2, %10;\n\t"
        "addc.cc.u32 %3, %3, %11;\n\t"
        "addc.u32 %4, %4, 0;\n\t"
        "add.cc.u32 %5, %5, %12;\n\t"
        "addc.cc.u32 %6, %6, %13;\n\t"
        "addc.u32 %7, %7, 0;\n\t"
        "add.cc.u32 %5, %5, %14;\n\t"
        "addc.cc.u32 %6, %6, %15;\n\t"
        "addc.u32 %7, %7, 0;"
        : "+r"(A.a0), "+r"(A.a1), "+r"(A.a2), "+r"(A.a3), "+r"(A.a4), "+r"(A.m0), "+r"(A.m1), "+r"(A.m2)
        : "r"(lo32(q.ll)), "r"(hi32(q.ll)), "r"(lo32(q.hh)), "r"(hi32(q.hh)), "r"(lo32(q.lh)),
          "r"(hi32(q.lh)), "r"(lo32(q.hl)), "r"(hi32(q.hl)));
#endif
}

// sum -> weak 64-bit residue.
__device__ __forceinline__ uint64_t acc_reduce(const Acc &A) {
#if PG12_ACC_MID64
    // middle sum = mlo + mhi 2^32 (each half-sum is below 2^33 per term, so the
    // sum stays below 2^96), as three words m0..m2 at weight 2^32
    const u128 mid = (u128)A.mlo + ((u128)A.mhi << 32);
    const uint32_t m0 = (uint32_t)mid, m1 = (uint32_t)(mid >> 32), m2 = (uint32_t)(mid >> 64);
#else
    const uint32_t m0 = A.m0, m1 = A.m1, m2 = A.m2;
#endif
    uint32_t a1, a2, a3, a4;
    asm("add.cc.u32 %0, %4, %8;\n\t"
        "addc.cc.u32 %1, %5, %9;\n\t"
        "addc.cc.u32 %2, %6, %10;\n\t"
        "addc.u32 %3, %7, 0;"
        : "=r"(a1), "=r"(a2), "=r"(a3), "=r"(a4)
        : "r"(A.a1), "r"(A.a2), "r"(A.a3), "r"(A.a4), "r"(m0), "r"(m1), "r"(m2));
    return fold(((uint64_t)a1 << 32) | A.a0, ((uint64_t)a3 << 32) | a2, a4);
}

}  // namespace dev
}  // namespace pg12
