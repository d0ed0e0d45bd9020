// Goldilocks number-theoretic transform and low-degree extension of
// row-major column data: the NTT hotspot Sec. 2.3 names next to Merkle
// building, in its textbook form (the paper does not define it):
//   pg_ntt  X_i = sum_j x_j w^(ij) for every column, w = 7^((p-1)/n) (7
//           generates the multiplicative group); the inverse uses w^-1 and
//           n^-1.  Natural row order in and out.
//   pg_lde  the n values of a column are evaluations on <w_n>; the output
//           holds the same polynomial's values on the coset 7 * <w_N>,
//           N = n 2^b, row by row: the leaves of a Merkle commitment.
//
// Everything runs as passes of one kernel.  A block loads the 2^t rows of
// up to eight columns whose row indices differ only in bits [lo, lo + t)
// (a 64 KiB tile: t <= 10 for eight columns, up to 11 for fewer), performs
// the t radix-2 stages of those bits in shared memory and stores the rows
// back; a transform of 2^L rows reads and writes its data ceil(L / t) times.
//   DIF (Gentleman-Sande) stages: natural order in, bit-reversed order out;
//   DIT (Cooley-Tukey) stages: bit-reversed order in, natural order out.
// Stage of bit q pairs rows i and i + 2^q (bit q of i clear) with twiddle
// w_{q+1}^(i mod 2^q).
//
// The stages of a tile go three at a time (radix 8; four remaining bits as
// two radix-4 steps, one last bit alone).  A step over bits [b, b + r) of the
// tile combines 2^r rows v0 + 2^b m, m < 2^r, whose twiddles all derive from
// one root power tau = w_{lo+b+r}^(i mod 2^(lo+b)): the three DIT stages equal
// multiplying input m by tau^bitrev(m) and then a 2^r-point DFT of the
// bit-reversed inputs (the DIF steps are the transpose: the small DFT first,
// then output m times tau^bitrev(m)).  The small DFT's own twiddles are the
// 8th roots of unity, which are powers of two in this field: w_2 = 2^48,
// w_3 = -2^24, w_3^2 = 2^48, w_3^3 = -2^72 (mod p), so a radix-8 step takes 7
// general products and 5 shift-and-fold products instead of 12 general ones.
// Inverse roots would turn these into -2^48, 2^72, ...; instead an inverse
// step runs the same forward small DFT with its outputs (DIT) or inputs
// (DIF) at the negated index -m mod 2^r, since sum_m y_m w^(-km) is the
// forward sum at -k.  The sums inside a small DFT carry a signed top word
// and are reduced once per output (struct Lz).
//
// The powers tau^j sit in a shared table per tile: for the step at bit b,
// tau^j of the rows with low bits k (k < 2^b) at 2^b - 1 + (j - 1) 2^b + k,
// so a tile's steps fill entries [0, 2^t - 1).  tau = beta * w_{b+r}^k with
// beta = w_{lo+b+r}^(i mod 2^lo) = w_30^((i mod 2^lo) 2^(30-lo-b-r)), read
// from three 10-bit digit tables of powers of w_30.
//
// The forward NTT is DIF passes plus a bit-reversal pass; the inverse the
// same with inverse roots and n^-1.  The LDE runs the inverse as DIF passes
// into the scratch buffer, scaling row r by 7^j / n with j = bitrev(r): the
// coefficients c_j 7^j of P(7x), in bit-reversed order.  In the bit-reversed
// order of N rows the zero-padded coefficient vector has its n nonzero
// entries at the multiples of 2^b, and the first b DIT stages only copy each
// of them into the 2^b rows that follow (the other input of every butterfly
// is zero); so the DIT passes over bits b .. log2 N - 1 start by reading
// coefficient row i >> b and need no padding pass.
#include "pg12.h"
#include "pg12_internal.h"
#include "field.cuh"

#include <cuda_runtime.h>

#include <cstring>

namespace pg12 {
namespace ntt {

using dev::canon;
using dev::fold;
using dev::hi32;
using dev::lo32;
using dev::mul;
using dev::P;

constexpr int kMaxLog = 30;      // at most 2^30 rows per transform
constexpr int kMaxT = 11;        // stages per pass
#ifndef PG12_NTT_MAXU
#define PG12_NTT_MAXU 5
#endif
#ifndef PG12_NTT_CPASYNC
#define PG12_NTT_CPASYNC 1       // 1: tile loads as asynchronous copies overlapping the table setup
#endif
#ifndef PG12_NTT_TILE_BITS8
#define PG12_NTT_TILE_BITS8 10   // log2 tile rows with eight columns (64 KiB of words)
#endif
constexpr int kMaxU = PG12_NTT_MAXU;  // a tile spans up to 2^kMaxU consecutive values of the low bits
constexpr int kMaxLogC = 3;      // and at most 8 columns
constexpr int kMaxSteps = 4;     // radix-8/4/2 steps of one pass (t <= 11)
constexpr int kThreads = 256;
constexpr int kRootTab = (1 << kMaxT) - 1;     // w_{b+1}^k at index 2^b - 1 + k
constexpr uint64_t kShift = 7;                 // generator and LDE coset shift

struct Consts {
    uint64_t root[2][33];            // [0] w_k = 7^((p-1)/2^k), [1] its inverse
    uint64_t tab[2][kRootTab];       // [dir][2^b - 1 + k] = w_{b+1}^k (dir 1: inverse roots)
    uint64_t pw[2][3][1024];         // [dir][d][m] = w_30^(m 2^(10 d)) (dir 1: inverse)
    uint64_t coset[3][1024];         // [d][m] = 7^(m 2^(10 d))
};
__device__ Consts g_ntt;

// canonical product (tables)
__device__ __forceinline__ uint64_t mul_c(uint64_t a, uint64_t b) { return canon(mul(a, b)); }

// Weak operands and results (any 64-bit word standing for its residue).  A
// carry out of bit 63 is worth 2^64 = 2^32 - 1 (mod p); adding it back can
// carry once more only when both inputs were near 2^64, and then the sum is
// below 2^33.  The carry itself becomes the 32-bit mask 0 - carry (0 or
// 2^32 - 1), so no compare or select is needed.  (The flag after an add is
// a carry; subtract-with-borrow reads it as "no borrow", so the mask takes
// an add-with-carry and a negation.)
__device__ __forceinline__ uint64_t add_w(uint64_t a, uint64_t b) {
    uint32_t s0, s1;
    asm("{\n\t.reg .u32 m;\n\t"
        "add.cc.u32 %0, %2, %4;\n\t"
        "addc.cc.u32 %1, %3, %5;\n\t"
        "addc.u32 m, 0, 0;\n\t"
        "sub.u32 m, 0, m;\n\t"
        "add.cc.u32 %0, %0, m;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.u32 m, 0, 0;\n\t"
        "sub.u32 m, 0, m;\n\t"
        "add.cc.u32 %0, %0, m;\n\t"
        "addc.u32 %1, %1, 0;\n\t}"
        : "=r"(s0), "=r"(s1)
        : "r"(lo32(a)), "r"(hi32(a)), "r"(lo32(b)), "r"(hi32(b)));
    return ((uint64_t)s1 << 32) | s0;
}
// A borrow is worth -(2^32 - 1): subtracting it borrows again only when the
// difference was within 2^32 - 1 of -2^64, and then twice is enough.  The
// borrow-out of subc (0 - 0 - borrow) is already the mask.
__device__ __forceinline__ uint64_t sub_w(uint64_t a, uint64_t b) {
    uint32_t d0, d1;
    asm("{\n\t.reg .u32 m;\n\t"
        "sub.cc.u32 %0, %2, %4;\n\t"
        "subc.cc.u32 %1, %3, %5;\n\t"
        "subc.u32 m, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, m;\n\t"
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.u32 m, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, m;\n\t"
        "subc.u32 %1, %1, 0;\n\t}"
        : "=r"(d0), "=r"(d1)
        : "r"(lo32(a)), "r"(hi32(a)), "r"(lo32(b)), "r"(hi32(b)));
    return ((uint64_t)d1 << 32) | d0;
}

// ---------------------------------------------------------------- lazy sums
// Value l0 + l1 2^32 + t 2^64 with t a signed 32-bit word: a sum or
// difference of two such values is one three-word carry chain, with no
// correction.  Inside a small DFT |t| stays below 2^28 (the largest comes from
// a 2^24 shift of a value with |t| <= 2).
struct Lz {
    uint32_t l0, l1, t;
};

__device__ __forceinline__ Lz lz(uint64_t a) { return Lz{lo32(a), hi32(a), 0u}; }

__device__ __forceinline__ Lz lz_add(Lz a, Lz b) {
    Lz r;
    asm("add.cc.u32 %0, %3, %6;\n\t"
        "addc.cc.u32 %1, %4, %7;\n\t"
        "addc.u32 %2, %5, %8;"
        : "=r"(r.l0), "=r"(r.l1), "=r"(r.t)
        : "r"(a.l0), "r"(a.l1), "r"(a.t), "r"(b.l0), "r"(b.l1), "r"(b.t));
    return r;
}

__device__ __forceinline__ Lz lz_sub(Lz a, Lz b) {
    Lz r;
    asm("sub.cc.u32 %0, %3, %6;\n\t"
        "subc.cc.u32 %1, %4, %7;\n\t"
        "subc.u32 %2, %5, %8;"
        : "=r"(r.l0), "=r"(r.l1), "=r"(r.t)
        : "r"(a.l0), "r"(a.l1), "r"(a.t), "r"(b.l0), "r"(b.l1), "r"(b.t));
    return r;
}

// (w1:w0) + tp (2^32 - 1) for the top word tp in {-1, 0, 1} of a 96-bit
// value whose low 64 bits cannot wrap in this correction (the callers' ranges
// guarantee it: for tp = 1 the low word is below 2^64 - 2^32, for tp = -1 at
// least 2^32).
__device__ __forceinline__ uint64_t fix_top(uint32_t w0, uint32_t w1, uint32_t tp) {
    uint32_t r0, r1;
    asm("{\n\t.reg .u32 sh;\n\t"
        "shr.s32 sh, %4, 31;\n\t"
        "sub.cc.u32 %0, %2, %4;\n\t"
        "subc.u32 %1, %3, sh;\n\t"
        "add.u32 %1, %1, %4;\n\t}"
        : "=r"(r0), "=r"(r1)
        : "r"(w0), "r"(w1), "r"(tp));
    return ((uint64_t)r1 << 32) | r0;
}

// weak word of a lazy value: lo + t (2^32 - 1) as a 96-bit chain, |t| < 2^31
__device__ __forceinline__ uint64_t lz_reduce(Lz a) {
    uint32_t w0, w1, w2;
    asm("{\n\t.reg .u32 sh;\n\t"
        "shr.s32 sh, %5, 31;\n\t"
        "add.cc.u32 %1, %4, %5;\n\t"       // + t 2^32
        "addc.u32 %2, sh, 0;\n\t"
        "sub.cc.u32 %0, %3, %5;\n\t"       // - t
        "subc.cc.u32 %1, %1, sh;\n\t"
        "subc.u32 %2, %2, sh;\n\t}"
        : "=r"(w0), "=r"(w1), "=r"(w2)
        : "r"(a.l0), "r"(a.l1), "r"(a.t));
    return fix_top(w0, w1, w2);
}

// a 2^24, lazy: l 2^24 = (l << 24) + (l >> 40) 2^64 and t 2^88 = (t 2^24) 2^64
// (|t| < 2^7)
__device__ __forceinline__ Lz lz_m24(Lz a) {
    return Lz{a.l0 << 24, __funnelshift_l(a.l0, a.l1, 24), (a.t << 24) + (a.l1 >> 8)};
}

// a 2^48: l 2^48 = (l << 48) + (l >> 16) 2^64, (l >> 16) = hh:hl folded as
// hl (2^32 - 1) - hh, and t 2^112 = -t 2^16 (2^96 = -1); |t| < 2^31
__device__ __forceinline__ uint64_t lz_m48(Lz a) {
    const uint32_t L1 = a.l0 << 16, hl = __funnelshift_r(a.l0, a.l1, 16), hh = a.l1 >> 16;
    uint32_t w0, w1, tp;
    asm("{\n\t.reg .u32 e0, e1, e2;\n\t"
        "shl.b32 e0, %6, 16;\n\t"
        "shr.s32 e1, %6, 16;\n\t"
        "shr.s32 e2, %6, 31;\n\t"
        "sub.cc.u32 %0, 0, e0;\n\t"         // L1 2^32 - t 2^16
        "subc.cc.u32 %1, %3, e1;\n\t"
        "subc.u32 %2, 0, e2;\n\t"
        "sub.cc.u32 %0, %0, %4;\n\t"        // - hl
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.u32 %2, %2, 0;\n\t"
        "sub.cc.u32 %0, %0, %5;\n\t"        // - hh
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.u32 %2, %2, 0;\n\t"
        "add.cc.u32 %1, %1, %4;\n\t"        // + hl 2^32
        "addc.u32 %2, %2, 0;\n\t}"
        : "=r"(w0), "=r"(w1), "=r"(tp)
        : "r"(L1), "r"(hl), "r"(hh), "r"(a.t));
    return fix_top(w0, w1, tp);
}

// a 2^72: l 2^72 = (l << 8) 2^64 + (l >> 56) 2^128, folded as for a product
// (2^64 = 2^32 - 1, 2^96 = -1, 2^128 = -2^32), and t 2^136 = -t 2^40;
// |t| < 2^23
__device__ __forceinline__ uint64_t lz_m72(Lz a) {
    const uint32_t hl = a.l0 << 8, hh = __funnelshift_l(a.l0, a.l1, 8), k = a.l1 >> 24;
    uint32_t w0, w1, tp;
    asm("{\n\t.reg .u32 e1, e2;\n\t"
        "shl.b32 e1, %6, 8;\n\t"
        "shr.s32 e2, %6, 31;\n\t"
        "sub.cc.u32 %0, 0, %3;\n\t"         // - hl - k 2^32
        "subc.cc.u32 %1, 0, %5;\n\t"
        "subc.u32 %2, 0, 0;\n\t"
        "sub.cc.u32 %0, %0, %4;\n\t"        // - hh
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.u32 %2, %2, 0;\n\t"
        "add.cc.u32 %1, %1, %3;\n\t"        // + hl 2^32
        "addc.u32 %2, %2, 0;\n\t"
        "sub.cc.u32 %1, %1, e1;\n\t"        // - t 2^40
        "subc.u32 %2, %2, e2;\n\t}"
        : "=r"(w0), "=r"(w1), "=r"(tp)
        : "r"(hl), "r"(hh), "r"(k), "r"(a.t));
    return fix_top(w0, w1, tp);
}

// ---------------------------------------------------------------- small DFTs
// Forward 8-point DFT, DIT order: input position m holds index bitrev3(m),
// output natural.  Stage twiddles: stage 1 w_2 = 2^48 on pairs (1,3), (5,7);
// stage 2 w_3^m = 1, -2^24, 2^48, -2^72 on pairs (m, m + 4).
__device__ __forceinline__ void dft8_dit(uint64_t (&a)[8]) {
    const Lz b0 = lz_add(lz(a[0]), lz(a[1])), b1 = lz_sub(lz(a[0]), lz(a[1]));
    const Lz b2 = lz_add(lz(a[2]), lz(a[3])), b3 = lz_sub(lz(a[2]), lz(a[3]));
    const Lz b4 = lz_add(lz(a[4]), lz(a[5])), b5 = lz_sub(lz(a[4]), lz(a[5]));
    const Lz b6 = lz_add(lz(a[6]), lz(a[7])), b7 = lz_sub(lz(a[6]), lz(a[7]));
    const Lz c0 = lz_add(b0, b2), c2 = lz_sub(b0, b2);
    const Lz y3 = lz(lz_m48(b3));
    const Lz c1 = lz_add(b1, y3), c3 = lz_sub(b1, y3);
    const Lz c4 = lz_add(b4, b6), c6 = lz_sub(b4, b6);
    const Lz y7 = lz(lz_m48(b7));
    const Lz c5 = lz_add(b5, y7), c7 = lz_sub(b5, y7);
    a[0] = lz_reduce(lz_add(c0, c4));
    a[4] = lz_reduce(lz_sub(c0, c4));
    const Lz z5 = lz_m24(c5);
    a[1] = lz_reduce(lz_sub(c1, z5));
    a[5] = lz_reduce(lz_add(c1, z5));
    const Lz z6 = lz(lz_m48(c6));
    a[2] = lz_reduce(lz_add(c2, z6));
    a[6] = lz_reduce(lz_sub(c2, z6));
    const Lz z7 = lz(lz_m72(c7));
    a[3] = lz_reduce(lz_sub(c3, z7));
    a[7] = lz_reduce(lz_add(c3, z7));
}

// Forward 8-point DFT, DIF order: natural input, output position m holds
// index bitrev3(m); the transpose of dft8_dit.
__device__ __forceinline__ void dft8_dif(uint64_t (&a)[8]) {
    const Lz b0 = lz_add(lz(a[0]), lz(a[4])), b4 = lz_sub(lz(a[0]), lz(a[4]));
    const Lz b1 = lz_add(lz(a[1]), lz(a[5])), b5 = lz_m24(lz_sub(lz(a[5]), lz(a[1])));
    const Lz b2 = lz_add(lz(a[2]), lz(a[6])), b6 = lz(lz_m48(lz_sub(lz(a[2]), lz(a[6]))));
    const Lz b3 = lz_add(lz(a[3]), lz(a[7])), b7 = lz(lz_m72(lz_sub(lz(a[7]), lz(a[3]))));
    const Lz c0 = lz_add(b0, b2), c2 = lz_sub(b0, b2);
    const Lz c1 = lz_add(b1, b3), c3 = lz(lz_m48(lz_sub(b1, b3)));
    const Lz c4 = lz_add(b4, b6), c6 = lz_sub(b4, b6);
    const Lz c5 = lz_add(b5, b7), c7 = lz(lz_m48(lz_sub(b5, b7)));
    a[0] = lz_reduce(lz_add(c0, c1));
    a[1] = lz_reduce(lz_sub(c0, c1));
    a[2] = lz_reduce(lz_add(c2, c3));
    a[3] = lz_reduce(lz_sub(c2, c3));
    a[4] = lz_reduce(lz_add(c4, c5));
    a[5] = lz_reduce(lz_sub(c4, c5));
    a[6] = lz_reduce(lz_add(c6, c7));
    a[7] = lz_reduce(lz_sub(c6, c7));
}

// Forward 4-point DFTs (w_2 = 2^48), DIT (input position m holds index
// bitrev2(m)) and DIF (output position m holds index bitrev2(m)).
__device__ __forceinline__ void dft4_dit(uint64_t (&a)[4]) {
    const Lz b0 = lz_add(lz(a[0]), lz(a[1])), b1 = lz_sub(lz(a[0]), lz(a[1]));
    const Lz b2 = lz_add(lz(a[2]), lz(a[3])), b3 = lz_sub(lz(a[2]), lz(a[3]));
    const Lz y3 = lz(lz_m48(b3));
    a[0] = lz_reduce(lz_add(b0, b2));
    a[2] = lz_reduce(lz_sub(b0, b2));
    a[1] = lz_reduce(lz_add(b1, y3));
    a[3] = lz_reduce(lz_sub(b1, y3));
}

__device__ __forceinline__ void dft4_dif(uint64_t (&a)[4]) {
    const Lz b0 = lz_add(lz(a[0]), lz(a[2])), b2 = lz_sub(lz(a[0]), lz(a[2]));
    const Lz b1 = lz_add(lz(a[1]), lz(a[3])), b3 = lz(lz_m48(lz_sub(lz(a[1]), lz(a[3]))));
    a[0] = lz_reduce(lz_add(b0, b1));
    a[1] = lz_reduce(lz_sub(b0, b1));
    a[2] = lz_reduce(lz_add(b2, b3));
    a[3] = lz_reduce(lz_sub(b2, b3));
}

// x^e for a 30-bit exponent from three 10-bit digit tables
__device__ __forceinline__ uint64_t pow_tab(const uint64_t (*t)[1024], uint64_t e) {
    return mul_c(mul_c(t[0][e & 1023], t[1][(e >> 10) & 1023]), t[2][(e >> 20) & 1023]);
}

struct Pass {
    const uint64_t *src;  // rows read (row i of the pass reads src row i >> src_shift)
    uint64_t *dst;        // rows written (may equal src)
    uint64_t ncols;
    uint64_t scale_c;     // scale 1 and 2: constant factor (n^-1)
    uint32_t log_n;       // the transform has 2^log_n rows
    uint32_t lo, t;       // row-index bits [lo, lo + t) are transformed
    uint32_t u;           // the tile spans 2^u consecutive values of bits [0, lo) (u <= lo)
    uint32_t dit;         // 0: DIF stages (top bit first), 1: DIT stages (bit lo first)
    uint32_t inverse;     // inverse roots
    uint32_t src_shift;
    uint32_t scale;       // 0: none; 1: times scale_c; 2: times scale_c * 7^bitrev(row) (needs lo = 0)
    uint32_t last;        // 1: store canonical words (last pass of a transform)
};

// log2 radix of the step after `done` of t bits: 3 while more than four bits
// remain (four go as 2 + 2), then 2, then a last single bit.
__host__ __device__ __forceinline__ uint32_t step_log_radix(uint32_t t, uint32_t done) {
    const uint32_t left = t - done;
    return left >= 3 && left != 4 ? 3u : left >= 2 ? 2u : 1u;
}

// One step of radix 2^R over the rows x[m s0] (m < 2^R) with tau^j at
// w[(j - 1) << b] (triv: tau = 1).
template <int DIT, int R>
__device__ __forceinline__ void step(uint64_t *x, uint32_t s0, const uint64_t *w, uint32_t b, bool inv, bool triv) {
    if constexpr (R == 1) {
        const uint64_t a0 = x[0], a1 = x[s0];
        if (DIT) {
            const uint64_t y = triv ? a1 : mul(a1, w[0]);
            x[0] = add_w(a0, y);
            x[s0] = sub_w(a0, y);
        } else {
            const uint64_t d = sub_w(a0, a1);
            x[0] = add_w(a0, a1);
            x[s0] = triv ? d : mul(d, w[0]);
        }
    } else {
        constexpr int N = 1 << R;
        // position m takes tau^bitrev(m): radix 8 {-, 4, 2, 6, 1, 5, 3, 7}, radix 4 {-, 2, 1, 3}
        constexpr int kE[8] = {0, R == 3 ? 4 : 2, R == 3 ? 2 : 1, R == 3 ? 6 : 3, 1, 5, 3, 7};
        uint64_t a[N];
        if (DIT) {
#pragma unroll
            for (int m = 0; m < N; ++m) a[m] = x[m * s0];
            if (!triv) {
#pragma unroll
                for (int m = 1; m < N; ++m) a[m] = mul(a[m], w[(kE[m] - 1) << b]);
            }
            if constexpr (R == 3) dft8_dit(a);
            else dft4_dit(a);
            x[0] = a[0];
            if (inv) {
#pragma unroll
                for (int m = 1; m < N; ++m) x[(N - m) * s0] = a[m];
            } else {
#pragma unroll
                for (int m = 1; m < N; ++m) x[m * s0] = a[m];
            }
        } else {
            a[0] = x[0];
            if (inv) {
#pragma unroll
                for (int m = 1; m < N; ++m) a[m] = x[(N - m) * s0];
            } else {
#pragma unroll
                for (int m = 1; m < N; ++m) a[m] = x[m * s0];
            }
            if constexpr (R == 3) dft8_dif(a);
            else dft4_dif(a);
            if (!triv) {
#pragma unroll
                for (int m = 1; m < N; ++m) a[m] = mul(a[m], w[(kE[m] - 1) << b]);
            }
#pragma unroll
            for (int m = 0; m < N; ++m) x[m * s0] = a[m];
        }
    }
}

// One pass.  The tile holds 2^t values of the transformed bits x 2^u
// consecutive values of the low bits x 2^LOG_C columns; element (v, l, c) at
// ((v 2^u + l) 2^LOG_C + c), so for fixed v the 2^u rows are one contiguous
// run in memory.  Columns past ncols are zero and not stored.  Each low value
// l has its own table of root powers (2^t - 1 of them, rows padded by one
// word so that different l fall in different banks).
template <int DIT, int LOG_C>
__global__ void __launch_bounds__(kThreads) k_ntt_pass(const Pass ps) {
    constexpr uint32_t C = 1u << LOG_C;
    extern __shared__ uint64_t sm[];
    const uint32_t t = ps.t, u = ps.u;
    const uint32_t rows = 1u << t;
    const uint32_t words = rows << (u + LOG_C);
    const uint32_t tws = rows + 1;
    uint64_t *tile = sm;                 // [rows][2^u][C]
    uint64_t *tw = sm + words;           // [2^u][tws]
    uint64_t *fac = tw + (tws << u);     // [rows], scale 2 only
    __shared__ uint64_t beta[1 << kMaxU][kMaxSteps];

    const uint64_t chunks = (ps.ncols + C - 1) >> LOG_C;
    const uint64_t outer = chunks == 1 ? blockIdx.x : blockIdx.x / chunks;
    const uint64_t col0 = (blockIdx.x - outer * chunks) << LOG_C;
    const uint32_t c_eff = (uint32_t)((ps.ncols - col0) < (uint64_t)C ? (ps.ncols - col0) : (uint64_t)C);
    const uint64_t low0 = (outer & ((1ull << (ps.lo - u)) - 1)) << u;
    const uint64_t high = outer >> (ps.lo - u);
    const uint64_t base = (high << (ps.lo + t)) | low0;
    const uint32_t dir = ps.inverse ? 1u : 0u;
    const bool inv = ps.inverse != 0;

    // the steps: log radix (2 bits each) and lowest bit (4 bits each)
    uint32_t plan_r = 0, plan_b = 0, nsteps = 0;
    for (uint32_t done = 0; done < t; ++nsteps) {
        const uint32_t r = step_log_radix(t, done);
        plan_r |= r << (2 * nsteps);
        plan_b |= (DIT ? done : t - done - r) << (4 * nsteps);
        done += r;
    }
    // Each thread keeps one (low value, column) slot: kThreads is a multiple
    // of 2^(u + LOG_C) <= 256, so its rows advance by a fixed stride.
    const uint32_t slot = threadIdx.x & ((C << u) - 1);
    const uint32_t c_me = slot & (C - 1), l_me = slot >> LOG_C;
    const uint32_t v_first = threadIdx.x >> (u + LOG_C), v_step = kThreads >> (u + LOG_C);
    const bool col_ok = c_me < c_eff;
    {
        // source row of tile row v: ((base | v << lo | l) >> src_shift); src_shift is
        // 0 or equal to lo, so it is linear in v either way.  With PG12_NTT_CPASYNC the
        // words go to shared memory as asynchronous copies, which stay in flight while
        // the root-power tables are built.
        const uint64_t r0 = (base | ((uint64_t)v_first << ps.lo) | l_me) >> ps.src_shift;
        const uint64_t rstep = ((uint64_t)v_step << ps.lo) >> ps.src_shift;
        const uint64_t *g = ps.src + r0 * ps.ncols + col0 + c_me;
        const uint64_t gstep = rstep * ps.ncols;
        for (uint32_t v = v_first, e = threadIdx.x; v < rows; v += v_step, e += kThreads, g += gstep) {
#if PG12_NTT_CPASYNC
            if (col_ok)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(tile + e)),
                             "l"(g)
                             : "memory");
            else
                tile[e] = 0;
#else
            tile[e] = col_ok ? *g : 0;
#endif
        }
#if PG12_NTT_CPASYNC
        asm volatile("cp.async.commit_group;" ::: "memory");
#endif
    }
    // beta[l][i] = w_{lo+b+r}^(low0 + l) for step i over bits [b, b + r)
    for (uint32_t q = threadIdx.x; q < (nsteps << u); q += kThreads) {
        const uint32_t i = q >> u, l = q & ((1u << u) - 1);
        const uint32_t top = ((plan_b >> (4 * i)) & 15) + ((plan_r >> (2 * i)) & 3);
        beta[l][i] = pow_tab(g_ntt.pw[dir], (low0 + l) << (30 - ps.lo - top));
    }
    if (ps.scale == 2) {
        // row factors scale_c 7^bitrev(row) (here lo = u = 0: row = base + v)
        for (uint32_t v = threadIdx.x; v < rows; v += kThreads) {
            const uint64_t row = base + v;
            const uint64_t j = ps.log_n ? (uint64_t)(__brevll(row) >> (64 - ps.log_n)) : 0;
            fac[v] = mul(pow_tab(g_ntt.coset, j), ps.scale_c);
        }
    }
    __syncthreads();
    // tau^j tables: step i at bit b, low value l, rows with low bits k < 2^b
    for (uint32_t i = 0; i < nsteps; ++i) {
        const uint32_t r = (plan_r >> (2 * i)) & 3, b = (plan_b >> (4 * i)) & 15;
        const uint32_t nb = 1u << b, s = b + r - 1;
        for (uint32_t q = threadIdx.x; q < (nb << u); q += kThreads) {
            const uint32_t l = q >> b, k = q & (nb - 1);
            const uint64_t tau = mul(beta[l][i], g_ntt.tab[dir][(1u << s) - 1 + k]);
            uint64_t *d = tw + l * tws + nb - 1 + k;
            uint64_t x = tau;
            d[0] = x;
            for (uint32_t j = 2; j < (1u << r); ++j) {
                x = mul(x, tau);
                d[(j - 1) << b] = x;
            }
        }
    }
#if PG12_NTT_CPASYNC
    asm volatile("cp.async.wait_all;" ::: "memory");
#endif
    __syncthreads();

    const uint32_t sh = u + LOG_C;
    for (uint32_t i = 0; i < nsteps; ++i) {
        const uint32_t r = (plan_r >> (2 * i)) & 3, b = (plan_b >> (4 * i)) & 15;
        const uint32_t nb = 1u << b, s0 = 1u << (b + sh);
        const uint32_t groups = (rows >> r) << sh;
        const bool triv = b == 0 && ps.lo == 0;  // tau = w^0 (lo = 0 means u = 0)
        for (uint32_t p = threadIdx.x; p < groups; p += kThreads) {
            const uint32_t lc = p & ((C << u) - 1), g = p >> sh;
            const uint32_t k = g & (nb - 1);
            const uint32_t v0 = ((g >> b) << (b + r)) | k;
            uint64_t *x = tile + ((v0 << sh) + lc);
            const uint64_t *w = tw + (lc >> LOG_C) * tws + nb - 1 + k;
            if (r == 3) step<DIT, 3>(x, s0, w, b, inv, triv);
            else if (r == 2) step<DIT, 2>(x, s0, w, b, inv, triv);
            else step<DIT, 1>(x, s0, w, b, inv, triv);
        }
        __syncthreads();
    }

    if (!col_ok) return;
    {
        const uint64_t r0 = base | ((uint64_t)v_first << ps.lo) | l_me;
        const uint64_t rstep = (uint64_t)v_step << ps.lo;
        uint64_t *g = ps.dst + r0 * ps.ncols + col0 + c_me;
        const uint64_t gstep = rstep * ps.ncols;
        for (uint32_t v = v_first, e = threadIdx.x; v < rows; v += v_step, e += kThreads, g += gstep) {
            uint64_t x = tile[e];
            if (ps.scale == 1) x = mul(x, ps.scale_c);
            else if (ps.scale == 2) x = mul(x, fac[v]);
            *g = ps.last ? canon(x) : x;
        }
    }
}

// Swaps rows i and bitrev(i) (i < bitrev(i)) of a 2^log_n-row array.
__global__ void k_ntt_bitrev(uint64_t *__restrict__ data, uint32_t log_n, uint64_t ncols) {
    const uint64_t total = (ncols << log_n);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const uint64_t i = e / ncols, c = e - i * ncols;
        const uint64_t r = log_n ? (__brevll(i) >> (64 - log_n)) : 0;
        if (i < r) {
            const uint64_t a = data[i * ncols + c], b = data[r * ncols + c];
            data[i * ncols + c] = b;
            data[r * ncols + c] = a;
        }
    }
}

// log2 of the tile's rows (transformed x low values) for 2^log_c columns:
// tile plus tables stay within 72-98 KiB of shared memory.
uint32_t tile_bits(uint32_t log_c) { return log_c >= 3 ? (uint32_t)PG12_NTT_TILE_BITS8 : log_c == 2 ? 11u : 12u; }
uint32_t max_t(uint32_t log_c) { return tile_bits(log_c) < (uint32_t)kMaxT ? tile_bits(log_c) : (uint32_t)kMaxT; }

// tile, root-power tables (2^t + 1 words per low value) and, for the LDE
// scaling, one factor per row
size_t pass_smem(uint32_t t, uint32_t u, uint32_t log_c, bool row_factors) {
    return (((size_t)1 << (t + u + log_c)) + ((((size_t)1 << t) + 1) << u) + (row_factors ? (size_t)1 << t : 0)) *
           sizeof(uint64_t);
}

// the largest pass_smem over the passes of 2^log_c columns (t + u <= tile_bits)
size_t max_pass_smem(uint32_t log_c) {
    const uint32_t tb = tile_bits(log_c);
    return (((size_t)1 << (tb + log_c)) + ((size_t)1 << tb) + ((size_t)1 << kMaxU) + ((size_t)1 << max_t(log_c))) *
           sizeof(uint64_t);
}

// columns per tile: the smallest power of two >= min(ncols, 8)
uint32_t tile_log_c(uint64_t ncols) {
    uint32_t lc = 0;
    while (lc < (uint32_t)kMaxLogC && (1ull << lc) < ncols) ++lc;
    return lc;
}

// low-bit span of a pass over bits [lo, lo + t)
uint32_t tile_u(uint32_t lo, uint32_t t, uint32_t log_c) {
    uint32_t u = tile_bits(log_c) - t;
    if (u > (uint32_t)kMaxU) u = kMaxU;
    return u < lo ? u : lo;
}

bool g_attr_set[64];

template <int DIT, int LOG_C>
cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_ntt_pass<DIT, LOG_C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)max_pass_smem(LOG_C));
}

template <int DIT, int LOG_C>
void launch_one(const Pass &ps, unsigned blocks, size_t smem, cudaStream_t st) {
    k_ntt_pass<DIT, LOG_C><<<blocks, kThreads, smem, st>>>(ps);
}

// Launches one pass; the grid is 2^(log_n - t) row groups x column chunks.
int launch_pass(Pass ps, cudaStream_t st) {
    const uint32_t lc = tile_log_c(ps.ncols);
    ps.u = tile_u(ps.lo, ps.t, lc);
    const uint64_t chunks = (ps.ncols + (1ull << lc) - 1) >> lc;
    const uint64_t blocks = (1ull << (ps.log_n - ps.t - ps.u)) * chunks;
    if (blocks > 0x7FFFFFFFull) return set_error(PG_ERR_INVALID_ARG, "NTT pass needs %llu blocks", (unsigned long long)blocks);
    if (ps.t > max_t(lc)) return set_error(PG_ERR_INVALID_ARG, "NTT pass of %u bits", ps.t);
    if (ps.scale == 2 && (ps.lo != 0 || ps.u != 0)) return set_error(PG_ERR_INVALID_ARG, "row factors need lo = 0");
    const size_t smem = pass_smem(ps.t, ps.u, lc, ps.scale == 2);
    int device = 0;
    cudaGetDevice(&device);
    if (device >= 0 && device < 64 && !g_attr_set[device]) {
        const cudaError_t es[8] = {set_smem_attr<0, 0>(), set_smem_attr<0, 1>(), set_smem_attr<0, 2>(),
                                   set_smem_attr<0, 3>(), set_smem_attr<1, 0>(), set_smem_attr<1, 1>(),
                                   set_smem_attr<1, 2>(), set_smem_attr<1, 3>()};
        for (cudaError_t e : es)
            if (e != cudaSuccess) return set_error(PG_ERR_CUDA, "NTT shared-memory attribute: %s", cudaGetErrorString(e));
        g_attr_set[device] = true;
    }
    ProfScope prof(kIdNttPass, st, 0);
    const unsigned nb = (unsigned)blocks;
    switch (lc + (ps.dit ? 4u : 0u)) {
        case 0: launch_one<0, 0>(ps, nb, smem, st); break;
        case 1: launch_one<0, 1>(ps, nb, smem, st); break;
        case 2: launch_one<0, 2>(ps, nb, smem, st); break;
        case 3: launch_one<0, 3>(ps, nb, smem, st); break;
        case 4: launch_one<1, 0>(ps, nb, smem, st); break;
        case 5: launch_one<1, 1>(ps, nb, smem, st); break;
        case 6: launch_one<1, 2>(ps, nb, smem, st); break;
        default: launch_one<1, 3>(ps, nb, smem, st); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PG_ERR_CUDA, "k_ntt_pass: %s", cudaGetErrorString(e));
    return PG_OK;
}

// Bits per pass for `bits` index bits, in execution order, each pass at most
// `tmax` bits, in the fewest passes.  When a multiple of three fits those
// passes in multiples of three, every step is radix 8 (three stages per
// shared-memory round trip, the cheapest per stage).  Otherwise: a tile's low
// values lie below its bits, so the pass over the lowest bits (lo = 0 in the
// DIF passes) has none and would otherwise get a small tile: it takes tmax
// bits and the other passes share the rest evenly.  low_first: the lowest
// pass runs first (DIT) rather than last (DIF).
int plan_passes(uint32_t bits, uint32_t tmax, bool low_first, uint32_t *t_out) {
    if (bits == 0) {
        t_out[0] = 0;
        return 1;
    }
    const uint32_t np = (bits + tmax - 1) / tmax, t3 = tmax - tmax % 3;
    uint32_t unit = 1, tl = bits < tmax ? bits : tmax;
    if (bits % 3 == 0 && bits <= np * t3) {
        unit = 3;
        tl = bits < t3 ? bits : t3;
    }
    const uint32_t rest = (bits - tl) / unit, n = np - 1;
    uint32_t k = 0;
    if (low_first) t_out[k++] = tl;
    for (uint32_t i = 0; i < n; ++i) t_out[k++] = unit * (rest / n + (i < rest % n ? 1u : 0u));
    if (!low_first) t_out[k++] = tl;
    return (int)k;
}

// DIF passes over all log_n bits of `dst` (first pass reads `src`).
int run_dif(const uint64_t *src, uint64_t *dst, uint32_t log_n, uint64_t ncols, bool inverse, uint32_t scale,
            uint64_t scale_c, cudaStream_t st) {
    uint32_t ts[32];
    const int np = plan_passes(log_n, max_t(tile_log_c(ncols)), false, ts);
    uint32_t top = log_n;
    for (int k = 0; k < np; ++k) {
        Pass ps;
        std::memset(&ps, 0, sizeof ps);
        ps.src = k == 0 ? src : dst;
        ps.dst = dst;
        ps.ncols = ncols;
        ps.log_n = log_n;
        ps.t = ts[k];
        ps.lo = top - ts[k];
        ps.dit = 0;
        ps.inverse = inverse ? 1u : 0u;
        ps.scale = k == np - 1 ? scale : 0u;
        ps.scale_c = scale_c;
        ps.last = k == np - 1 ? 1u : 0u;
        int s = launch_pass(ps, st);
        if (s != PG_OK) return s;
        top -= ts[k];
    }
    return PG_OK;
}

uint64_t host_pow(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = host::fp_mul(r, a);
        a = host::fp_mul(a, a);
        e >>= 1;
    }
    return r;
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }
uint32_t log2u(uint64_t x) {
    uint32_t k = 0;
    while ((1ull << k) < x) ++k;
    return k;
}

}  // namespace ntt

int ntt_upload_constants() {
    using namespace ntt;
    static Consts h;
    const uint64_t pm1 = 0xFFFFFFFF00000000ull;  // p - 1
    for (int k = 0; k <= 32; ++k) {
        h.root[0][k] = host_pow(kShift, pm1 >> k);
        h.root[1][k] = host::fp_inv(h.root[0][k]);
    }
    for (int dir = 0; dir < 2; ++dir)
        for (int b = 0; b < kMaxT; ++b) {
            uint64_t x = 1;
            for (int k = 0; k < (1 << b); ++k) {
                h.tab[dir][(1 << b) - 1 + k] = x;
                x = host::fp_mul(x, h.root[dir][b + 1]);
            }
        }
    for (int d = 0; d < 3; ++d) {
        const uint64_t step = host_pow(kShift, 1ull << (10 * d));
        uint64_t x = 1;
        for (int m = 0; m < 1024; ++m) {
            h.coset[d][m] = x;
            x = host::fp_mul(x, step);
        }
        for (int dir = 0; dir < 2; ++dir) {
            const uint64_t wstep = host_pow(h.root[dir][30], 1ull << (10 * d));
            uint64_t y = 1;
            for (int m = 0; m < 1024; ++m) {
                h.pw[dir][d][m] = y;
                y = host::fp_mul(y, wstep);
            }
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(g_ntt, &h, sizeof h);
    if (e != cudaSuccess) return set_error(PG_ERR_CUDA, "NTT constants: %s", cudaGetErrorString(e));
    return PG_OK;
}

}  // namespace pg12

extern "C" {

pg_status pg_ntt(uint64_t *data, size_t n, size_t ncols, int inverse, void *stream) {
    using namespace pg12::ntt;
    if (!data) return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "data is NULL");
    if (ncols == 0) return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "ncols must be >= 1");
    if (!is_pow2(n)) return (pg_status)pg12::set_error(PG_ERR_NOT_POW2, "n=%zu is not a power of two", n);
    if (n > (1ull << kMaxLog)) return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "n=%zu above 2^%d", n, kMaxLog);
    if (reinterpret_cast<uintptr_t>(data) % 8) return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "data not 8-byte aligned");
    int s = pg12::ntt_require_init();
    if (s != PG_OK) return (pg_status)s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint32_t log_n = log2u(n);
    const uint64_t ninv = pg12::host::fp_inv((uint64_t)n);
    s = run_dif(data, data, log_n, ncols, inverse != 0, inverse ? 1u : 0u, ninv, st);
    if (s != PG_OK) return (pg_status)s;
    if (log_n > 0) {
        pg12::ProfScope prof(pg12::kIdNttBitrev, st, 0);
        const uint64_t total = (uint64_t)ncols << log_n;
        const uint64_t want = (total + 255) / 256;
        const unsigned grid = (unsigned)(want < 152ull * 16 ? want : 152ull * 16);
        k_ntt_bitrev<<<grid, 256, 0, st>>>(data, log_n, (uint64_t)ncols);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return (pg_status)pg12::set_error(PG_ERR_CUDA, "k_ntt_bitrev: %s", cudaGetErrorString(e));
    }
    return PG_OK;
}

pg_status pg_lde(const uint64_t *evals, size_t n, size_t ncols, uint32_t log_blowup, uint64_t *out,
                 uint64_t *scratch, void *stream) {
    using namespace pg12::ntt;
    if (!evals || !out || !scratch) return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "evals, out or scratch is NULL");
    if (ncols == 0) return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "ncols must be >= 1");
    if (!is_pow2(n)) return (pg_status)pg12::set_error(PG_ERR_NOT_POW2, "n=%zu is not a power of two", n);
    if (log_blowup > 16) return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "log_blowup=%u above 16", log_blowup);
    const uint32_t log_n = log2u(n);
    if (log_n + log_blowup > (uint32_t)kMaxLog)
        return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "n * 2^log_blowup above 2^%d rows", kMaxLog);
    if ((reinterpret_cast<uintptr_t>(evals) | reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(scratch)) % 8)
        return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "buffers must be 8-byte aligned");
    {
        const uintptr_t o0 = reinterpret_cast<uintptr_t>(out), o1 = o0 + ((uint64_t)ncols << (log_n + log_blowup)) * 8;
        const uintptr_t s0 = reinterpret_cast<uintptr_t>(scratch), s1 = s0 + ((uint64_t)ncols << log_n) * 8;
        const uintptr_t e0 = reinterpret_cast<uintptr_t>(evals), e1 = e0 + ((uint64_t)ncols << log_n) * 8;
        if ((s0 < o1 && o0 < s1) || (e0 < o1 && o0 < e1))
            return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "out overlaps evals or scratch");
        if (scratch != evals && s0 < e1 && e0 < s1)
            return (pg_status)pg12::set_error(PG_ERR_INVALID_ARG, "scratch partly overlaps evals");
    }
    int s = pg12::ntt_require_init();
    if (s != PG_OK) return (pg_status)s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // coefficients c_j 7^j in bit-reversed order into scratch
    s = run_dif(evals, scratch, log_n, ncols, true, 2u, pg12::host::fp_inv((uint64_t)n), st);
    if (s != PG_OK) return (pg_status)s;
    // DIT passes over bits [b, log N) of out; the first reads coefficient row i >> b
    const uint32_t log_big = log_n + log_blowup;
    uint32_t ts[32];
    const int np = plan_passes(log_n, max_t(tile_log_c(ncols)), true, ts);
    uint32_t lo = log_blowup;
    for (int k = 0; k < np; ++k) {
        Pass ps;
        std::memset(&ps, 0, sizeof ps);
        ps.src = k == 0 ? scratch : out;
        ps.dst = out;
        ps.ncols = ncols;
        ps.log_n = log_big;
        ps.t = ts[k];
        ps.lo = log_n ? lo : 0;
        ps.dit = 1;
        ps.src_shift = k == 0 ? log_blowup : 0;
        ps.last = k == np - 1 ? 1u : 0u;
        s = launch_pass(ps, st);
        if (s != PG_OK) return (pg_status)s;
        lo += ts[k];
    }
    return PG_OK;
}

}  // extern "C"
