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
// the t radix-2 stages of those bits in shared memory, two at a time as
// radix-4 groups of four rows per thread, and stores the rows back; a
// transform of 2^L rows reads and writes its data ceil(L / t) times.
//   DIF (Gentleman-Sande) stages: natural order in, bit-reversed order out;
//   DIT (Cooley-Tukey) stages: bit-reversed order in, natural order out.
// Stage of bit q pairs rows i and i + 2^q (bit q of i clear) with twiddle
// w_{q+1}^(i mod 2^q).  Within a block the low part (i mod 2^lo) is fixed, so
// the twiddles of stage lo + b are beta_b * w_{b+1}^k, k < 2^b, with
// beta_b = w_{lo+b+1}^(i mod 2^lo) = w_30^((i mod 2^lo) 2^(29-lo-b)), read from
// three 10-bit digit tables of powers of w_30, then one product per twiddle
// from a shared table of the powers of w_{b+1}.
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
using dev::mul;
using dev::P;

constexpr int kMaxLog = 30;      // at most 2^30 rows per transform
constexpr int kMaxT = 11;        // stages per pass
#ifndef PG12_NTT_MAXU
#define PG12_NTT_MAXU 4
#endif
#ifndef PG12_NTT_TILE_BITS8
#define PG12_NTT_TILE_BITS8 10   // log2 tile rows with eight columns (64 KiB of words)
#endif
#ifndef PG12_NTT_RADIX8
#define PG12_NTT_RADIX8 1        // 1: three stages per shared-memory round trip where they fit
#endif
#ifndef PG12_NTT_NO_R2
#define PG12_NTT_NO_R2 1         // 1: split 4 remaining stages 2 + 2 instead of 3 + 1
#endif
constexpr int kMaxU = PG12_NTT_MAXU;  // a tile spans up to 2^kMaxU consecutive values of the low bits
constexpr int kMaxLogC = 3;      // and at most 8 columns
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

// canonical product (tables and scale factors)
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
        : "r"(dev::lo32(a)), "r"(dev::hi32(a)), "r"(dev::lo32(b)), "r"(dev::hi32(b)));
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
        : "r"(dev::lo32(a)), "r"(dev::hi32(a)), "r"(dev::lo32(b)), "r"(dev::hi32(b)));
    return ((uint64_t)d1 << 32) | d0;
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
    uint32_t scale;       // 0: none; 1: times scale_c; 2: times scale_c * 7^bitrev(row)
    uint32_t last;        // 1: store canonical words (last pass of a transform)
};

// DIF butterfly (a, b) -> (a + b, (a - b) w); DIT (a, b) -> (a + b w, a - b w).
template <int DIT>
__device__ __forceinline__ void bfly(uint64_t &a, uint64_t &b, uint64_t w) {
    if (DIT) {
        const uint64_t y = mul(b, w);
        b = sub_w(a, y);
        a = add_w(a, y);
    } else {
        const uint64_t d = sub_w(a, b);
        a = add_w(a, b);
        b = mul(d, w);
    }
}

// One pass.  The tile holds 2^t values of the transformed bits x 2^u
// consecutive values of the low bits x 2^LOG_C columns; element (v, l, c) at
// ((v 2^u + l) 2^LOG_C + c), so for fixed v the 2^u rows are one contiguous
// run in memory.  Columns past ncols are zero and not stored.  Each low value
// l has its own twiddles (rows - 1 of them).  Stages go in pairs (radix 4:
// four rows per thread, two stages between barriers), with one radix-2 stage
// when t is odd.
template <int DIT, int LOG_C>
__global__ void __launch_bounds__(kThreads) k_ntt_pass(const Pass ps) {
    constexpr uint32_t C = 1u << LOG_C;
    extern __shared__ uint64_t sm[];
    const uint32_t t = ps.t, u = ps.u;
    const uint32_t rows = 1u << t;
    const uint32_t words = rows << (u + LOG_C);
    uint64_t *tile = sm;          // [rows][2^u][C]
    uint64_t *tw = sm + words;    // [2^u][rows], entry rows - 1 unused
    __shared__ uint64_t beta[1 << (kMaxU > 4 ? kMaxU : 4)][16];

    const uint64_t chunks = (ps.ncols + C - 1) >> LOG_C;
    const uint64_t outer = blockIdx.x / chunks;
    const uint64_t col0 = (blockIdx.x - outer * chunks) << LOG_C;
    const uint32_t c_eff = (uint32_t)((ps.ncols - col0) < (uint64_t)C ? (ps.ncols - col0) : (uint64_t)C);
    const uint64_t low0 = (outer & ((1ull << (ps.lo - u)) - 1)) << u;
    const uint64_t high = outer >> (ps.lo - u);
    const uint64_t base = (high << (ps.lo + t)) | low0;
    const uint32_t dir = ps.inverse ? 1u : 0u;

    // beta[l][b] = w_{lo+b+1}^(low0+l) = w_30^((low0+l) 2^(29 - lo - b))
    for (uint32_t e = threadIdx.x; e < (16u << u); e += kThreads) {
        const uint32_t l = e >> 4, b = e & 15;
        if (b < t) beta[l][b] = pow_tab(g_ntt.pw[dir], (low0 + l) << (29 - ps.lo - b));
    }
    // Each thread keeps one (low value, column) slot: kThreads is a multiple
    // of 2^(u + LOG_C) <= 128, so its rows advance by a fixed stride.
    const uint32_t slot = threadIdx.x & ((C << u) - 1);
    const uint32_t c_me = slot & (C - 1), l_me = slot >> LOG_C;
    const uint32_t v_first = threadIdx.x >> (u + LOG_C), v_step = kThreads >> (u + LOG_C);
    const bool col_ok = c_me < c_eff;
    {
        // source row of tile row v: ((base | v << lo | l) >> src_shift); src_shift is
        // 0 or equal to lo, so it is linear in v either way
        const uint64_t r0 = (base | ((uint64_t)v_first << ps.lo) | l_me) >> ps.src_shift;
        const uint64_t rstep = ((uint64_t)v_step << ps.lo) >> ps.src_shift;
        const uint64_t *g = ps.src + r0 * ps.ncols + col0 + c_me;
        const uint64_t gstep = rstep * ps.ncols;
        for (uint32_t v = v_first, e = threadIdx.x; v < rows; v += v_step, e += kThreads, g += gstep)
            tile[e] = col_ok ? *g : 0;
    }
    __syncthreads();
    for (uint32_t f = threadIdx.x; f < (rows << u); f += kThreads) {
        const uint32_t l = f >> t, e = f & (rows - 1);
        if (e + 1 < rows) tw[f] = mul_c(beta[l][31 - __clz(e + 1)], g_ntt.tab[dir][e]);
    }
    __syncthreads();

    uint32_t done = 0;
#if PG12_NTT_RADIX8
    // Three stages between barriers (radix 8: eight rows per thread, twelve
    // butterflies): stage b needs one twiddle per group, stage b + 1 two and
    // stage b + 2 four, indexed by the row bits below each stage's bit.
    // (four stages left go as two radix-4 steps rather than radix 8 and a
    // lone radix-2 stage)
    const uint32_t groups8 = (rows >> 3) << (u + LOG_C);
    while (done + 3 <= t && (!PG12_NTT_NO_R2 || t - done != 4)) {
        const uint32_t b = DIT ? done : t - 3 - done;  // lowest bit of the three
        const uint32_t m0 = (1u << b) - 1, m1 = (2u << b) - 1, m2 = (4u << b) - 1;
        const uint32_t s0 = 1u << (b + u + LOG_C), s1 = 2u << (b + u + LOG_C), s2 = 4u << (b + u + LOG_C);
        for (uint32_t p = threadIdx.x; p < groups8; p += kThreads) {
            const uint32_t lc = p & ((C << u) - 1), g = p >> (u + LOG_C);
            const uint32_t v0 = ((g >> b) << (b + 3)) | (g & m0);
            uint64_t *x = tile + ((v0 << (u + LOG_C)) + lc);
            const uint64_t *w = tw + ((lc >> LOG_C) << t);
            const uint32_t k = v0 & m0;
            uint64_t a[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = x[(i & 1) * s0 + ((i >> 1) & 1) * s1 + (i >> 2) * s2];
            const uint64_t w0 = w[m0 + k];                                  // stage b
            const uint64_t w10 = w[m1 + k], w11 = w[m1 + k + (1u << b)];    // stage b + 1
            const uint64_t w20 = w[m2 + k], w21 = w[m2 + k + (1u << b)];    // stage b + 2
            const uint64_t w22 = w[m2 + k + (2u << b)], w23 = w[m2 + k + (3u << b)];
            if (DIT) {
                bfly<1>(a[0], a[1], w0);
                bfly<1>(a[2], a[3], w0);
                bfly<1>(a[4], a[5], w0);
                bfly<1>(a[6], a[7], w0);
                bfly<1>(a[0], a[2], w10);
                bfly<1>(a[1], a[3], w11);
                bfly<1>(a[4], a[6], w10);
                bfly<1>(a[5], a[7], w11);
                bfly<1>(a[0], a[4], w20);
                bfly<1>(a[1], a[5], w21);
                bfly<1>(a[2], a[6], w22);
                bfly<1>(a[3], a[7], w23);
            } else {
                bfly<0>(a[0], a[4], w20);
                bfly<0>(a[1], a[5], w21);
                bfly<0>(a[2], a[6], w22);
                bfly<0>(a[3], a[7], w23);
                bfly<0>(a[0], a[2], w10);
                bfly<0>(a[1], a[3], w11);
                bfly<0>(a[4], a[6], w10);
                bfly<0>(a[5], a[7], w11);
                bfly<0>(a[0], a[1], w0);
                bfly<0>(a[2], a[3], w0);
                bfly<0>(a[4], a[5], w0);
                bfly<0>(a[6], a[7], w0);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) x[(i & 1) * s0 + ((i >> 1) & 1) * s1 + (i >> 2) * s2] = a[i];
        }
        __syncthreads();
        done += 3;
    }
#endif
    const uint32_t groups = (rows >> 2) << (u + LOG_C);
    while (done + 2 <= t) {
        const uint32_t b = DIT ? done : t - 2 - done;  // lower bit of the pair
        const uint32_t m0 = (1u << b) - 1, m1 = (2u << b) - 1;
        const uint32_t s0 = 1u << (b + u + LOG_C), s1 = 2u << (b + u + LOG_C);
        for (uint32_t p = threadIdx.x; p < groups; p += kThreads) {
            const uint32_t lc = p & ((C << u) - 1), g = p >> (u + LOG_C);
            const uint32_t v0 = ((g >> b) << (b + 2)) | (g & m0);
            uint64_t *x = tile + ((v0 << (u + LOG_C)) + lc);
            const uint64_t *w = tw + ((lc >> LOG_C) << t);
            uint64_t a0 = x[0], a1 = x[s0], a2 = x[s1], a3 = x[s0 + s1];
            const uint64_t wl = w[m0 + (v0 & m0)];               // stage b
            const uint64_t wh0 = w[m1 + (v0 & m1)];              // stage b + 1, rows v0, v0 + 2^(b+1)
            const uint64_t wh1 = w[m1 + (v0 & m1) + (1u << b)];  // rows v0 + 2^b, v0 + 2^b + 2^(b+1)
            if (DIT) {
                bfly<1>(a0, a1, wl);
                bfly<1>(a2, a3, wl);
                bfly<1>(a0, a2, wh0);
                bfly<1>(a1, a3, wh1);
            } else {
                bfly<0>(a0, a2, wh0);
                bfly<0>(a1, a3, wh1);
                bfly<0>(a0, a1, wl);
                bfly<0>(a2, a3, wl);
            }
            x[0] = a0;
            x[s0] = a1;
            x[s1] = a2;
            x[s0 + s1] = a3;
        }
        __syncthreads();
        done += 2;
    }
    if (done < t) {  // one radix-2 stage left: bit t - 1 (DIT) or bit 0 (DIF)
        const uint32_t b = DIT ? t - 1 : 0;
        const uint32_t m0 = (1u << b) - 1;
        const uint32_t pairs = (rows >> 1) << (u + LOG_C);
        const uint32_t s0 = 1u << (b + u + LOG_C);
        for (uint32_t p = threadIdx.x; p < pairs; p += kThreads) {
            const uint32_t lc = p & ((C << u) - 1), q = p >> (u + LOG_C);
            const uint32_t v0 = ((q >> b) << (b + 1)) | (q & m0);
            uint64_t *x = tile + ((v0 << (u + LOG_C)) + lc);
            uint64_t a0 = x[0], a1 = x[s0];
            bfly<DIT>(a0, a1, tw[((lc >> LOG_C) << t) + m0 + (v0 & m0)]);
            x[0] = a0;
            x[s0] = a1;
        }
        __syncthreads();
    }

    if (!col_ok) return;
    {
        const uint64_t r0 = base | ((uint64_t)v_first << ps.lo) | l_me;
        const uint64_t rstep = (uint64_t)v_step << ps.lo;
        uint64_t *g = ps.dst + r0 * ps.ncols + col0 + c_me;
        const uint64_t gstep = rstep * ps.ncols;
        uint64_t row = r0;
        for (uint32_t v = v_first, e = threadIdx.x; v < rows; v += v_step, e += kThreads, g += gstep, row += rstep) {
            uint64_t x = tile[e];
            if (ps.scale == 1) {
                x = mul(x, ps.scale_c);
            } else if (ps.scale == 2) {
                const uint64_t j = ps.log_n ? (uint64_t)(__brevll(row) >> (64 - ps.log_n)) : 0;
                x = mul(x, mul_c(pow_tab(g_ntt.coset, j), ps.scale_c));
            }
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
// tile plus twiddles stay within 72-96 KiB of shared memory.
uint32_t tile_bits(uint32_t log_c) { return log_c >= 3 ? (uint32_t)PG12_NTT_TILE_BITS8 : log_c == 2 ? 11u : 12u; }
uint32_t max_t(uint32_t log_c) { return tile_bits(log_c) < (uint32_t)kMaxT ? tile_bits(log_c) : (uint32_t)kMaxT; }

size_t pass_smem(uint32_t t, uint32_t u, uint32_t log_c) {
    return (((size_t)1 << (t + u + log_c)) + ((size_t)1 << (t + u))) * sizeof(uint64_t);
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
                                (int)pass_smem(tile_bits(LOG_C), 0, LOG_C));
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
    const size_t smem = pass_smem(ps.t, ps.u, lc);
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

// `bits` index bits in passes of at most `tmax` bits, as even as possible.
int split_passes(uint32_t bits, uint32_t tmax, uint32_t *t_out) {
    if (bits == 0) {
        t_out[0] = 0;
        return 1;
    }
    const uint32_t n = (bits + tmax - 1) / tmax;
    for (uint32_t k = 0; k < n; ++k) t_out[k] = bits / n + (k < bits % n ? 1u : 0u);
    return (int)n;
}

// DIF passes over all log_n bits of `dst` (first pass reads `src`).
int run_dif(const uint64_t *src, uint64_t *dst, uint32_t log_n, uint64_t ncols, bool inverse, uint32_t scale,
            uint64_t scale_c, cudaStream_t st) {
    uint32_t ts[32];
    const int np = split_passes(log_n, max_t(tile_log_c(ncols)), ts);
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
    const int np = split_passes(log_n, max_t(tile_log_c(ncols)), ts);
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
