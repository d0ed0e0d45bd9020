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
// Everything runs as passes of one kernel.  A block loads the 2^t rows
// (t <= 10) of up to eight columns whose row indices differ only in bits
// [lo, lo + t), performs the t radix-2 stages of those bits in shared memory
// and stores the rows back, so a transform of 2^L rows reads and writes its
// data ceil(L / 10) times.
//   DIF (Gentleman-Sande) stages: natural order in, bit-reversed order out;
//   DIT (Cooley-Tukey) stages: bit-reversed order in, natural order out.
// Stage of bit q pairs rows i and i + 2^q (bit q of i clear) with twiddle
// w_{q+1}^(i mod 2^q).  Within a block the low part (i mod 2^lo) is fixed, so
// the twiddles of stage lo + b are beta_b * w_{b+1}^k, k < 2^b, with
// beta_b = w_{lo+b+1}^(i mod 2^lo): one power per block, then one product per
// twiddle from a shared table of the first 2^10 - 1 powers.
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
constexpr int kTileLog = 10;     // rows of one pass tile
constexpr int kCols = 8;         // columns of one pass tile
constexpr int kThreads = 256;
constexpr int kRootTab = (1 << kTileLog) - 1;  // w_{b+1}^k at index 2^b - 1 + k
constexpr int kCosetTab = 1024;                // 7^(j), split in three 10-bit digits
constexpr uint64_t kShift = 7;                 // generator and LDE coset shift

struct Consts {
    uint64_t root[2][33];            // [0] w_k = 7^((p-1)/2^k), [1] its inverse
    uint64_t tab[2][kRootTab];       // [dir][2^b - 1 + k] = w_{b+1}^k (dir 1: inverse roots)
    uint64_t coset[3][kCosetTab];    // [d][m] = 7^(m 2^(10 d))
};
__device__ Consts g_ntt;

// canonical in, canonical out
__device__ __forceinline__ uint64_t add_c(uint64_t a, uint64_t b) { return canon(dev::add_canon(a, b)); }
__device__ __forceinline__ uint64_t sub_c(uint64_t a, uint64_t b) { return a >= b ? a - b : a - b + P; }
__device__ __forceinline__ uint64_t mul_c(uint64_t a, uint64_t b) { return canon(mul(a, b)); }

__device__ __forceinline__ uint64_t pow_c(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = mul_c(r, a);
        a = mul_c(a, a);
        e >>= 1;
    }
    return r;
}

struct Pass {
    const uint64_t *src;  // rows read (row i of the pass reads src row i >> src_shift)
    uint64_t *dst;        // rows written (may equal src)
    uint64_t ncols;
    uint64_t scale_c;     // scale 1 and 2: constant factor (n^-1)
    uint32_t log_n;       // the transform has 2^log_n rows
    uint32_t lo, t;       // row-index bits [lo, lo + t)
    uint32_t dit;         // 0: DIF stages (top bit first), 1: DIT stages (bit lo first)
    uint32_t inverse;     // inverse roots
    uint32_t src_shift;
    uint32_t scale;       // 0: none; 1: times scale_c; 2: times scale_c * 7^bitrev(row)
    uint32_t pad;
};

template <int DIT>
__global__ void __launch_bounds__(kThreads) k_ntt_pass(const Pass ps) {
    extern __shared__ uint64_t sm[];
    const uint32_t t = ps.t;
    const uint32_t rows = 1u << t;
    uint64_t *tile = sm;                      // [rows][kCols]
    uint64_t *tw = sm + (size_t)rows * kCols; // [rows - 1]
    __shared__ uint64_t beta[kTileLog + 1];

    const uint64_t chunks = (ps.ncols + kCols - 1) / kCols;
    const uint64_t outer = blockIdx.x / chunks;
    const uint64_t col0 = (blockIdx.x % chunks) * kCols;
    const uint32_t C = (uint32_t)((ps.ncols - col0) < (uint64_t)kCols ? (ps.ncols - col0) : (uint64_t)kCols);
    const uint64_t low = outer & ((1ull << ps.lo) - 1);
    const uint64_t high = outer >> ps.lo;
    const uint64_t base = (high << (ps.lo + t)) | low;
    const uint32_t dir = ps.inverse ? 1u : 0u;

    if (threadIdx.x == 0 && t > 0) {
        uint64_t b = pow_c(g_ntt.root[dir][ps.lo + t], low);
        for (int k = (int)t - 1; k >= 0; --k) {
            beta[k] = b;
            b = mul_c(b, b);
        }
    }
    for (uint32_t e = threadIdx.x; e < rows * C; e += kThreads) {
        const uint32_t v = e / C, c = e - v * C;
        const uint64_t row = base | ((uint64_t)v << ps.lo);
        const uint64_t x = ps.src[(row >> ps.src_shift) * ps.ncols + col0 + c];
        tile[v * kCols + c] = canon(x);
    }
    __syncthreads();
    for (uint32_t e = threadIdx.x; e + 1 < rows; e += kThreads) {
        const uint32_t b = 31 - __clz(e + 1);
        tw[e] = mul_c(beta[b], g_ntt.tab[dir][e]);
    }
    __syncthreads();

    const uint32_t pairs = (rows >> 1) * C;
    for (uint32_t s = 0; s < t; ++s) {
        const uint32_t b = DIT ? s : t - 1 - s;
        const uint32_t mask = (1u << b) - 1;
        for (uint32_t p = threadIdx.x; p < pairs; p += kThreads) {
            const uint32_t q = p / C, c = p - q * C;
            const uint32_t v0 = ((q >> b) << (b + 1)) | (q & mask);
            const uint32_t v1 = v0 | (1u << b);
            const uint64_t w = tw[mask + (v0 & mask)];
            const uint64_t x0 = tile[v0 * kCols + c], x1 = tile[v1 * kCols + c];
            if (DIT) {
                const uint64_t y = mul_c(x1, w);
                tile[v0 * kCols + c] = add_c(x0, y);
                tile[v1 * kCols + c] = sub_c(x0, y);
            } else {
                tile[v0 * kCols + c] = add_c(x0, x1);
                tile[v1 * kCols + c] = mul_c(sub_c(x0, x1), w);
            }
        }
        __syncthreads();
    }

    for (uint32_t e = threadIdx.x; e < rows * C; e += kThreads) {
        const uint32_t v = e / C, c = e - v * C;
        const uint64_t row = base | ((uint64_t)v << ps.lo);
        uint64_t x = tile[v * kCols + c];
        if (ps.scale == 1) {
            x = mul_c(x, ps.scale_c);
        } else if (ps.scale == 2) {
            const uint64_t j = ps.log_n ? (uint64_t)(__brevll(row) >> (64 - ps.log_n)) : 0;
            const uint64_t f = mul_c(mul_c(g_ntt.coset[0][j & 1023], g_ntt.coset[1][(j >> 10) & 1023]),
                                     mul_c(g_ntt.coset[2][(j >> 20) & 1023], ps.scale_c));
            x = mul_c(x, f);
        }
        ps.dst[row * ps.ncols + col0 + c] = x;
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

size_t pass_smem(uint32_t t) { return ((size_t)(1u << t) * kCols + (1u << t)) * sizeof(uint64_t); }

bool g_attr_set[64];

// Launches one pass; the grid is 2^(log_n - t) row groups x column chunks.
int launch_pass(const Pass &ps, cudaStream_t st) {
    const uint64_t chunks = (ps.ncols + kCols - 1) / kCols;
    const uint64_t blocks = (1ull << (ps.log_n - ps.t)) * chunks;
    if (blocks > 0x7FFFFFFFull) return set_error(PG_ERR_INVALID_ARG, "NTT pass needs %llu blocks", (unsigned long long)blocks);
    const size_t smem = pass_smem(ps.t);
    int device = 0;
    cudaGetDevice(&device);
    if (device >= 0 && device < 64 && !g_attr_set[device]) {
        const size_t max_smem = pass_smem(kTileLog);
        cudaError_t e1 = cudaFuncSetAttribute(k_ntt_pass<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
        cudaError_t e2 = cudaFuncSetAttribute(k_ntt_pass<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem);
        if (e1 != cudaSuccess || e2 != cudaSuccess)
            return set_error(PG_ERR_CUDA, "NTT shared-memory attribute: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        g_attr_set[device] = true;
    }
    ProfScope prof(kIdNttPass, st, 0);
    if (ps.dit) k_ntt_pass<1><<<(unsigned)blocks, kThreads, smem, st>>>(ps);
    else k_ntt_pass<0><<<(unsigned)blocks, kThreads, smem, st>>>(ps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PG_ERR_CUDA, "k_ntt_pass: %s", cudaGetErrorString(e));
    return PG_OK;
}

// Bits [lo0, lo0 + bits) in passes of at most kTileLog bits, as even as possible.
int split_passes(uint32_t bits, uint32_t *t_out) {
    const uint32_t n = (bits + kTileLog - 1) / kTileLog;
    for (uint32_t k = 0; k < n; ++k) t_out[k] = bits / n + (k < bits % n ? 1u : 0u);
    return (int)n;
}

// DIF passes over all log_n bits of `dst` (first pass reads `src`).
int run_dif(const uint64_t *src, uint64_t *dst, uint32_t log_n, uint64_t ncols, bool inverse, uint32_t scale,
            uint64_t scale_c, cudaStream_t st) {
    uint32_t ts[8];
    const int np = log_n ? split_passes(log_n, ts) : 1;
    if (!log_n) ts[0] = 0;
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
        for (int b = 0; b < kTileLog; ++b) {
            uint64_t x = 1;
            for (int k = 0; k < (1 << b); ++k) {
                h.tab[dir][(1 << b) - 1 + k] = x;
                x = host::fp_mul(x, h.root[dir][b + 1]);
            }
        }
    for (int d = 0; d < 3; ++d) {
        const uint64_t step = host_pow(kShift, 1ull << (10 * d));
        uint64_t x = 1;
        for (int m = 0; m < kCosetTab; ++m) {
            h.coset[d][m] = x;
            x = host::fp_mul(x, step);
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
    uint32_t ts[8];
    int np = log_n ? split_passes(log_n, ts) : 1;
    if (!log_n) ts[0] = 0;
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
        s = launch_pass(ps, st);
        if (s != PG_OK) return (pg_status)s;
        lo += ts[k];
    }
    return PG_OK;
}

}  // extern "C"
