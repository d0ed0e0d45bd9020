// Element-wise Goldilocks operations and their throughput microbenchmarks:
// the GPU counterparts of the basic functions the paper profiles one by one
// (Table 1: add, sub, reduce_128_64, square_128, mult_128, mult_72, and the
// dot products of the MDS layers; Sec. 4.3 measures them with hardware
// counters).  These use the same device arithmetic as the permutation.
#include "pg12.h"
#include "pg12_internal.h"
#include "field.cuh"
#include "poseidon.cuh"

#include <cuda_runtime.h>

#include <cstdio>

namespace pg12 {
namespace dev {

// a - b for weak a and canonical-or-weak b: a borrow is worth -2^64, i.e.
// subtract 2^32 - 1 once more (Alg. 6 for canonical operands).
__device__ __forceinline__ uint64_t sub_weak(uint64_t a, uint64_t b) {
    const uint64_t bc = canon(b);
    uint64_t d = a - bc;
    if (a < bc) d -= EPS;
    return d;
}

// Product with an operand below 2^8 (Table 1's mult_72): two 32x8 partial
// products, then the usual fold.
__device__ __forceinline__ uint64_t mul_small(uint64_t a, uint32_t m8) {
    const uint64_t lo = (uint64_t)lo32(a) * m8;  // < 2^40
    const uint64_t hi = (uint64_t)hi32(a) * m8;  // < 2^40, weight 2^32
    const u128 r = (u128)lo + ((u128)hi << 32);
    return reduce128(r);
}

__device__ __forceinline__ uint64_t apply(int op, uint64_t a, uint64_t b) {
    switch (op) {
        case PG_OP_ADD: return add_canon(a, canon(b));
        case PG_OP_SUB: return sub_weak(a, b);
        case PG_OP_MUL: return mul(a, b);
        case PG_OP_SQR: return sqr(a);
        case PG_OP_REDUCE: return reduce128(((u128)b << 64) | a);
        case PG_OP_MUL_SMALL: return mul_small(a, (uint32_t)(b & 0xFF));
        case PG_OP_SBOX: return sbox(a);
        default: return a;
    }
}

__global__ void k_field_eval(int op, const uint64_t *__restrict__ a, const uint64_t *__restrict__ b,
                             uint64_t *__restrict__ out, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = canon(apply(op, a[i], b ? b[i] : 0));
}

// Arbitrary distinct matrix entries for the dot-product benchmark (a
// SplitMix64 finaliser of the position, reduced below p).  Both 32-bit halves
// differ from entry to entry, so the compiler cannot share a partial product
// between rows.
__host__ __device__ constexpr uint64_t bench_entry(int i, int j) {
    uint64_t z = 0x9E3779B97F4A7C15ull * (uint64_t)(i * 12 + j + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (z ^ (z >> 31)) % P;
}

// The benchmark matrix, filled by the host before a dot-product run (the
// permutation also reads its matrices from the constant bank).
__constant__ uint64_t c_bench_m[12][12];

// Twelve independent chains per thread; clock64 brackets the timed loop.
template <int OP>
__global__ void __launch_bounds__(256) k_field_bench(uint64_t *out, long long *cycles, int iters) {
    uint64_t x[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) x[i] = 0x9E3779B97F4A7C15ull * (threadIdx.x + 131 * i + blockIdx.x * 7 + 1);
    const uint64_t c = 0xC3A5C85C97CB3127ull % P;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            if (OP == PG_OP_DOT12) {
                // one 12-term lazy dot product per step, writing back to cell i
                Acc A;
                acc_zero(A);
#pragma unroll
                for (int j = 0; j < 12; ++j) acc_mac(A, x[j], c_bench_m[i][j]);
                x[i] = acc_reduce(A);
            } else {
                x[i] = apply(OP, x[i], x[(i + 1) % 12] ^ c);
            }
        }
    }
    const long long t1 = clock64();
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < 12; ++i) s ^= x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Raw pipe probes (bench only): 16 independent chains of one instruction
// kind per thread, rotating operands so nothing folds at compile time.
template <int KIND>
__global__ void __launch_bounds__(256) k_pipe_bench(uint64_t *out, long long *cycles, int iters) {
    uint32_t a[16];
    uint64_t d[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        a[k] = 0x9E3779B9u * (threadIdx.x + 17 * k + 1) + blockIdx.x;
        d[k] = a[k] * 0x2545F4914F6CDD1Dull;
    }
    const uint32_t b = 0x85EBCA6Bu ^ blockIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (KIND == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(b), "r"(a[(k + 5) & 15]));
            if (KIND == 1) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(d[k]) : "r"(a[k]), "r"(b));
            if (KIND == 2) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[k]) : "r"(a[(k + 3) & 15]));
        }
        if (KIND == 1) {
#pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = (uint32_t)d[(k + 1) & 15];
        }
    }
    const long long t1 = clock64();
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k] + d[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}


// Latency chains: one warp, each operation consumes the previous result.
// The constant tables are arbitrary words (latency does not depend on them).
template <int OP>
__global__ void k_lat_bench(uint64_t *out, long long *cycles, int iters) {
    __shared__ __align__(16) DevConsts K;
    __shared__ uint64_t slots[kT * 32];
    uint64_t *w = reinterpret_cast<uint64_t *>(&K);
    for (unsigned i = threadIdx.x; i < sizeof(DevConsts) / 8; i += blockDim.x) w[i] = 0x9E3779B97F4A7C15ull * (i + 1);
    uint64_t *slot = slots + threadIdx.x;
    for (int i = 0; i < kT; ++i) slot[i * 32] = 0x100000001ull * (threadIdx.x + 7 * i + 1);
    __syncthreads();
    uint64_t x = 0x9E3779B97F4A7C15ull + threadIdx.x;
    const uint64_t y = 0x123456789ABCDEFull;
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
        if (OP == PG_OP_LAT_MUL) {
            x = mul(x, y);
        } else if (OP == PG_OP_LAT_SBOX) {
            x = sbox(x);
        } else if (OP == PG_OP_LAT_DOT12) {
            Acc A;
            acc_zero(A);
#pragma unroll
            for (int j = 0; j < kT; ++j) acc_mac(A, x + j, y + 977 * j);
            x = acc_reduce(A);
        } else if (OP == PG_OP_LAT_PERM) {
            slot[0] += x;
            permute_slot<32>(slot);
            x = slot[0];
        } else {
            x = permute_wide(x, threadIdx.x & 15, 0xFFFFFFFFu, K);
        }
    }
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[0] = t1 - t0;
    out[threadIdx.x] = x;
}

}  // namespace dev
}  // namespace pg12

using namespace pg12;

namespace {


pg_status ops_fail(pg_status s, const char *what, cudaError_t e) {
    return (pg_status)set_error(s, "%s: %s", what, cudaGetErrorString(e));
}

template <int OP>
pg_status lat_one(int sms, double *ops_per_s, double *ops_per_clk_sm) {
    (void)sms;
    const int iters = OP == PG_OP_LAT_PERM || OP == PG_OP_LAT_PERM_WIDE ? 16 : 1024;
    uint64_t *out = nullptr;
    long long *cyc = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&out, sizeof(uint64_t) * 32)) != cudaSuccess) return ops_fail(PG_ERR_OOM, "malloc", e);
    if ((e = cudaMalloc(&cyc, sizeof(long long))) != cudaSuccess) {
        cudaFree(out);
        return ops_fail(PG_ERR_OOM, "malloc", e);
    }
    dev::k_lat_bench<OP><<<1, 32>>>(out, cyc, 2);
    dev::k_lat_bench<OP><<<1, 32>>>(out, cyc, iters);
    e = cudaDeviceSynchronize();
    long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, cyc, sizeof h, cudaMemcpyDeviceToHost);
    int dev_id = 0, khz = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev_id);
    cudaFree(out);
    cudaFree(cyc);
    if (e != cudaSuccess) return ops_fail(PG_ERR_CUDA, "latency kernel", e);
    const double per_op = (double)h / iters;
    if (ops_per_clk_sm) *ops_per_clk_sm = per_op;
    if (ops_per_s) *ops_per_s = per_op > 0 ? (double)khz * 1e3 / per_op : 0.0;
    return PG_OK;
}

template <int KIND>
pg_status pipe_one(int sms, double *ops_per_s, double *ops_per_clk_sm) {
    const int grid = sms * 4, threads = 256, iters = 400;
    uint64_t *out = nullptr;
    long long *cyc = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&out, sizeof(uint64_t) * grid * threads)) != cudaSuccess) return ops_fail(PG_ERR_OOM, "malloc", e);
    if ((e = cudaMalloc(&cyc, sizeof(long long) * grid)) != cudaSuccess) {
        cudaFree(out);
        return ops_fail(PG_ERR_OOM, "malloc", e);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dev::k_pipe_bench<KIND><<<grid, threads>>>(out, cyc, 2);
    cudaEventRecord(e0);
    dev::k_pipe_bench<KIND><<<grid, threads>>>(out, cyc, iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    long long *h = new long long[grid];
    cudaMemcpy(h, cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
    double cmax = 0;
    for (int i = 0; i < grid; ++i) cmax = h[i] > cmax ? (double)h[i] : cmax;
    delete[] h;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    if (e != cudaSuccess) return ops_fail(PG_ERR_CUDA, "pipe kernel", e);
    const double ops = (double)grid * threads * iters * 16;
    if (ops_per_s) *ops_per_s = ops / (ms * 1e-3);
    if (ops_per_clk_sm) *ops_per_clk_sm = cmax > 0 ? ops / (double)sms / cmax : 0.0;
    return PG_OK;
}

template <int OP>
pg_status bench_one(int sms, double *ops_per_s, double *ops_per_clk_sm) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dev::k_field_bench<OP>, 256, 0);
    if (e != cudaSuccess || occ < 1) return ops_fail(PG_ERR_CUDA, "occupancy", e);
    const int grid = sms * occ, threads = 256;
    const int iters = OP == PG_OP_DOT12 ? 20 : (OP == PG_OP_SBOX ? 50 : 200);
    if (OP == PG_OP_DOT12) {
        uint64_t m[12][12];
        for (int i = 0; i < 12; ++i)
            for (int j = 0; j < 12; ++j) m[i][j] = dev::bench_entry(i, j);
        if ((e = cudaMemcpyToSymbol(dev::c_bench_m, m, sizeof(m))) != cudaSuccess)
            return ops_fail(PG_ERR_CUDA, "bench constants", e);
    }
    uint64_t *out = nullptr;
    long long *cyc = nullptr;
    if ((e = cudaMalloc(&out, sizeof(uint64_t) * grid * threads)) != cudaSuccess) return ops_fail(PG_ERR_OOM, "malloc", e);
    if ((e = cudaMalloc(&cyc, sizeof(long long) * grid)) != cudaSuccess) {
        cudaFree(out);
        return ops_fail(PG_ERR_OOM, "malloc", e);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dev::k_field_bench<OP><<<grid, threads>>>(out, cyc, 1);
    cudaEventRecord(e0);
    dev::k_field_bench<OP><<<grid, threads>>>(out, cyc, iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    long long *h = new long long[grid];
    cudaMemcpy(h, cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
    double cmax = 0;
    for (int i = 0; i < grid; ++i) cmax = h[i] > cmax ? (double)h[i] : cmax;
    delete[] h;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(cyc);
    if (e != cudaSuccess) return ops_fail(PG_ERR_CUDA, "bench kernel", e);
    const double ops = (double)grid * threads * iters * 12;
    if (ops_per_s) *ops_per_s = ops / (ms * 1e-3);
    if (ops_per_clk_sm) *ops_per_clk_sm = cmax > 0 ? ops / (double)sms / cmax : 0.0;
    return PG_OK;
}
}  // namespace

extern "C" {

pg_status pg_field_eval(int op, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n, void *stream) {
    if (op < PG_OP_ADD || op > PG_OP_SBOX) return (pg_status)set_error(PG_ERR_INVALID_ARG, "unknown op %d", op);
    if (n == 0) return PG_OK;
    if (!a || !out) return (pg_status)set_error(PG_ERR_INVALID_ARG, "a or out is NULL");
    const unsigned grid = (unsigned)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
    dev::k_field_eval<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(op, a, b, out, (uint64_t)n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PG_OK : ops_fail(PG_ERR_CUDA, "k_field_eval", e);
}

pg_status pg_field_bench(int op, double *ops_per_s, double *ops_per_clk_sm) {
    int dev_id = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev_id);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    if (e != cudaSuccess) return ops_fail(PG_ERR_CUDA, "device query", e);
    switch (op) {
        case PG_OP_ADD: return bench_one<PG_OP_ADD>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_SUB: return bench_one<PG_OP_SUB>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_MUL: return bench_one<PG_OP_MUL>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_SQR: return bench_one<PG_OP_SQR>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_REDUCE: return bench_one<PG_OP_REDUCE>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_MUL_SMALL: return bench_one<PG_OP_MUL_SMALL>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_SBOX: return bench_one<PG_OP_SBOX>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_DOT12: return bench_one<PG_OP_DOT12>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_PIPE_IMAD: return pipe_one<0>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_PIPE_IMAD_WIDE: return pipe_one<1>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_PIPE_IADD: return pipe_one<2>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_LAT_MUL: return lat_one<PG_OP_LAT_MUL>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_LAT_SBOX: return lat_one<PG_OP_LAT_SBOX>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_LAT_DOT12: return lat_one<PG_OP_LAT_DOT12>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_LAT_PERM: return lat_one<PG_OP_LAT_PERM>(sms, ops_per_s, ops_per_clk_sm);
        case PG_OP_LAT_PERM_WIDE: return lat_one<PG_OP_LAT_PERM_WIDE>(sms, ops_per_s, ops_per_clk_sm);
        default: return (pg_status)set_error(PG_ERR_INVALID_ARG, "unknown op %d", op);
    }
}

}  // extern "C"
