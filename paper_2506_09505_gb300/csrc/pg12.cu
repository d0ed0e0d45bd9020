// Kernels and C ABI of the GB300 Poseidon-12 / Goldilocks Merkle library.
//
//   k_permute   Alg. 1 on a batch of independent states, one thread each.
//   k_hash_rows Sec. 2.4 sponge (rate 8, capacity 4, overwrite mode) per row.
//   k_merkle    Sec. 4.2 tree build as one persistent launch: blocks pull
//               leaf tiles from a global counter, hash a tile of rows and
//               fuse the next levels in shared memory; the block that
//               completes the last child tile of a parent tile (an atomic
//               arrival counter, never a spin) goes on to build that parent
//               tile, so the upper levels start as soon as their subtree is
//               ready instead of after a grid-wide barrier.
#include "pg12.h"
#include "pg12_internal.h"
#include "poseidon.cuh"

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

namespace pg12 {
namespace dev {

// ------------------------------------------------------------- geometry
constexpr int kBlock = 256;     // threads per Merkle block
constexpr int kLeafTile = 256;  // rows per leaf tile
constexpr int kNodeTile = 512;  // child nodes consumed per node tile
constexpr int kTileOut = 32;    // outputs of a tile that is not the last one
constexpr int kMaxStages = 12;

struct StagePlan {
    uint32_t n_tiles;       // tiles in this stage
    uint32_t in_per_tile;   // rows (stage 0) or child nodes per tile
    uint32_t levels;        // tree levels written by one tile
    uint32_t in_level;      // level of the child nodes (stages >= 1)
    uint32_t counter_base;  // first arrival counter of this stage (stages >= 1)
    uint32_t fan_in;        // child tiles per tile (stages >= 1)
};

struct TreePlan {
    const uint64_t *rows;
    uint64_t *nodes;
    uint64_t n_leaves;
    uint64_t width;
    uint32_t n_stages;
    uint32_t leaf_task_begin;  // first global leaf-task index of this tree
    uint32_t counter_base;     // first arrival counter of this tree
    uint32_t vec16;            // rows can be read with 16-byte loads
    StagePlan st[kMaxStages];
};

__device__ __forceinline__ uint64_t level_off(uint64_t n, uint32_t level) {
    return 2 * n - ((2 * n) >> level);
}

// ------------------------------------------------------------- memory
__device__ __forceinline__ void ld2_nc(const uint64_t *p, uint64_t &a, uint64_t &b) {
    asm volatile("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}
__device__ __forceinline__ void ld2_cg(const uint64_t *p, uint64_t &a, uint64_t &b) {
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}
__device__ __forceinline__ void st2(uint64_t *p, uint64_t a, uint64_t b) {
    asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

// Chunk c of a row (8 elements, zero-filled past the row's end).
__device__ __forceinline__ void load_chunk(const uint64_t *row, uint64_t w, uint64_t c, bool vec16,
                                           uint64_t (&ch)[kRate]) {
    const uint64_t base = c * kRate;
    if (base + kRate <= w) {
        if (vec16) {
#pragma unroll
            for (int i = 0; i < kRate; i += 2) ld2_nc(row + base + i, ch[i], ch[i + 1]);
        } else {
#pragma unroll
            for (int i = 0; i < kRate; ++i) ch[i] = __ldg(row + base + i);
        }
    } else {
#pragma unroll
        for (int i = 0; i < kRate; ++i) ch[i] = (base + i < w) ? __ldg(row + base + i) : 0ull;
    }
}

// Overwrite-mode sponge over one row; digest is canonical.
__device__ __forceinline__ void sponge_row(const uint64_t *row, uint64_t w, bool vec16,
                                           uint64_t (&d)[kDigest]) {
    uint64_t x[kT];
#pragma unroll
    for (int i = 0; i < kT; ++i) x[i] = 0;
    const uint64_t chunks = w == 0 ? 1 : (w + kRate - 1) / kRate;
    uint64_t nxt[kRate];
    load_chunk(row, w, 0, vec16, nxt);
    for (uint64_t c = 0; c < chunks; ++c) {
#pragma unroll
        for (int i = 0; i < kRate; ++i) x[i] = nxt[i];
        if (c + 1 < chunks) load_chunk(row, w, c + 1, vec16, nxt);
        permute(x);
    }
#pragma unroll
    for (int i = 0; i < kDigest; ++i) d[i] = canon(x[i]);
}

// ------------------------------------------------------------- kernels
__global__ void __launch_bounds__(128) k_permute(uint64_t *__restrict__ st, uint64_t n, int vec16) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        uint64_t *p = st + kT * k;
        uint64_t x[kT];
        if (vec16) {
#pragma unroll
            for (int i = 0; i < kT; i += 2) ld2_nc(p + i, x[i], x[i + 1]);
        } else {
#pragma unroll
            for (int i = 0; i < kT; ++i) x[i] = p[i];
        }
        permute(x);
        if (vec16) {
#pragma unroll
            for (int i = 0; i < kT; i += 2) st2(p + i, canon(x[i]), canon(x[i + 1]));
        } else {
#pragma unroll
            for (int i = 0; i < kT; ++i) p[i] = canon(x[i]);
        }
    }
}

__global__ void __launch_bounds__(128) k_hash_rows(const uint64_t *__restrict__ rows, uint64_t n,
                                                   uint64_t w, int vec16, uint64_t *__restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        uint64_t d[kDigest];
        sponge_row(rows + r * w, w, vec16 != 0, d);
        st2(out + kDigest * r, d[0], d[1]);
        st2(out + kDigest * r + 2, d[2], d[3]);
    }
}

// One tile: its first level from rows (stage 0) or from child nodes in
// global memory, then the following levels from shared memory.  Every
// permutation of the tile goes through a single call site (several inlined
// copies of the permutation would multiply its register footprint).
__device__ void run_tile(const TreePlan &tp, uint32_t s, uint32_t tile,
                         uint64_t (&buf)[2][kBlock][kDigest]) {
    const int t = threadIdx.x;
    const StagePlan st = tp.st[s];
    const uint64_t n = tp.n_leaves;
    const uint64_t w = tp.width;
    const bool vec16 = tp.vec16 != 0;
    // first level: stage 0 hashes rows, later stages hash child pairs
    uint32_t cnt = s == 0 ? st.in_per_tile : st.in_per_tile / 2;
    uint32_t level = s == 0 ? 0 : st.in_level + 1;
    const uint64_t row_chunks = w == 0 ? 1 : (w + kRate - 1) / kRate;
    int b = 0;
    for (uint32_t k = 0; k < st.levels; ++k) {
        if (k > 0) {
            __syncthreads();
            cnt /= 2;
            ++level;
        }
        if (t < (int)cnt) {
            const bool sponge = (s == 0 && k == 0);
            const uint64_t nperm = sponge ? row_chunks : 1;
            const uint64_t *row = tp.rows + ((uint64_t)tile * cnt + t) * w;
            const uint64_t *kids = nullptr;
            if (s != 0 && k == 0)
                kids = tp.nodes + kDigest * (level_off(n, st.in_level) + (uint64_t)tile * st.in_per_tile + 2 * t);
            uint64_t x[kT];
#pragma unroll
            for (int i = 0; i < kT; ++i) x[i] = 0;
            for (uint64_t c = 0; c < nperm; ++c) {
                if (sponge) {
                    uint64_t ch[kRate];
                    load_chunk(row, w, c, vec16, ch);
#pragma unroll
                    for (int i = 0; i < kRate; ++i) x[i] = ch[i];
                } else if (k == 0) {
#pragma unroll
                    for (int i = 0; i < 2 * kDigest; i += 2) ld2_cg(kids + i, x[i], x[i + 1]);
                } else {
#pragma unroll
                    for (int i = 0; i < kDigest; ++i) {
                        x[i] = buf[b][2 * t][i];
                        x[kDigest + i] = buf[b][2 * t + 1][i];
                    }
                }
                permute(x);
            }
            uint64_t d[kDigest];
#pragma unroll
            for (int i = 0; i < kDigest; ++i) d[i] = canon(x[i]);
            uint64_t *dst = tp.nodes + kDigest * (level_off(n, level) + (uint64_t)tile * cnt + t);
            st2(dst, d[0], d[1]);
            st2(dst + 2, d[2], d[3]);
            const int ob = k == 0 ? 0 : (b ^ 1);
#pragma unroll
            for (int i = 0; i < kDigest; ++i) buf[ob][t][i] = d[i];
        }
        if (k > 0) b ^= 1;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBlock) k_merkle(const TreePlan *__restrict__ plans, uint32_t n_trees,
                                                   uint32_t total_tasks, uint32_t *__restrict__ counters,
                                                   uint32_t *__restrict__ next_task) {
    __shared__ uint64_t buf[2][kBlock][kDigest];
    __shared__ uint32_t s_task, s_go;
    const int t = threadIdx.x;
    for (;;) {
        if (t == 0) s_task = atomicAdd(next_task, 1u);
        __syncthreads();
        const uint32_t task = s_task;
        __syncthreads();
        if (task >= total_tasks) return;
        uint32_t lo = 0, hi = n_trees - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) / 2;
            if (plans[mid].leaf_task_begin <= task) lo = mid;
            else hi = mid - 1;
        }
        const TreePlan &tp = plans[lo];
        uint32_t tile = task - tp.leaf_task_begin;
        run_tile(tp, 0, tile, buf);
        for (uint32_t s = 1; s < tp.n_stages; ++s) {
            const uint32_t fan = tp.st[s].fan_in;
            const uint32_t parent = tile / fan;
            __threadfence();  // this tile's node writes before the arrival
            __syncthreads();
            if (t == 0)
                s_go = (atomicAdd(&counters[tp.counter_base + tp.st[s].counter_base + parent], 1u) == fan - 1);
            __syncthreads();
            if (!s_go) break;
            __threadfence();  // the siblings' writes are visible from here on
            tile = parent;
            run_tile(tp, s, tile, buf);
        }
    }
}

}  // namespace dev

// ================================================================ host side
namespace {

struct Context {
    bool params_ready = false;
    PlainParams plain;
    OptParams opt;
    bool init = false;
    int device = -1;
    int sms = 0;
    int merkle_blocks_per_sm = 0;
    int permute_blocks_per_sm = 0;
    uint8_t *ws = nullptr;  // device workspace
    size_t ws_bytes = 0;
};
Context g;
std::mutex g_mu;
char g_err[512] = "";

pg_status fail(pg_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

#define PG_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(PG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr size_t kWorkspaceBytes = 16u << 20;  // counters + tree plans
constexpr size_t kPlanBytes = 4u << 20;        // first part: plans; rest: counters

pg_status ensure_params() {
    if (g.params_ready) return PG_OK;
    host::generate_plain(g.plain);
    if (!host::derive_optimized(g.plain, g.opt))
        return fail(PG_ERR_PARAMS, "parameter set pg12_v1: sparse rewrite failed (singular block)");
    g.params_ready = true;
    return PG_OK;
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }
uint32_t log2u(uint64_t x) {
    uint32_t l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

// Stage geometry of one tree (see k_merkle).  Returns false if the tree
// needs more stages than the plan holds.
bool plan_tree(dev::TreePlan &tp, const uint64_t *rows, uint64_t n, uint64_t w, uint64_t *nodes,
               uint32_t leaf_task_begin, uint32_t counter_base, uint32_t &n_counters) {
    tp.rows = rows;
    tp.nodes = nodes;
    tp.n_leaves = n;
    tp.width = w;
    tp.leaf_task_begin = leaf_task_begin;
    tp.counter_base = counter_base;
    tp.vec16 = ((w % 2) == 0 && (reinterpret_cast<uintptr_t>(rows) % 16) == 0) ? 1u : 0u;
    n_counters = 0;
    uint32_t s = 0;
    // stage 0: leaf tiles
    {
        dev::StagePlan &st = tp.st[0];
        st.in_per_tile = (uint32_t)(n < (uint64_t)dev::kLeafTile ? n : dev::kLeafTile);
        st.n_tiles = (uint32_t)(n / st.in_per_tile);
        st.in_level = 0;
        st.counter_base = 0;
        st.fan_in = 0;
        st.levels = st.n_tiles == 1 ? log2u(st.in_per_tile) + 1 : log2u(st.in_per_tile / dev::kTileOut) + 1;
    }
    uint64_t out_total = (uint64_t)tp.st[0].n_tiles * (tp.st[0].in_per_tile >> (tp.st[0].levels - 1));
    uint32_t out_level = tp.st[0].levels - 1;
    uint32_t prev_out = tp.st[0].in_per_tile >> (tp.st[0].levels - 1);
    s = 1;
    while (tp.st[s - 1].n_tiles > 1) {
        if (s >= (uint32_t)dev::kMaxStages) return false;
        dev::StagePlan &st = tp.st[s];
        st.in_per_tile = (uint32_t)(out_total < (uint64_t)dev::kNodeTile ? out_total : dev::kNodeTile);
        st.n_tiles = (uint32_t)(out_total / st.in_per_tile);
        st.in_level = out_level;
        st.fan_in = st.in_per_tile / prev_out;
        st.counter_base = n_counters;
        n_counters += st.n_tiles;
        st.levels = st.n_tiles == 1 ? log2u(st.in_per_tile) : log2u(st.in_per_tile / dev::kTileOut);
        prev_out = st.in_per_tile >> st.levels;
        out_total = (uint64_t)st.n_tiles * prev_out;
        out_level = st.in_level + st.levels;
        ++s;
    }
    tp.n_stages = s;
    return true;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

pg_status require_init() {
    if (!g.init) return fail(PG_ERR_NOT_INIT, "pg_init() has not been called");
    return PG_OK;
}

}  // namespace
}  // namespace pg12

using namespace pg12;

extern "C" {

const char *pg_version(void) { return "pg12 1.0 sm_103a"; }

const char *pg_last_error(void) { return g_err; }

pg_status pg_params_export(uint64_t *rc, uint64_t *mds) {
    std::lock_guard<std::mutex> lk(g_mu);
    pg_status s = ensure_params();
    if (s != PG_OK) return s;
    if (rc) std::memcpy(rc, g.plain.rc, sizeof g.plain.rc);
    if (mds) std::memcpy(mds, g.plain.mds, sizeof g.plain.mds);
    return PG_OK;
}

pg_status pg_params_export_optimized(uint64_t *full_rc, uint64_t *mds, uint64_t *pre, uint64_t *part_rc,
                                     uint64_t *part_v, uint64_t *part_w) {
    std::lock_guard<std::mutex> lk(g_mu);
    pg_status s = ensure_params();
    if (s != PG_OK) return s;
    if (full_rc) std::memcpy(full_rc, g.opt.full_rc, sizeof g.opt.full_rc);
    if (mds) std::memcpy(mds, g.opt.mds, sizeof g.opt.mds);
    if (pre) std::memcpy(pre, g.opt.pre, sizeof g.opt.pre);
    if (part_rc) std::memcpy(part_rc, g.opt.part_rc, sizeof g.opt.part_rc);
    if (part_v) std::memcpy(part_v, g.opt.part_v, sizeof g.opt.part_v);
    if (part_w) std::memcpy(part_w, g.opt.part_w, sizeof g.opt.part_w);
    return PG_OK;
}

pg_status pg_init(int device, const char *params_path) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (params_path != nullptr) return fail(PG_ERR_PARAMS, "only the built-in parameter set pg12_v1 is supported");
    if (g.init && g.device == device) return PG_OK;
    if (g.init) return fail(PG_ERR_INVALID_ARG, "already initialised on device %d", g.device);
    pg_status s = ensure_params();
    if (s != PG_OK) return s;
    int ndev = 0;
    PG_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(PG_ERR_INVALID_ARG, "device %d out of range (%d)", device, ndev);
    PG_CUDA(cudaSetDevice(device));
    PG_CUDA(cudaMemcpyToSymbol(dev::c_opt, &g.opt, sizeof(OptParams)));
    PG_CUDA(cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, device));
    PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.merkle_blocks_per_sm, dev::k_merkle, dev::kBlock, 0));
    PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g.permute_blocks_per_sm, dev::k_permute, 128, 0));
    if (g.merkle_blocks_per_sm < 1 || g.permute_blocks_per_sm < 1)
        return fail(PG_ERR_CUDA, "kernels cannot be resident (occupancy 0)");
    void *ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, kWorkspaceBytes);
    if (e != cudaSuccess) return fail(PG_ERR_OOM, "workspace cudaMalloc(%zu): %s", kWorkspaceBytes, cudaGetErrorString(e));
    g.ws = static_cast<uint8_t *>(ws);
    g.ws_bytes = kWorkspaceBytes;
    g.device = device;
    g.init = true;
    return PG_OK;
}

pg_status pg_shutdown(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g.init) return PG_OK;
    cudaSetDevice(g.device);
    if (g.ws) cudaFree(g.ws);
    g.ws = nullptr;
    g.init = false;
    g.device = -1;
    return PG_OK;
}

pg_status pg_permute_batch(uint64_t *states, size_t n, void *stream) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    if (n == 0) return PG_OK;
    if (!states) return fail(PG_ERR_INVALID_ARG, "states is NULL");
    if (reinterpret_cast<uintptr_t>(states) % 8) return fail(PG_ERR_INVALID_ARG, "states not 8-byte aligned");
    const int vec16 = (reinterpret_cast<uintptr_t>(states) % 16) == 0;
    const uint64_t want = (n + 127) / 128;
    const uint64_t cap = (uint64_t)g.sms * g.permute_blocks_per_sm * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    dev::k_permute<<<grid, 128, 0, as_stream(stream)>>>(states, (uint64_t)n, vec16);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

pg_status pg_hash_rows(const uint64_t *rows, size_t n_rows, size_t width, uint64_t *digests, void *stream) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    if (width == 0) return fail(PG_ERR_INVALID_ARG, "width must be >= 1");
    if (n_rows == 0) return PG_OK;
    if (!rows || !digests) return fail(PG_ERR_INVALID_ARG, "rows or digests is NULL");
    if (reinterpret_cast<uintptr_t>(rows) % 8) return fail(PG_ERR_INVALID_ARG, "rows not 8-byte aligned");
    if (reinterpret_cast<uintptr_t>(digests) % 16) return fail(PG_ERR_INVALID_ARG, "digests not 16-byte aligned");
    const int vec16 = (width % 2 == 0) && (reinterpret_cast<uintptr_t>(rows) % 16) == 0;
    const uint64_t want = (n_rows + 127) / 128;
    const uint64_t cap = (uint64_t)g.sms * g.permute_blocks_per_sm * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    dev::k_hash_rows<<<grid, 128, 0, as_stream(stream)>>>(rows, (uint64_t)n_rows, (uint64_t)width, vec16, digests);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

pg_status pg_merkle_build(const uint64_t *rows, size_t n_leaves, size_t width, uint64_t *nodes, uint64_t *root_out,
                          void *stream) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    if (!rows || !nodes) return fail(PG_ERR_INVALID_ARG, "rows or nodes is NULL");
    if (width == 0) return fail(PG_ERR_INVALID_ARG, "width must be >= 1");
    if (!is_pow2(n_leaves)) return fail(PG_ERR_NOT_POW2, "n_leaves=%zu is not a power of two", n_leaves);
    if (n_leaves > (1ull << 31)) return fail(PG_ERR_INVALID_ARG, "n_leaves=%zu above 2^31", n_leaves);
    if (reinterpret_cast<uintptr_t>(rows) % 8) return fail(PG_ERR_INVALID_ARG, "rows not 8-byte aligned");
    if (reinterpret_cast<uintptr_t>(nodes) % 16) return fail(PG_ERR_INVALID_ARG, "nodes not 16-byte aligned");
    dev::TreePlan tp;
    std::memset(&tp, 0, sizeof tp);
    uint32_t n_counters = 0;
    if (!plan_tree(tp, rows, n_leaves, width, nodes, 0, 0, n_counters))
        return fail(PG_ERR_INVALID_ARG, "tree needs too many stages");
    const size_t counter_bytes = sizeof(uint32_t) * (1 + n_counters);
    if (sizeof(tp) > kPlanBytes || counter_bytes > g.ws_bytes - kPlanBytes)
        return fail(PG_ERR_OOM, "workspace too small for %zu leaves", n_leaves);
    cudaStream_t st = as_stream(stream);
    auto *d_plan = reinterpret_cast<dev::TreePlan *>(g.ws);
    auto *d_counters = reinterpret_cast<uint32_t *>(g.ws + kPlanBytes);
    PG_CUDA(cudaMemcpyAsync(d_plan, &tp, sizeof tp, cudaMemcpyHostToDevice, st));
    PG_CUDA(cudaMemsetAsync(d_counters, 0, counter_bytes, st));
    const uint32_t tasks = tp.st[0].n_tiles;
    const uint32_t cap = (uint32_t)(g.sms * g.merkle_blocks_per_sm);
    const unsigned grid = tasks < cap ? tasks : cap;
    dev::k_merkle<<<grid, dev::kBlock, 0, st>>>(d_plan, 1u, tasks, d_counters + 1, d_counters);
    PG_CUDA(cudaGetLastError());
    if (root_out) {
        PG_CUDA(cudaMemcpyAsync(root_out, nodes + 4 * (2 * n_leaves - 2), 32, cudaMemcpyDeviceToHost, st));
        PG_CUDA(cudaStreamSynchronize(st));
    }
    return PG_OK;
}

}  // extern "C"
