// Kernels and C ABI of the GB300 Poseidon-12 / Goldilocks Merkle library.
//
//   k_permute   Alg. 1 on a batch of independent states, one thread each.
//   k_hash_rows Sec. 2.4 sponge (rate 8, capacity 4, overwrite mode) per row.
//   k_merkle_level  one tree level, one thread per node (a node is the
//               sponge of its children's eight words).
//   k_merkle    Sec. 4.2 persistent tree kernel: warps pull 32-leaf tasks
//               from a global counter and hash those rows; up to a plan's
//               climb limit, the warp that completes the second of two
//               sibling 32-node groups (an atomic arrival counter, never a
//               spin) goes on to hash their 32 parents.  Single trees use it
//               for the leaves only (then one launch per level); batches
//               climb to every tree's root.
//   k_merkle_top / k_merkle_top_leaf
//               the levels with few nodes, 16 lanes per state (latency form).
//   k_merkle_top_tail
//               every level of at most 64 nodes up to the root in one launch
//               of an 8-block cluster, a cluster barrier between levels.
//   k_merkle_open / k_merkle_verify  authentication paths (Sec. 2.4).
// The level launches of a single-tree build use programmatic dependent
// launch (pdl_trigger / pdl_wait below).
#include "pg12.h"
#include "pg12_internal.h"
#include "poseidon.cuh"
#include "tc_perm.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

namespace pg12 {
namespace dev {

// ------------------------------------------------------------- geometry
constexpr int kBlock = 256;     // threads per Merkle block (8 independent warps)
constexpr int kWarpNodes = 32;  // nodes of one level hashed by one warp task
#ifndef PG12_MERKLE_MIN_BLOCKS
// resident 256-thread blocks per SM the register budget of k_merkle targets:
// 4 caps it at 64 registers (32 warps per SM; measured 0.75% faster together
// with PG12_PARTIAL_PAIRS than 3 blocks at 76 registers)
#define PG12_MERKLE_MIN_BLOCKS 4
#endif
constexpr int kMaxLevels = 40;

// One tree of a build.  A "task" is 32 consecutive nodes of one level,
// hashed by one warp (one node per lane).  Level l has ceil((N>>l)/32)
// tasks; task u of level l >= 1 needs tasks 2u and 2u+1 of level l-1.
struct TreePlan {
    const uint64_t *rows;
    uint64_t *nodes;
    uint64_t n_leaves;
    uint64_t width;
    uint32_t log_n;
    uint32_t leaf_task_begin;  // first global leaf-task index of this tree
    uint32_t counter_base;     // first arrival counter of this tree
    uint32_t vec16;            // rows can be read with 16-byte loads
    uint32_t climb_limit;      // highest level the persistent kernel builds
    uint32_t *done_flag;       // set to 1 once the root is stored (NULL = none)
    uint32_t level_counter[kMaxLevels];  // counter offset of level l's tasks (l >= 1)
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

// The same, through L2 only: for rows written while the kernel runs.
__device__ __forceinline__ void load_chunk_cg(const uint64_t *row, uint64_t w, uint64_t c, bool vec16,
                                              uint64_t (&ch)[kRate]) {
    const uint64_t base = c * kRate;
    if (base + kRate <= w && vec16) {
#pragma unroll
        for (int i = 0; i < kRate; i += 2) ld2_cg(row + base + i, ch[i], ch[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < kRate; ++i) ch[i] = (base + i < w) ? __ldcg(row + base + i) : 0ull;
    }
}

// Overwrite-mode sponge over one row in the thread's state slot; returns
// with the (weak) final state in the slot.
template <int S, int MDS>
__device__ __forceinline__ void sponge_slot(const uint64_t *row, uint64_t w, bool vec16, uint64_t *slot) {
#pragma unroll
    for (int i = kRate; i < kT; ++i) slot[i * S] = 0;
    const uint64_t chunks = w == 0 ? 1 : (w + kRate - 1) / kRate;
    for (uint64_t c = 0; c < chunks; ++c) {
        uint64_t ch[kRate];
        load_chunk(row, w, c, vec16, ch);
#pragma unroll
        for (int i = 0; i < kRate; ++i) slot[i * S] = ch[i];
        permute_slot<S, MDS>(slot, c == 0, c + 1 == chunks);
    }
}

// ------------------------------------------------------------- kernels
constexpr int kSmallBlock = 128;

// Programmatic dependent launch.  The level kernels of a tree are launched
// with programmatic stream serialisation: each may be scheduled while the
// kernel before it is still running, once every block of that kernel has
// executed pdl_trigger().  Until pdl_wait() returns it only copies the
// constant tables (never written during a build); pdl_wait() returns when
// the kernel before it has completed and its stores are visible.  For a
// kernel launched without the attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <int MDS>
__global__ void __launch_bounds__(kSmallBlock) k_permute(uint64_t *__restrict__ st, uint64_t n, int vec16) {
    __shared__ uint64_t slots[kT * kSmallBlock];
    uint64_t *slot = slots + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        uint64_t *p = st + kT * k;
        if (vec16) {
#pragma unroll
            for (int i = 0; i < kT; i += 2) {
                uint64_t a, b;
                ld2_nc(p + i, a, b);
                slot[i * kSmallBlock] = a;
                slot[(i + 1) * kSmallBlock] = b;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kT; ++i) slot[i * kSmallBlock] = p[i];
        }
        permute_slot<kSmallBlock, MDS>(slot);
        if (vec16) {
#pragma unroll
            for (int i = 0; i < kT; i += 2) st2(p + i, canon(slot[i * kSmallBlock]), canon(slot[(i + 1) * kSmallBlock]));
        } else {
#pragma unroll
            for (int i = 0; i < kT; ++i) p[i] = canon(slot[i * kSmallBlock]);
        }
    }
}

template <int MDS>
__global__ void __launch_bounds__(kSmallBlock) k_hash_rows(const uint64_t *__restrict__ rows, uint64_t n,
                                                           uint64_t w, int vec16, uint64_t *__restrict__ out) {
    __shared__ uint64_t slots[kT * kSmallBlock];
    uint64_t *slot = slots + threadIdx.x;
    pdl_trigger();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        sponge_slot<kSmallBlock, MDS>(rows + r * w, w, vec16 != 0, slot);
        st2(out + kDigest * r, canon(slot[0]), canon(slot[kSmallBlock]));
        st2(out + kDigest * r + 2, canon(slot[2 * kSmallBlock]), canon(slot[3 * kSmallBlock]));
    }
}

// One tree level, one thread per node: node k is the sponge of the eight
// words of children 2k and 2k+1 (contiguous in the level below, 16-byte
// aligned), i.e. perm([L, R, 0^4])[0..3].
template <int MDS>
__global__ void __launch_bounds__(kSmallBlock) k_merkle_level(const uint64_t *__restrict__ below, uint64_t count,
                                                              uint64_t *__restrict__ here) {
    __shared__ uint64_t slots[kT * kSmallBlock];
    uint64_t *slot = slots + threadIdx.x;
    pdl_trigger();
    pdl_wait();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        sponge_slot<kSmallBlock, MDS>(below + 2 * kDigest * k, 2 * kDigest, true, slot);
        st2(here + kDigest * k, canon(slot[0]), canon(slot[kSmallBlock]));
        st2(here + kDigest * k + 2, canon(slot[2 * kSmallBlock]), canon(slot[3 * kSmallBlock]));
    }
}

// ------------------------------------------------- tensor-core kernels
// Persistent kernels of kTcGroups groups of 128 threads (one CTA per SM:
// its digit tables (124 KB) and the groups' A operands take 225 KB of shared
// memory, its groups 128 columns of tensor memory each; every thread keeps
// its state in registers).
// Group q of CTA c takes units c * kTcGroups + q, then every
// gridDim.x * kTcGroups-th after: a static schedule with no shared counter,
// so launches on different streams are independent.  A unit is 128
// consecutive states or rows; rows past the end are computed on zeros and
// not stored.
// PG12_TC_CHAIN 1 (default): the partial rounds in their unrolled form on the
// tensor cores (tc_partial, 87 KB of the tables); 0: on the integer pipes.
#ifndef PG12_TC_CHAIN
#define PG12_TC_CHAIN 1
#endif
#ifndef PG12_TC_GROUPS
#define PG12_TC_GROUPS 4
#endif
constexpr bool kTcChain = PG12_TC_CHAIN != 0;
constexpr int kTcGroups = PG12_TC_GROUPS;
constexpr int kTcThreads = kTcGroup * kTcGroups;
using TcL = TcLayout<kTcGroups, kTcChain>;
using TcL1 = TcLayout<1, false>;  // one-group CTAs of small launches

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_permute(uint64_t *__restrict__ st, uint64_t n, int vec16) {
    extern __shared__ __align__(1024) uint8_t tc_sm[];
    TcGroup G = tc_setup<kTcGroups, kTcChain>(tc_sm);
    const uint64_t units = (n + kTcGroup - 1) / kTcGroup;
    const uint64_t step = (uint64_t)gridDim.x * kTcGroups;
    for (uint64_t u = (uint64_t)blockIdx.x * kTcGroups + threadIdx.x / kTcGroup; u < units; u += step) {
        const uint64_t k = u * kTcGroup + G.t;
        const bool valid = k < n;
        uint64_t *p = st + kT * k;
        uint64_t x[kT];
        if (valid && vec16) {
#pragma unroll
            for (int i = 0; i < kT; i += 2) ld2_nc(p + i, x[i], x[i + 1]);
        } else {
#pragma unroll
            for (int i = 0; i < kT; ++i) x[i] = valid ? p[i] : 0ull;
        }
        if (!tc_permute<kTcChain>(G, x, false, false)) break;
        if (valid) {
            if (vec16) {
#pragma unroll
                for (int i = 0; i < kT; i += 2) st2(p + i, canon(x[i]), canon(x[i + 1]));
            } else {
#pragma unroll
                for (int i = 0; i < kT; ++i) p[i] = canon(x[i]);
            }
        }
    }
    tc_teardown<kTcGroups, kTcChain>(tc_sm, G);
}

// Sponge digests of n rows of width w (Sec. 2.4): the leaves of a tree, or a
// tree level (the level below read as rows of its children's 8 words), or
// pg_hash_rows.  Launched as a dependent launch it may set up while the
// kernel before it finishes, and reads `rows` only after pdl_wait().
// GROUPS = kTcGroups for large launches (one CTA per SM); GROUPS = 1 with
// the partial rounds on the integer pipes for launches of few units (62 KB
// of shared memory and 128 tensor-memory columns per CTA, up to three CTAs
// per SM), which spread them over more SMs.
template <int GROUPS, bool CHAIN>
__global__ void __launch_bounds__(kTcGroup * GROUPS, 1) k_tc_sponge(const uint64_t *__restrict__ rows, uint64_t n,
                                                                    uint64_t w, int vec16, uint64_t *__restrict__ out) {
    extern __shared__ __align__(1024) uint8_t tc_sm[];
    pdl_trigger();
    TcGroup G = tc_setup<GROUPS, CHAIN>(tc_sm);
    pdl_wait();
    const uint64_t units = (n + kTcGroup - 1) / kTcGroup;
    const uint64_t step = (uint64_t)gridDim.x * GROUPS;
    const uint64_t chunks = (w + kRate - 1) / kRate;
    for (uint64_t u = (uint64_t)blockIdx.x * GROUPS + threadIdx.x / kTcGroup; u < units; u += step) {
        const uint64_t r = u * kTcGroup + G.t;
        const bool valid = r < n;
        const uint64_t *row = rows + (valid ? r : 0) * w;
        uint64_t x[kT];
#pragma unroll
        for (int i = kRate; i < kT; ++i) x[i] = 0;
        bool ok = true;
        for (uint64_t c = 0; c < chunks && ok; ++c) {
            uint64_t ch[kRate];
            load_chunk(row, w, c, vec16 != 0, ch);
#pragma unroll
            for (int i = 0; i < kRate; ++i) x[i] = valid ? ch[i] : 0ull;
            ok = tc_permute<CHAIN>(G, x, c == 0, c + 1 == chunks);
        }
        if (!ok) break;
        if (valid) {
            st2(out + kDigest * r, canon(x[0]), canon(x[1]));
            st2(out + kDigest * r + 2, canon(x[2]), canon(x[3]));
        }
    }
    tc_teardown<GROUPS, CHAIN>(tc_sm, G);
}

// Leaf sponges over rows that arrive in chunks while the kernel runs
// (pg_merkle_build_host): rows [end[c-1], end[c]) are chunk c, and the copy
// stream writes base + c + 1 into *ready once chunk c is in device memory.
// Before a unit's rows are read, thread 0 of its group waits (bounded, with
// an acquire load) until *ready shows the chunk of the unit's last row; the
// group's barrier passes that on, and the rows are read through L2.  Units
// go out in increasing order, so the first chunks are hashed while later
// ones are still being copied, in one launch.
struct ChunkMap {
    uint64_t end[16];
    uint32_t count;
    uint32_t base;
};

__device__ __forceinline__ bool wait_ready(const uint32_t *ready, uint32_t want) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ready) : "memory");
        if ((int32_t)(v - want) >= 0) return true;  // serial-number order: base wraps
        if (clock64() - t0 > kTcWaitClocks) return false;
        __nanosleep(200);
    }
}

template <int GROUPS, bool CHAIN>
__global__ void __launch_bounds__(kTcGroup * GROUPS, 1)
    k_tc_leaves_stream(const uint64_t *__restrict__ rows, uint64_t n, uint64_t w, int vec16,
                       uint64_t *__restrict__ out, const uint32_t *__restrict__ ready, const ChunkMap cm) {
    extern __shared__ __align__(1024) uint8_t tc_sm[];
    TcGroup G = tc_setup<GROUPS, CHAIN>(tc_sm);
    const uint64_t units = (n + kTcGroup - 1) / kTcGroup;
    const uint64_t step = (uint64_t)gridDim.x * GROUPS;
    const uint64_t chunks = (w + kRate - 1) / kRate;
    uint32_t have = 0;  // chunks this group has seen arrive
    for (uint64_t u = (uint64_t)blockIdx.x * GROUPS + threadIdx.x / kTcGroup; u < units; u += step) {
        const uint64_t last = (u + 1) * kTcGroup < n ? (u + 1) * kTcGroup - 1 : n - 1;
        uint32_t c = 0;
        while (c + 1 < cm.count && cm.end[c] <= last) ++c;
        if (c >= have) {
            const uint32_t late = G.t == 0 && !wait_ready(ready, cm.base + c + 1);
            if (group_sync_or(G.bar, late)) {
                G.failed = 1;
                break;
            }
            have = c + 1;
        }
        const uint64_t r = u * kTcGroup + G.t;
        const bool valid = r < n;
        const uint64_t *row = rows + (valid ? r : 0) * w;
        uint64_t x[kT];
#pragma unroll
        for (int i = kRate; i < kT; ++i) x[i] = 0;
        bool ok = true;
        for (uint64_t k = 0; k < chunks && ok; ++k) {
            uint64_t ch[kRate];
            load_chunk_cg(row, w, k, vec16 != 0, ch);
#pragma unroll
            for (int i = 0; i < kRate; ++i) x[i] = valid ? ch[i] : 0ull;
            ok = tc_permute<CHAIN>(G, x, k == 0, k + 1 == chunks);
        }
        if (!ok) break;
        if (valid) {
            st2(out + kDigest * r, canon(x[0]), canon(x[1]));
            st2(out + kDigest * r + 2, canon(x[2]), canon(x[3]));
        }
    }
    tc_teardown<GROUPS, CHAIN>(tc_sm, G);
}

// One warp task: lane i of task u at level l hashes node 32u+i of that level
// -- a row through the sponge at level 0, else the pair of children at
// level l-1 -- in the lane's shared-memory state slot (stride S = threads
// per block).  Both cases feed one permutation call site, so the kernel holds
// a single copy of the permutation code.  ZC: the first permutation of a task
// takes the zero-capacity round 0 (a second copy of round 0's dense layer in
// the kernel; measured a gain where every warp hashes single-chunk leaves, a
// loss of 7% in the batched launch, where warps sit in different phases).
template <int S, int MDS, bool ZC = false>
__device__ __forceinline__ void run_warp_task(const TreePlan &tp, uint32_t level, uint64_t u, int lane,
                                              uint64_t *slot) {
    const uint64_t n = tp.n_leaves;
    const uint64_t count = n >> level;
    const uint64_t i = u * kWarpNodes + lane;
    if (i >= count) return;
    const uint64_t w = tp.width;
    const bool leaf = level == 0;
    const uint64_t nperm = leaf ? (w == 0 ? 1 : (w + kRate - 1) / kRate) : 1;
    const uint64_t *row = tp.rows + i * w;
    const uint64_t *kids = tp.nodes + kDigest * (level_off(n, leaf ? 0 : level - 1) + 2 * i);
#pragma unroll
    for (int k = kRate; k < kT; ++k) slot[k * S] = 0;
    for (uint64_t c = 0; c < nperm; ++c) {
        if (leaf) {
            uint64_t ch[kRate];
            load_chunk(row, w, c, tp.vec16 != 0, ch);
#pragma unroll
            for (int k = 0; k < kRate; ++k) slot[k * S] = ch[k];
        } else {
#pragma unroll
            for (int k = 0; k < 2 * kDigest; k += 2) {
                uint64_t a, b;
                ld2_cg(kids + k, a, b);
                slot[k * S] = a;
                slot[(k + 1) * S] = b;
            }
        }
        permute_slot<S, MDS>(slot, ZC && c == 0, c + 1 == nperm);
    }
    uint64_t *dst = tp.nodes + kDigest * (level_off(n, level) + i);
    st2(dst, canon(slot[0]), canon(slot[S]));
    st2(dst + 2, canon(slot[2 * S]), canon(slot[3 * S]));
}

// Completion flag of a tree: the root is stored by lane 0 of the warp that
// built it; make its stores (and, through the climb's fences, the whole
// tree) visible system-wide before raising the flag.
__device__ __forceinline__ void signal_root(const TreePlan &tp, int lane) {
    if (lane == 0 && tp.done_flag != nullptr) {
        __threadfence_system();
        *reinterpret_cast<volatile uint32_t *>(tp.done_flag) = 1u;
    }
}

// Leaf sponges of one tree on the integer pipes, one 32-leaf task per warp
// in a static schedule (warp w of the grid takes tasks w, w + W, ...; tasks
// are uniform, so no counter is needed), the plan passed by value: the
// launch reads and writes nothing but the rows and the leaf digests, so
// builds on different streams do not share any state.
template <int MDS>
__global__ void __launch_bounds__(kBlock, PG12_MERKLE_MIN_BLOCKS) k_merkle_leaves(const TreePlan tp,
                                                                                uint32_t total_tasks) {
    __shared__ uint64_t slots[kT * kBlock];
    uint64_t *slot = slots + threadIdx.x;
    const int lane = threadIdx.x & 31;
    pdl_trigger();
    const uint32_t warps = gridDim.x * (kBlock / 32);
    for (uint32_t task = blockIdx.x * (kBlock / 32) + threadIdx.x / 32; task < total_tasks; task += warps)
        run_warp_task<kBlock, MDS, true>(tp, 0, task, lane, slot);
}

// Persistent Merkle kernel: every warp pulls leaf tasks from a global
// counter (in order, so sibling subtrees finish close together), hashes
// them, and announces each finished task to its parent's arrival counter.
// The warp that brings a parent's count to two (its second child) builds
// the parent and keeps climbing; the first arriver goes back for a new leaf
// task.  Levels with at most 32 nodes have a single task and are climbed
// without counters.  No block-wide barrier and no waiting anywhere.
template <int S, int MDS, bool ZC = false>
__global__ void __launch_bounds__(S, PG12_MERKLE_MIN_BLOCKS * 256 / S) k_merkle(const TreePlan *__restrict__ plans, uint32_t n_trees,
                                             uint32_t total_tasks, uint32_t *__restrict__ counters,
                                             uint32_t *__restrict__ next_task) {
    __shared__ uint64_t slots[kT * S];
    uint64_t *slot = slots + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xFFFFFFFFu;
    pdl_trigger();
    for (;;) {
        uint32_t task = 0;
        if (lane == 0) task = atomicAdd(next_task, 1u);
        task = __shfl_sync(full, task, 0);
        if (task >= total_tasks) return;
        uint32_t lo = 0, hi = n_trees - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) / 2;
            if (plans[mid].leaf_task_begin <= task) lo = mid;
            else hi = mid - 1;
        }
        const TreePlan &tp = plans[lo];
        const uint64_t n = tp.n_leaves;
        const uint32_t log_n = tp.log_n;
        uint64_t u = task - tp.leaf_task_begin;
        run_warp_task<S, MDS, ZC>(tp, 0, u, lane, slot);
        if (log_n == 0) signal_root(tp, lane);
        const uint32_t top = log_n < tp.climb_limit ? log_n : tp.climb_limit;
        for (uint32_t level = 1; level <= top; ++level) {
            const uint64_t below = n >> (level - 1);
            if (below > (uint64_t)kWarpNodes) {
                // two child tasks: only the second to finish continues
                __threadfence();
                __syncwarp();
                uint32_t old = 0;
                if (lane == 0) old = atomicAdd(&counters[tp.counter_base + tp.level_counter[level] + (u >> 1)], 1u);
                old = __shfl_sync(full, old, 0);
                if (old == 0) break;
                __threadfence();
            } else {
                __syncwarp();
            }
            u >>= 1;
            run_warp_task<S, MDS, ZC>(tp, level, u, lane, slot);
            if (level == log_n) signal_root(tp, lane);
        }
    }
}

// ------------------------------------------- tensor-core batch kernel
// Units of 128 nodes: level l of a tree of n leaves has
// ceil((n >> l) / 128) of them.  A task is 2^fuse consecutive leaf units;
// the group that takes it builds them and the fuse levels above them on its
// own, then climbs with arrival counters: when the level below has at least
// two units, the group that completes the second of two sibling units
// builds their parent unit and goes on, the first goes back for a new task.
// Levels of at most 128 nodes have one unit and are climbed directly.
__device__ __forceinline__ uint64_t tc_units(uint64_t n, uint32_t l) {
    return ((n >> l) + kTcGroup - 1) / kTcGroup;
}

// Unit u of level l of a tree: node k = 128 u + t of the level is the
// sponge of leaf row k (l = 0) or the compression of children 2k, 2k + 1
// (read from L2: other groups of this launch wrote them).  Rows past the
// level's end are computed on zeros and not stored.
__device__ __forceinline__ bool tc_unit(TcGroup &G, const TreePlan &tp, uint32_t l, uint64_t u) {
    const uint64_t n = tp.n_leaves, cnt = n >> l;
    const uint64_t k = u * kTcGroup + G.t;
    const bool valid = k < cnt;
    // a node is the one-chunk sponge of its children's 8 words; one
    // permutation call site for leaves and nodes keeps the kernel's code small
    const bool leaf = l == 0;
    const uint64_t w = leaf ? tp.width : 2 * kDigest, chunks = (w + kRate - 1) / kRate;
    const uint64_t *row = leaf ? tp.rows + (valid ? k : 0) * w
                               : tp.nodes + kDigest * (level_off(n, l - 1) + 2 * (valid ? k : 0));
    uint64_t x[kT];
#pragma unroll
    for (int i = kRate; i < kT; ++i) x[i] = 0;
    for (uint64_t c = 0; c < chunks; ++c) {
        uint64_t ch[kRate];
        if (leaf) {
            load_chunk(row, w, c, tp.vec16 != 0, ch);
        } else {  // written by this launch: coherent loads
#pragma unroll
            for (int i = 0; i < kRate; i += 2) ld2_cg(row + i, ch[i], ch[i + 1]);
        }
#pragma unroll
        for (int i = 0; i < kRate; ++i) x[i] = valid ? ch[i] : 0ull;
        if (!tc_permute<kTcChain>(G, x, c == 0, c + 1 == chunks)) return false;
    }
    if (valid) {
        uint64_t *dst = tp.nodes + kDigest * (level_off(n, l) + k);
        st2(dst, canon(x[0]), canon(x[1]));
        st2(dst + 2, canon(x[2]), canon(x[3]));
    }
    return true;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_batch(const TreePlan *__restrict__ plans, uint32_t n_trees,
                                                            uint32_t total_tasks, uint32_t fuse,
                                                            uint32_t *__restrict__ counters,
                                                            uint32_t *__restrict__ next_task) {
    extern __shared__ __align__(1024) uint8_t tc_sm[];
    TcGroup G = tc_setup<kTcGroups, kTcChain>(tc_sm);
    bool ok = true;
    while (ok) {
        const uint32_t task = group_fetch_add(G, next_task);
        if (task >= total_tasks) break;
        uint32_t lo_t = 0, hi_t = n_trees - 1;
        while (lo_t < hi_t) {
            const uint32_t mid = (lo_t + hi_t + 1) / 2;
            if (plans[mid].leaf_task_begin <= task) lo_t = mid;
            else hi_t = mid - 1;
        }
        const TreePlan &tp = plans[lo_t];
        const uint64_t n = tp.n_leaves;
        const uint32_t log_n = tp.log_n;
        const uint32_t top = log_n < tp.climb_limit ? log_n : tp.climb_limit;
        uint64_t lo = (uint64_t)(task - tp.leaf_task_begin) << fuse;
        const uint64_t units0 = tc_units(n, 0);
        uint64_t cnt = units0 - lo < (1ull << fuse) ? units0 - lo : (1ull << fuse);
        for (uint32_t l = 0;; ++l) {
            for (uint64_t i = 0; i < cnt && ok; ++i) ok = tc_unit(G, tp, l, lo + i);
            if (!ok) break;
            if (l == log_n) {
                if (G.t == 0) signal_root(tp, 0);
                break;
            }
            if (l == top) break;  // the levels above are built by k_batch_top
            __threadfence();
            if (cnt >= 2) {
                // both children of every parent unit are this task's: no counter
                group_sync(G.bar);
                lo >>= 1;
                cnt >>= 1;
                continue;
            }
            if (tc_units(n, l) >= 2) {
                const uint32_t old = group_fetch_add(G, &counters[tp.counter_base + tp.level_counter[l + 1] + (lo >> 1)]);
                if (old == 0) break;  // the sibling unit is not done: its group builds the parent
                __threadfence();
            } else {
                group_sync(G.bar);
            }
            lo >>= 1;
        }
    }
    tc_teardown<kTcGroups, kTcChain>(tc_sm, G);
}

// The top levels of every tree of a batch whose persistent launch stopped
// below them (climb_limit): one block per tree, 16 lanes per node (the
// latency form), a block barrier between levels; at most 64 nodes a level.
constexpr int kBatchTopThreads = 1024;
constexpr uint64_t kBatchTopNodes = kBatchTopThreads / 16;
__global__ void __launch_bounds__(kBatchTopThreads) k_batch_top(const TreePlan *__restrict__ plans) {
    __shared__ __align__(16) DevConsts K;
    load_consts(K);
    const TreePlan &tp = plans[blockIdx.x];
    const uint64_t n = tp.n_leaves;
    const uint32_t log_n = tp.log_n;
    if (tp.climb_limit >= log_n) return;  // this tree was climbed to its root
    const uint64_t gid = threadIdx.x >> 4;
    const int l16 = threadIdx.x & 15;
    for (uint32_t level = tp.climb_limit + 1; level <= log_n; ++level) {
        const uint64_t count = n >> level;
        if ((gid & ~1ull) < count) {  // whole warps (groups 2w, 2w + 1)
            const bool valid = gid < count;
            const uint64_t node = valid ? gid : 0;
            const uint64_t *kids = tp.nodes + kDigest * (level_off(n, level - 1) + 2 * node);
            uint64_t x = 0;
            if (l16 < 2 * kDigest) {
                asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(x) : "l"(kids + l16));
            }
            x = permute_wide(x, l16, 0xFFFFFFFFu, K);
            if (valid && l16 < kDigest) tp.nodes[kDigest * (level_off(n, level) + node) + l16] = canon(x);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) signal_root(tp, 0);
}

// ---------------------------------------------------- allocation-free build
// For callers that cannot allocate device memory (for example code running
// under an allocator that forbids cudaMalloc, or inside a host process that
// only owns the buffers it was handed): the arrival counters live in this
// file-scope array instead of the pg_init() workspace, and the tree plan is
// passed by value as a kernel argument.  Every GPU that loads the library
// holds the array (512 KiB) until the process exits.
constexpr uint64_t kNoAllocMaxLeaves = 1ull << 22;
constexpr size_t kNoAllocWords = (size_t)(kNoAllocMaxLeaves / kWarpNodes);  // task counter + arrival counters
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

template <int MDS>
__global__ void __launch_bounds__(kBlock) k_merkle_single(const TreePlan tp, uint32_t total_tasks,
                                                          uint32_t *__restrict__ counters,
                                                          uint32_t *__restrict__ next_task) {
    __shared__ uint64_t slots[kT * kBlock];
    uint64_t *slot = slots + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xFFFFFFFFu;
    const uint64_t n = tp.n_leaves;
    for (;;) {
        uint32_t task = 0;
        if (lane == 0) task = atomicAdd(next_task, 1u);
        task = __shfl_sync(full, task, 0);
        if (task >= total_tasks) return;
        uint64_t u = task;
        run_warp_task<kBlock, MDS>(tp, 0, u, lane, slot);
        for (uint32_t level = 1; level <= tp.log_n; ++level) {
            if ((n >> (level - 1)) > (uint64_t)kWarpNodes) {
                __threadfence();
                __syncwarp();
                uint32_t old = 0;
                if (lane == 0) old = atomicAdd(&counters[tp.level_counter[level] + (u >> 1)], 1u);
                old = __shfl_sync(full, old, 0);
                if (old == 0) break;
                __threadfence();
            } else {
                __syncwarp();
            }
            u >>= 1;
            run_warp_task<kBlock, MDS>(tp, level, u, lane, slot);
        }
    }
}


// Upper levels of a tree with the 16-lanes-per-state permutation: one group
// per node of `level`, one launch per level.  Lanes 0..7 load the children,
// lanes 0..3 store the digest.  Every lane reaches the shuffles (groups past
// the level's end compute on a dummy node and skip the store).
constexpr int kTopBlock = 256;
// The last levels of a tree (at most kTailNodes nodes each) in one launch of
// one thread-block cluster: kTailCtas blocks on as many SMs, one 16-lane
// group per node, a cluster barrier between levels.  Saves a launch and a
// constant copy per level where each level is one permutation's latency
// anyway; spread over eight SMs (one warp per scheduler at the widest level)
// the permutations do not queue for issue slots as they do in one block.
// Children are read with ld.global.cg (from L2): a line of a small level can
// sit in an SM's L1 from an earlier level's read before another block of the
// cluster has written it.
constexpr int kTailCtas = 8;
constexpr int kTailBlock = 128;
constexpr uint64_t kTailNodes = kTailCtas * kTailBlock / 16;
__global__ void __cluster_dims__(kTailCtas, 1, 1) __launch_bounds__(kTailBlock)
    k_merkle_top_tail(uint64_t *__restrict__ nodes, uint64_t n, uint32_t first) {
    __shared__ __align__(16) DevConsts K;
    load_consts(K);
    pdl_trigger();
    pdl_wait();
    const uint32_t log_n = 63 - __clzll(n);
    const uint64_t gid = ((uint64_t)blockIdx.x * kTailBlock + threadIdx.x) >> 4;
    const int l16 = threadIdx.x & 15;
    for (uint32_t level = first; level <= log_n; ++level) {
        const uint64_t count = n >> level;
        // whole warps hold groups 2w and 2w + 1; a warp past the level's end skips it
        if ((gid & ~1ull) < count) {
            const bool valid = gid < count;
            const uint64_t node = valid ? gid : 0;
            const uint64_t *kids = nodes + kDigest * (level_off(n, level - 1) + 2 * node);
            uint64_t x = 0;
            if (l16 < 2 * kDigest) {
                asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(x) : "l"(kids + l16));
            }
            x = permute_wide(x, l16, 0xFFFFFFFFu, K);
            if (valid && l16 < kDigest) nodes[kDigest * (level_off(n, level) + node) + l16] = canon(x);
        }
        // every thread of the cluster arrives: stores above are released to, and
        // the next level's loads acquire from, the whole cluster
        asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                     "barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
}

__global__ void __launch_bounds__(kTopBlock) k_merkle_top(uint64_t *__restrict__ nodes, uint64_t n, uint32_t level) {
    __shared__ __align__(16) DevConsts K;
    load_consts(K);
    pdl_trigger();
    pdl_wait();
    const uint64_t count = n >> level;
    const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
    const int l16 = threadIdx.x & 15;
    const bool valid = gid < count;
    const uint64_t node = valid ? gid : 0;
    const uint64_t *kids = nodes + kDigest * (level_off(n, level - 1) + 2 * node);
    uint64_t x = 0;
    if (l16 < 2 * kDigest) {
        asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(x) : "l"(kids + l16));
    }
    x = permute_wide(x, l16, 0xFFFFFFFFu, K);
    if (valid && l16 < kDigest) nodes[kDigest * (level_off(n, level) + node) + l16] = canon(x);
}

// Leaf level of a small tree with the wide permutation: one group per row,
// lanes 0..7 absorb the chunk words, lanes 8..11 carry the capacity.
__global__ void __launch_bounds__(kTopBlock) k_merkle_top_leaf(const uint64_t *__restrict__ rows, uint64_t n,
                                                               uint64_t w, uint64_t *__restrict__ nodes) {
    __shared__ __align__(16) DevConsts K;
    load_consts(K);
    pdl_trigger();
    const uint64_t gid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
    const int l16 = threadIdx.x & 15;
    const bool valid = gid < n;
    const uint64_t node = valid ? gid : 0;
    const uint64_t *row = rows + node * w;
    const uint64_t chunks = (w + kRate - 1) / kRate;
    uint64_t x = 0;
    for (uint64_t c = 0; c < chunks; ++c) {
        if (l16 < kRate) {
            const uint64_t k = c * kRate + l16;
            x = k < w ? __ldg(row + k) : 0ull;
        }
        x = permute_wide(x, l16, 0xFFFFFFFFu, K);
    }
    if (valid && l16 < kDigest) nodes[kDigest * node + l16] = canon(x);
}


// Authentication paths: thread per (query, level) copies one sibling digest.
__global__ void k_merkle_open(const uint64_t *__restrict__ nodes, uint64_t n, uint32_t depth,
                              const uint64_t *__restrict__ idx, uint64_t k, uint64_t *__restrict__ paths) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= k * depth) return;
    const uint64_t q = t / depth;
    const uint32_t l = (uint32_t)(t % depth);
    const uint64_t leaf = idx[q];
    uint64_t *dst = paths + kDigest * t;
    if (leaf >= n) {
        for (int i = 0; i < kDigest; ++i) dst[i] = ~0ull;
        return;
    }
    const uint64_t sib = (leaf >> l) ^ 1ull;
    const uint64_t *src = nodes + kDigest * (level_off(n, l) + sib);
    for (int i = 0; i < kDigest; ++i) dst[i] = src[i];
}

// Path verification: one thread per query climbs log2(N) permutations.
constexpr int kVerifyBlock = 128;
template <int MDS>
__global__ void __launch_bounds__(kVerifyBlock) k_merkle_verify(const uint64_t *__restrict__ root, uint32_t depth,
                                                                uint64_t n, const uint64_t *__restrict__ leaves,
                                                                const uint64_t *__restrict__ idx, uint64_t k,
                                                                const uint64_t *__restrict__ paths,
                                                                uint8_t *__restrict__ ok) {
    __shared__ uint64_t slots[kT * kVerifyBlock];
    uint64_t *slot = slots + threadIdx.x;
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= k) return;
    uint64_t cur[kDigest];
    for (int i = 0; i < kDigest; ++i) cur[i] = leaves[kDigest * q + i];
    uint64_t pos = idx[q];
    const bool in_range = pos < n;
    for (uint32_t l = 0; l < depth; ++l) {
        const uint64_t *sib = paths + kDigest * (q * depth + l);
        const bool right = pos & 1;
        for (int i = 0; i < kDigest; ++i) {
            slot[i * kVerifyBlock] = right ? sib[i] : cur[i];
            slot[(kDigest + i) * kVerifyBlock] = right ? cur[i] : sib[i];
            slot[(2 * kDigest + i) * kVerifyBlock] = 0;
        }
        permute_slot<kVerifyBlock, MDS>(slot, true, true);
        for (int i = 0; i < kDigest; ++i) cur[i] = canon(slot[i * kVerifyBlock]);
        pos >>= 1;
    }
    bool eq = in_range;
    for (int i = 0; i < kDigest; ++i) eq = eq && (cur[i] == root[i]);
    ok[q] = eq ? 1 : 0;
}

}  // namespace dev

// ================================================================ host side
namespace {

// tensor engine: tree levels of at least this many nodes use the tensor-core
// kernel (one-group CTAs while a level has fewer units than the GPU has
// groups).  Measured on the 2^22 x 8 tree: 2^15 10.25 ms, 2^13 10.11 ms,
// 2^12 10.14 ms; below that the 16-lane latency form is faster per level.
#ifndef PG12_TC_MIN_NODES
#define PG12_TC_MIN_NODES (1ull << 13)
#endif
#ifndef PG12_TC_SMALL_TREE
#define PG12_TC_SMALL_TREE 8192
#endif

#ifndef PG12_HOST_STREAM
#define PG12_HOST_STREAM 1  // 0: one leaf launch per copied chunk (also at run time: PG12_HOST_STREAM=0)
#endif
constexpr uint32_t kReadyVals = 1u << 16;  // values of the chunk arrival counter

struct Context {
    bool params_ready = false;
    int params_set = 0;  // 0 = pg12_v1, 1 = pg12_small
    int params_gen = 1;  // bumped whenever the active set changes
    uint32_t small_row[kT] = {};
    PlainParams plain;
    OptParams opt;
    bool init = false;
    int device = -1;
    int sms = 0;
    int merkle_blocks_per_sm = 0;      // k_merkle<256, *> (both matrix kinds: minimum)
    int leaves_blocks_per_sm = 0;      // k_merkle_leaves<*>
    int merkle128_blocks_per_sm = 0;   // k_merkle<128, *>
    int permute_blocks_per_sm = 0;
    uint8_t *ws = nullptr;  // device workspace
    size_t ws_bytes = 0;
    // 1: permutations of batches, rows, leaves and large levels run their full
    // rounds' dense layers on the tensor cores; 0: integer pipes only
    int engine = 1;
    uint64_t tc_min_nodes = PG12_TC_MIN_NODES;  // smallest tree level built by the tensor-core kernel
    cudaStream_t copy_st = nullptr;  // host-row copies of pg_merkle_build_host
    cudaEvent_t host_ev[17] = {};    // one per chunk, plus "previous work done"
    // chunk arrival counter of the streaming leaf launch: the copy stream
    // copies ready_vals[v] = v into *d_ready; every build takes 16 new values
    uint32_t *d_ready = nullptr;
    uint32_t *ready_vals = nullptr;  // page-locked, kReadyVals entries
    uint32_t ready_base = 0;
    cudaEvent_t ready_ev = nullptr;  // after the last streaming leaf launch
    // the streamed form is used when the device overlaps copies with kernels
    // and the environment does not set PG12_HOST_STREAM=0 (tools that hold
    // copies back while a kernel runs, such as profilers replaying kernels,
    // would make its waits run out)
    bool host_stream = false;
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

}  // namespace

int set_error(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return status;
}

namespace {

#define PG_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(PG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

constexpr size_t kWorkspaceBytes = 32u << 20;  // tree plans + arrival counters
// pg_merkle_build's split of a tree between kernels.  Trees of at most
// kSmallTree leaves run entirely in the 16-lanes-per-state kernels.  In
// larger trees one launch hashes the leaves and every level is one launch
// (one launch per level measured faster than climbing with arrival counters
// in one persistent launch: 16.7 against 17.4 ms for a 2^22 x 8 tree on the
// integer pipes, 10.20 against 10.73 ms with the tensor-core kernel): the
// tensor-core kernel for levels of at least tc_min_nodes nodes, one thread
// per node (k_merkle_level) while the level has more than kWideNodes nodes
// (integer engine), the 16-lanes-per-state kernel above that, and one
// cluster launch for the levels of at most 64 nodes.
#ifndef PG12_WIDE_NODES
#define PG12_WIDE_NODES 8192
#endif
constexpr uint64_t kWideNodes = PG12_WIDE_NODES;
constexpr uint64_t kSmallTree = kWideNodes;
// tensor engine: trees of at most this many leaves run in the 16-lane form
constexpr uint64_t kTcSmallTree = PG12_TC_SMALL_TREE;
constexpr size_t kPlanBytes = 4u << 20;        // first part: plans; rest: counters

// ------------------------------------------------------------ launch timing
// Optional per-kernel timing (pg_profile_enable / pg_profile_read): a pair of
// CUDA events is recorded on the launching stream around each launch and
// resolved when the records are read.  Launches inside a stream capture are
// not recorded (the graph launch is, as one entry).
const char *const kKernelNames[kIdCount] = {"k_merkle",      "k_merkle_top",    "k_merkle_top_leaf",
                                            "k_permute",     "k_hash_rows",     "k_merkle_open",
                                            "k_merkle_verify", "k_merkle_single", "batch_graph",
                                            "k_ntt_pass",    "k_ntt_bitrev",    "k_merkle_level",
                                            "k_merkle_top_tail",
                                            "k_tc_permute",  "k_tc_sponge:leaves", "k_tc_sponge:level",
                                            "k_tc_sponge:rows", "k_tc_batch",  "k_batch_top"};
constexpr size_t kProfMaxRecords = 1u << 16;

struct ProfRecord {
    int kid;
    int device;
    uint64_t perms;
    cudaEvent_t a, b;
};

struct Profiler {
    std::mutex mu;
    std::atomic<bool> on{false};
    std::vector<ProfRecord> recs;
    std::vector<std::pair<int, cudaEvent_t>> spare;  // (device, event)
    uint64_t dropped = 0;

    cudaEvent_t take(int device) {  // mu held
        for (size_t k = spare.size(); k-- > 0;)
            if (spare[k].first == device) {
                cudaEvent_t e = spare[k].second;
                spare.erase(spare.begin() + (long)k);
                return e;
            }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
};
Profiler g_prof;

// Permutations of a whole tree: ceil(w/8) per leaf plus one per inner node.
uint64_t tree_perms(uint64_t n, uint64_t w) { return n * ((w + kRate - 1) / kRate) + (n - 1); }

uint64_t batch_perms(const pg_tree *trees, size_t n_trees) {
    uint64_t p = 0;
    for (size_t k = 0; k < n_trees; ++k) p += tree_perms(trees[k].n_leaves, trees[k].width);
    return p;
}

pg_status ensure_params() {
    if (g.params_ready) return PG_OK;
    if (g.params_set == 1) host::generate_small(g.plain, g.small_row);
    else host::generate_plain(g.plain);
    if (!host::derive_optimized(g.plain, g.opt))
        return fail(PG_ERR_PARAMS, "parameter set %s: sparse rewrite failed (singular block)",
                    g.params_set == 1 ? "pg12_small" : "pg12_v1");
    g.params_ready = true;
    return PG_OK;
}

// Constant tables of the active parameter set onto the current device: the
// permutation constants of both permutation forms and the digit tables of
// the tensor-core dense layers.
pg_status upload_tables() {
    dev::DevConsts dc;
    dev::make_dev_consts(g.opt, dc);
    PG_CUDA(cudaMemcpyToSymbol(dev::c_dev, &dc, sizeof(dc)));
    PG_CUDA(cudaMemcpyToSymbol(dev::g_dev, &dc, sizeof(dc)));
    static TcTables tt;  // 105 KB; built under g_mu
    if (!host::build_tc_tables(g.opt, tt))
        return fail(PG_ERR_PARAMS, "parameter set %s: a tensor-core sum could leave the exact fp32 window",
                    g.params_set == 1 ? "pg12_small" : "pg12_v1");
    PG_CUDA(cudaMemcpyToSymbol(dev::g_tc, &tt, sizeof(tt)));
    static ChainParams cp;
    host::derive_chain(g.opt, cp);
    PG_CUDA(cudaMemcpyToSymbol(dev::c_beta, cp.beta, sizeof(cp.beta)));
    return PG_OK;
}

bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }

// Do the byte ranges [a, a + na) and [b, b + nb) share an address?
bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return na && nb && x < y + nb && y < x + na;
}
uint32_t log2u(uint64_t x) {
    uint32_t l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

// Task geometry of one tree.  Integer engine (k_merkle): a task is 32
// nodes of one level (unit_log 5, fuse 0).  Tensor engine (k_tc_batch): a
// unit is 128 nodes (unit_log 7) and a leaf task 2^fuse leaf units.  Level
// l >= 1 gets arrival counters (one per unit) when level l - 1 has at least
// two units.  n_counters receives their number; returns the leaf tasks.
uint32_t plan_tree(dev::TreePlan &tp, const uint64_t *rows, uint64_t n, uint64_t w, uint64_t *nodes,
                   uint32_t leaf_task_begin, uint32_t counter_base, uint32_t &n_counters, uint32_t unit_log = 5,
                   uint32_t fuse = 0) {
    tp.rows = rows;
    tp.nodes = nodes;
    tp.n_leaves = n;
    tp.width = w;
    tp.log_n = log2u(n);
    tp.leaf_task_begin = leaf_task_begin;
    tp.counter_base = counter_base;
    tp.vec16 = ((w % 2) == 0 && (reinterpret_cast<uintptr_t>(rows) % 16) == 0) ? 1u : 0u;
    tp.climb_limit = tp.log_n;
    tp.done_flag = nullptr;
    n_counters = 0;
    const uint64_t unit = 1ull << unit_log;
    auto units = [&](uint32_t l) { return ((n >> l) + unit - 1) / unit; };
    for (uint32_t l = 0; l < (uint32_t)dev::kMaxLevels; ++l) tp.level_counter[l] = 0;
    for (uint32_t l = 1; l <= tp.log_n; ++l) {
        if (units(l - 1) >= 2) {
            tp.level_counter[l] = n_counters;
            n_counters += (uint32_t)units(l);
        }
    }
    return (uint32_t)((units(0) + (1ull << fuse) - 1) >> fuse);
}

// First level of a tree with at most 64 nodes (the top levels a 16-lane
// launch builds when a schedule asks for top_lanes = 16).
uint32_t first_small_level(uint64_t n) {
    uint32_t l = 0;
    while ((n >> l) > dev::kBatchTopNodes) ++l;
    return l;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

pg_status require_init() {
    if (!g.init) return fail(PG_ERR_NOT_INIT, "pg_init() has not been called");
    return PG_OK;
}

bool batch_uses_tc(const pg_schedule *sched) {
    const uint32_t e = sched ? sched->engine : PG_BATCH_ENGINE_DEFAULT;
    return e == PG_BATCH_ENGINE_TENSOR || (e == PG_BATCH_ENGINE_DEFAULT && g.engine == 1);
}

// Validate a batch and build its plans (in launch order).  Returns the
// number of leaf tasks and counters through the out-parameters.
pg_status plan_batch(const pg_tree *trees, size_t n_trees, const pg_schedule *sched_in,
                     std::vector<dev::TreePlan> &plans, uint32_t &tasks, uint64_t &counters, pg_schedule &resolved) {
    // the schedule with its engine resolved once, so that plans and launch agree
    std::memset(&resolved, 0, sizeof resolved);
    if (sched_in) resolved = *sched_in;
    if (resolved.engine == PG_BATCH_ENGINE_DEFAULT && resolved.reserved[0] == 0 && resolved.reserved[1] == 0)
        resolved.engine = g.engine == 1 ? PG_BATCH_ENGINE_TENSOR : PG_BATCH_ENGINE_INT;
    const pg_schedule *sched = &resolved;
    if (!trees || n_trees == 0) return fail(PG_ERR_INVALID_ARG, "empty batch");
    if (sched && (sched->reserved[0] != 0 || sched->reserved[1] != 0 ||
                  (sched->block != 0 && sched->block != 128 && sched->block != 256) || sched->order > 1 ||
                  sched->engine > PG_BATCH_ENGINE_TENSOR || sched->fuse_levels > 3 ||
                  (sched->top_lanes != 0 && sched->top_lanes != 1 && sched->top_lanes != 16)))
        return fail(PG_ERR_INVALID_ARG, "bad schedule");
    const bool tc = batch_uses_tc(sched);
    const uint32_t unit_log = tc ? 7 : 5, fuse = tc && sched ? sched->fuse_levels : 0;
    const bool handoff = sched && sched->top_lanes == 16;
    std::vector<size_t> idx(n_trees);
    for (size_t k = 0; k < n_trees; ++k) {
        const pg_tree &t = trees[k];
        if (!t.rows || !t.nodes) return fail(PG_ERR_INVALID_ARG, "tree %zu: rows or nodes is NULL", k);
        if (t.width == 0) return fail(PG_ERR_INVALID_ARG, "tree %zu: width must be >= 1", k);
        if (!is_pow2(t.n_leaves)) return fail(PG_ERR_NOT_POW2, "tree %zu: n_leaves=%llu is not a power of two", k,
                                              (unsigned long long)t.n_leaves);
        if (t.n_leaves > (1ull << 34)) return fail(PG_ERR_INVALID_ARG, "tree %zu: too many leaves", k);
        if (reinterpret_cast<uintptr_t>(t.rows) % 8) return fail(PG_ERR_INVALID_ARG, "tree %zu: rows not 8-byte aligned", k);
        if (reinterpret_cast<uintptr_t>(t.nodes) % 16)
            return fail(PG_ERR_INVALID_ARG, "tree %zu: nodes not 16-byte aligned", k);
        if (overlaps(t.rows, (size_t)t.n_leaves * t.width * 8, t.nodes, ((size_t)2 * t.n_leaves - 1) * 32))
            return fail(PG_ERR_INVALID_ARG, "tree %zu: rows and nodes overlap", k);
        idx[k] = k;
    }
    // node buffers are written concurrently: no two may share an address
    {
        std::vector<std::pair<uintptr_t, size_t>> spans(n_trees);
        for (size_t k = 0; k < n_trees; ++k)
            spans[k] = {reinterpret_cast<uintptr_t>(trees[k].nodes), k};
        std::sort(spans.begin(), spans.end());
        for (size_t k = 1; k < n_trees; ++k) {
            const pg_tree &a = trees[spans[k - 1].second];
            if (spans[k - 1].first + ((size_t)2 * a.n_leaves - 1) * 32 > spans[k].first)
                return fail(PG_ERR_INVALID_ARG, "trees %zu and %zu: node buffers overlap", spans[k - 1].second,
                            spans[k].second);
        }
    }
    if (sched && sched->order == 1) {
        auto work = [&](size_t k) {
            const pg_tree &t = trees[k];
            return (double)t.n_leaves * (double)((t.width + kRate - 1) / kRate + 1);
        };
        std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return work(a) > work(b); });
    }
    plans.assign(n_trees, dev::TreePlan{});
    uint64_t task_sum = 0, counter_sum = 0;
    for (size_t k = 0; k < n_trees; ++k) {
        const pg_tree &t = trees[idx[k]];
        uint32_t nc = 0;
        std::memset(&plans[k], 0, sizeof(dev::TreePlan));
        const uint32_t tk = plan_tree(plans[k], t.rows, t.n_leaves, t.width, t.nodes, (uint32_t)task_sum,
                                      (uint32_t)counter_sum, nc, unit_log, fuse);
        if (handoff) {
            const uint32_t f = first_small_level(t.n_leaves);
            plans[k].climb_limit = f == 0 ? 0 : f - 1;
        }
        task_sum += tk;
        counter_sum += nc;
        if (task_sum >= (1ull << 32) || counter_sum >= (1ull << 32))
            return fail(PG_ERR_INVALID_ARG, "batch too large (task or counter index above 2^32)");
    }
    tasks = (uint32_t)task_sum;
    counters = counter_sum;
    return PG_OK;
}

// One launch per level for levels first..log2(n_leaves) of a tree whose
// lower levels are in `nodes`: one thread per node (k_merkle_level) while a
// level has more than kWideNodes nodes, the 16-lanes-per-state kernel above.
// Launch a level kernel with programmatic stream serialisation (see
// pdl_trigger / pdl_wait): it may start, and copy its constants, while the
// kernel before it on `st` finishes.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Tensor-core kernels: one CTA per SM at most, each CTA four 128-row units at a time.
unsigned tc_grid(uint64_t n) {
    const uint64_t units = (n + dev::kTcGroup - 1) / dev::kTcGroup;
    const uint64_t want = (units + dev::kTcGroups - 1) / dev::kTcGroups;
    return (unsigned)(want < (uint64_t)g.sms ? want : (uint64_t)g.sms);
}

pg_status launch_tc_sponge(const uint64_t *rows, uint64_t n, uint64_t w, uint64_t *out, cudaStream_t st, bool dependent,
                           int kid) {
    if (n == 0) return PG_OK;
    const int vec16 = ((w % 2) == 0 && (reinterpret_cast<uintptr_t>(rows) % 16) == 0) ? 1 : 0;
    const uint64_t units = (n + dev::kTcGroup - 1) / dev::kTcGroup;
    // fewer units than the big CTAs' groups on the whole GPU: one group per CTA
    const bool one = units < (uint64_t)g.sms * dev::kTcGroups;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(one ? (unsigned)units : tc_grid(n));
    cfg.blockDim = dim3(one ? dev::kTcGroup : dev::kTcThreads);
    cfg.dynamicSmemBytes = one ? dev::TcL1::kBytes : dev::TcL::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = dependent ? 1 : 0;
    ProfScope prof(kid, st, n * ((w + kRate - 1) / kRate));
    if (one) PG_CUDA(cudaLaunchKernelEx(&cfg, dev::k_tc_sponge<1, false>, rows, n, w, vec16, out));
    else PG_CUDA(cudaLaunchKernelEx(&cfg, dev::k_tc_sponge<dev::kTcGroups, dev::kTcChain>, rows, n, w, vec16, out));
    return PG_OK;
}

// The leaf launch of a streamed host-rows build (k_tc_leaves_stream), in
// the same CTA shapes as launch_tc_sponge.
pg_status launch_leaves_stream(const uint64_t *rows, uint64_t n, uint64_t w, uint64_t *out, const uint32_t *ready,
                               const dev::ChunkMap &cm, cudaStream_t st) {
    const int vec16 = ((w % 2) == 0 && (reinterpret_cast<uintptr_t>(rows) % 16) == 0) ? 1 : 0;
    const uint64_t units = (n + dev::kTcGroup - 1) / dev::kTcGroup;
    const bool one = units < (uint64_t)g.sms * dev::kTcGroups;
    ProfScope prof(kIdTcLeaves, st, n * ((w + kRate - 1) / kRate));
    if (one)
        dev::k_tc_leaves_stream<1, false><<<(unsigned)units, dev::kTcGroup, dev::TcL1::kBytes, st>>>(rows, n, w, vec16, out,
                                                                                                  ready, cm);
    else
        dev::k_tc_leaves_stream<dev::kTcGroups, dev::kTcChain>
            <<<tc_grid(n), dev::kTcThreads, dev::TcL::kBytes, st>>>(rows, n, w, vec16, out, ready, cm);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

pg_status launch_levels(uint64_t *nodes, uint64_t n_leaves, uint32_t first, cudaStream_t st) {
    const uint32_t log_n = log2u(n_leaves);
    for (uint32_t l = first; l <= log_n; ++l) {
        const uint64_t cnt = n_leaves >> l;
        if (cnt <= dev::kTailNodes && l < log_n) {
            // this level and all above it in one cluster
            ProfScope prof(kIdMerkleTopTail, st, 2 * cnt - 1);
            PG_CUDA(launch_dependent(dev::k_merkle_top_tail, dev::kTailCtas, dev::kTailBlock, st, nodes, n_leaves, l));
            break;
        }
        if (g.engine == 1 && cnt >= g.tc_min_nodes) {
            // the level below, read as cnt rows of 8 words (children 2k, 2k+1)
            const uint64_t *below = nodes + 4 * (2 * n_leaves - ((2 * n_leaves) >> (l - 1)));
            uint64_t *here = nodes + 4 * (2 * n_leaves - ((2 * n_leaves) >> l));
            pg_status s = launch_tc_sponge(below, cnt, 2 * kDigest, here, st, true, kIdTcLevel);
            if (s != PG_OK) return s;
        } else if (cnt > kWideNodes) {
            const uint64_t *below = nodes + 4 * (2 * n_leaves - ((2 * n_leaves) >> (l - 1)));
            uint64_t *here = nodes + 4 * (2 * n_leaves - ((2 * n_leaves) >> l));
            const unsigned grid = (unsigned)((cnt + 127) / 128);
            ProfScope prof(kIdMerkleLevel, st, cnt);
            if (g.params_set == 1)
                PG_CUDA(launch_dependent(dev::k_merkle_level<dev::kMdsSmall>, grid, 128, st, below, cnt, here));
            else
                PG_CUDA(launch_dependent(dev::k_merkle_level<dev::kMdsFull>, grid, 128, st, below, cnt, here));
        } else {
            const unsigned grid = (unsigned)((cnt * 16 + dev::kTopBlock - 1) / dev::kTopBlock);
            ProfScope prof(kIdMerkleTop, st, cnt);
            PG_CUDA(launch_dependent(dev::k_merkle_top, grid, dev::kTopBlock, st, nodes, n_leaves, l));
        }
    }
    return PG_OK;
}

// Leaf digests of rows[0 .. n) on `st` (k_hash_rows, grid capped like pg_hash_rows).
pg_status launch_leaves(const uint64_t *rows, uint64_t n, uint64_t width, uint64_t *digests, cudaStream_t st) {
    if (g.engine == 1) return launch_tc_sponge(rows, n, width, digests, st, false, kIdTcRows);
    const int vec16 = ((width % 2) == 0 && (reinterpret_cast<uintptr_t>(rows) % 16) == 0) ? 1 : 0;
    const uint64_t want = (n + 127) / 128;
    const uint64_t cap = (uint64_t)g.sms * g.permute_blocks_per_sm * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    ProfScope prof(kIdHashRows, st, n * ((width + kRate - 1) / kRate));
    if (g.params_set == 1) dev::k_hash_rows<dev::kMdsSmall><<<grid, 128, 0, st>>>(rows, n, width, vec16, digests);
    else dev::k_hash_rows<dev::kMdsFull><<<grid, 128, 0, st>>>(rows, n, width, vec16, digests);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

// Launch the persistent Merkle kernel for `tasks` leaf tasks.
pg_status launch_merkle(const pg_schedule *sched, const dev::TreePlan *d_plans, uint32_t n_trees, uint32_t tasks,
                        uint32_t *d_counters, cudaStream_t st, uint64_t perms, bool zcap = false) {
    const uint32_t block = (sched && sched->block == 128) ? 128u : 256u;
    const int occ = block == 128 ? g.merkle128_blocks_per_sm : g.merkle_blocks_per_sm;
    int bps = occ;
    if (sched && sched->blocks_per_sm > 0 && (int)sched->blocks_per_sm < occ) bps = (int)sched->blocks_per_sm;
    const uint32_t warps_per_block = block / 32;
    const uint32_t want = (tasks + warps_per_block - 1) / warps_per_block;
    const uint32_t cap = (uint32_t)(g.sms * bps);
    const unsigned grid = want < cap ? want : cap;
    if (grid == 0) return PG_OK;
    const bool small = g.params_set == 1;
    ProfScope prof(kIdMerkle, st, perms);
    if (block == 128) {
        if (small) dev::k_merkle<128, dev::kMdsSmall><<<grid, 128, 0, st>>>(d_plans, n_trees, tasks, d_counters + 1, d_counters);
        else dev::k_merkle<128, dev::kMdsFull><<<grid, 128, 0, st>>>(d_plans, n_trees, tasks, d_counters + 1, d_counters);
    } else {
        if (zcap && small)
            dev::k_merkle<256, dev::kMdsSmall, true><<<grid, 256, 0, st>>>(d_plans, n_trees, tasks, d_counters + 1, d_counters);
        else if (zcap)
            dev::k_merkle<256, dev::kMdsFull, true><<<grid, 256, 0, st>>>(d_plans, n_trees, tasks, d_counters + 1, d_counters);
        else if (small)
            dev::k_merkle<256, dev::kMdsSmall><<<grid, 256, 0, st>>>(d_plans, n_trees, tasks, d_counters + 1, d_counters);
        else
            dev::k_merkle<256, dev::kMdsFull><<<grid, 256, 0, st>>>(d_plans, n_trees, tasks, d_counters + 1, d_counters);
    }
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

// Permutations of the levels a top-level launch builds (climb_limit < log_n).
uint64_t top_perms_of(const dev::TreePlan *plans, size_t n) {
    uint64_t p = 0;
    for (size_t k = 0; k < n; ++k)
        if (plans[k].climb_limit < plans[k].log_n) p += (plans[k].n_leaves >> plans[k].climb_limit) - 1;
    return p;
}

// The persistent kernel of a batch (tensor or integer engine), then, for
// top_lanes = 16, the 16-lane launch of every tree's top levels.
pg_status launch_batch(const pg_schedule *sched, const dev::TreePlan *d_plans, uint32_t n_trees, uint32_t tasks,
                       uint32_t *d_counters, cudaStream_t st, uint64_t perms, uint64_t top_perms) {
    if (batch_uses_tc(sched)) {
        const uint32_t fuse = sched ? sched->fuse_levels : 0;
        const uint32_t want = (tasks + dev::kTcGroups - 1) / dev::kTcGroups;
        const unsigned grid = want < (uint32_t)g.sms ? want : (uint32_t)g.sms;
        if (grid > 0) {
            ProfScope prof(kIdTcBatch, st, perms - top_perms);
            dev::k_tc_batch<<<grid, dev::kTcThreads, dev::TcL::kBytes, st>>>(d_plans, n_trees, tasks, fuse, d_counters + 1,
                                                                              d_counters);
            PG_CUDA(cudaGetLastError());
        }
    } else {
        pg_status s = launch_merkle(sched, d_plans, n_trees, tasks, d_counters, st, perms - top_perms);
        if (s != PG_OK) return s;
    }
    if (sched && sched->top_lanes == 16) {
        ProfScope prof(kIdBatchTop, st, top_perms);
        dev::k_batch_top<<<n_trees, dev::kBatchTopThreads, 0, st>>>(d_plans);
        PG_CUDA(cudaGetLastError());
    }
    return PG_OK;
}

}  // namespace

int ntt_require_init() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g.init ? (int)PG_OK : fail(PG_ERR_NOT_INIT, "pg_init() has not been called");
}

ProfScope::ProfScope(int kid, void *stream, uint64_t perms) : st_(stream), kid_(kid), perms_(perms) {
    if (!g_prof.on.load(std::memory_order_relaxed)) return;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaGetDevice(&device_) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (g_prof.recs.size() >= kProfMaxRecords) {
        ++g_prof.dropped;
        return;
    }
    cudaEvent_t a = g_prof.take(device_);
    cudaEvent_t b = a ? g_prof.take(device_) : nullptr;
    if (!a || !b || cudaEventRecord(a, st) != cudaSuccess) {
        if (a) g_prof.spare.emplace_back(device_, a);
        if (b) g_prof.spare.emplace_back(device_, b);
        return;
    }
    a_ = a;
    b_ = b;
    active_ = true;
}

ProfScope::~ProfScope() {
    if (!active_) return;
    cudaEvent_t a = static_cast<cudaEvent_t>(a_), b = static_cast<cudaEvent_t>(b_);
    const bool ok = cudaEventRecord(b, static_cast<cudaStream_t>(st_)) == cudaSuccess;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (ok) {
        g_prof.recs.push_back(ProfRecord{kid_, device_, perms_, a, b});
    } else {
        g_prof.spare.emplace_back(device_, a);
        g_prof.spare.emplace_back(device_, b);
    }
}

}  // namespace pg12

struct pg_batch_graph {
    int device;
    pg_schedule sched;
    void *dmem;
    size_t plan_bytes;
    uint32_t n_trees, tasks;
    uint64_t counters;
    uint64_t perms, top_perms;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaStream_t capture;
};

// ------------------------------------------------------------ serving runtime
namespace pg12 {
namespace {

// First-fit allocator over offsets of one device region (256-byte units),
// coalescing freed neighbours.
class PoolAlloc {
  public:
    void init(size_t bytes) {
        free_.clear();
        free_[0] = bytes;
        total_ = bytes;
    }
    static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }
    bool alloc(size_t bytes, size_t &off) {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            off = it->first;
            const size_t rest = it->second - bytes;
            free_.erase(it);
            if (rest) free_[off + bytes] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = round(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t total() const { return total_; }

  private:
    std::map<size_t, size_t> free_;
    size_t total_ = 0;
};

struct ServerReq {
    const uint64_t *rows = nullptr;
    uint64_t n = 0, w = 0;
    size_t off = 0, bytes = 0;
    bool admitted = false;
    int state = PG_REQ_QUEUED;
    int batch = 0;
    double t_submit = 0, t_launch = 0, t_done = 0;
};

struct ServerSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    dev::TreePlan *d_plans = nullptr;
    dev::TreePlan *h_plans = nullptr;  // pinned staging for the plan upload
    uint32_t *d_counters = nullptr;
    size_t counter_words = 0;
    uint32_t *h_flags = nullptr;  // mapped pinned: per-request root-done flags
    uint32_t *d_flags = nullptr;  // device view of h_flags
    std::vector<uint64_t> ids;
    bool busy = false;
};

}  // namespace
}  // namespace pg12

struct pg_server {
    int device = 0;
    pg_server_config cfg{};
    uint8_t *pool = nullptr;
    pg12::PoolAlloc alloc;
    std::vector<pg12::ServerSlot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;  // submitted, not yet launched (arrival order)
    std::unordered_map<uint64_t, pg12::ServerReq> reqs;
    uint64_t next_id = 1;
    size_t outstanding = 0;  // submitted and not yet done or failed
    bool stop = false;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace pg12 {
namespace {

// One scheduling pass (called with the server lock held): retire finished
// batches, then launch what is admissible on a free stream.  Returns true if
// anything changed.
bool server_step(pg_server *s) {
    bool progress = false;
    for (auto &sl : s->slots) {
        if (!sl.busy) continue;
        // requests whose root is already stored finish before their batch does
        const double tf = s->now();
        for (size_t k = 0; k < sl.ids.size(); ++k) {
            if (reinterpret_cast<volatile uint32_t *>(sl.h_flags)[k] == 0u) continue;
            auto &r = s->reqs[sl.ids[k]];
            if (r.state == PG_REQ_RUNNING) {
                r.state = PG_REQ_DONE;
                r.t_done = tf;
                --s->outstanding;
                progress = true;
            }
        }
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        const double t = s->now();
        for (uint64_t id : sl.ids) {
            auto &r = s->reqs[id];
            if (r.state != PG_REQ_RUNNING) continue;  // finished through its flag
            r.state = q == cudaSuccess ? PG_REQ_DONE : PG_REQ_FAILED;
            r.t_done = t;
            --s->outstanding;
        }
        sl.ids.clear();
        sl.busy = false;
        progress = true;
    }
    if (s->queue.empty()) return progress;
    ServerSlot *slot = nullptr;
    for (auto &sl : s->slots)
        if (!sl.busy) {
            slot = &sl;
            break;
        }
    if (!slot) return progress;
    // admit in arrival order; a request whose node buffer does not fit waits
    // while later, smaller ones may pass it
    std::vector<uint64_t> take;
    size_t words = 1;
    for (auto it = s->queue.begin(); it != s->queue.end() && take.size() < s->cfg.max_batch;) {
        auto &r = s->reqs[*it];
        const size_t need = (size_t)((r.n + dev::kWarpNodes - 1) / dev::kWarpNodes) + 1;
        if (words + need > slot->counter_words) break;
        if (!r.admitted) {
            size_t off = 0;
            if (s->alloc.alloc(r.bytes, off)) {
                r.off = off;
                r.admitted = true;
            }
        }
        if (r.admitted) {
            take.push_back(*it);
            words += need;
            it = s->queue.erase(it);
        } else {
            ++it;
        }
    }
    if (take.empty()) return progress;
    std::vector<pg_tree> trees(take.size());
    for (size_t k = 0; k < take.size(); ++k) {
        const auto &r = s->reqs[take[k]];
        trees[k].rows = r.rows;
        trees[k].n_leaves = r.n;
        trees[k].width = r.w;
        trees[k].nodes = reinterpret_cast<uint64_t *>(s->pool + r.off);
    }
    std::vector<dev::TreePlan> plans;
    uint32_t tasks = 0;
    uint64_t counters = 0;
    pg_schedule rs;
    pg_status st = plan_batch(trees.data(), trees.size(), &s->cfg.sched, plans, tasks, counters, rs);
    cudaError_t e = cudaSuccess;
    if (st == PG_OK) {
        // plans may be reordered: match each plan to its request by node buffer
        for (size_t k = 0; k < take.size(); ++k) slot->h_flags[k] = 0u;
        for (auto &pl : plans)
            for (size_t k = 0; k < take.size(); ++k)
                if (pl.nodes == trees[k].nodes) {
                    pl.done_flag = slot->d_flags + k;
                    break;
                }
        std::memcpy(slot->h_plans, plans.data(), plans.size() * sizeof(dev::TreePlan));
        e = cudaMemcpyAsync(slot->d_plans, slot->h_plans, plans.size() * sizeof(dev::TreePlan),
                            cudaMemcpyHostToDevice, slot->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(slot->d_counters, 0, sizeof(uint32_t) * (1 + (size_t)counters), slot->stream);
        if (e == cudaSuccess)
            st = launch_batch(&rs, slot->d_plans, (uint32_t)plans.size(), tasks, slot->d_counters,
                              slot->stream, batch_perms(trees.data(), trees.size()),
                              top_perms_of(plans.data(), plans.size()));
        if (e == cudaSuccess && st == PG_OK) e = cudaEventRecord(slot->done, slot->stream);
    }
    const double t = s->now();
    if (st != PG_OK || e != cudaSuccess) {
        for (uint64_t id : take) {
            auto &r = s->reqs[id];
            r.state = PG_REQ_FAILED;
            r.t_done = t;
            --s->outstanding;
        }
        return true;
    }
    for (uint64_t id : take) {
        auto &r = s->reqs[id];
        r.state = PG_REQ_RUNNING;
        r.t_launch = t;
        r.batch = (int)take.size();
    }
    slot->ids = take;
    slot->busy = true;
    return true;
}

void server_loop(pg_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        const bool progress = server_step(s);
        if (progress) s->cv.notify_all();
        else s->cv.wait_for(lk, std::chrono::microseconds(50));
    }
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

const char *pg_params_sha256(void) {
    static char hex[2][65];
    std::lock_guard<std::mutex> lk(g_mu);
    if (ensure_params() != PG_OK) return nullptr;
    // rc[30][12] then mds[12][12], little-endian words
    uint8_t buf[sizeof g.plain.rc + sizeof g.plain.mds];
    size_t o = 0;
    auto put = [&](uint64_t w) {
        for (int b = 0; b < 8; ++b) buf[o++] = (uint8_t)(w >> (8 * b));
    };
    for (int r = 0; r < kRounds; ++r)
        for (int i = 0; i < kT; ++i) put(g.plain.rc[r][i]);
    for (int i = 0; i < kT; ++i)
        for (int j = 0; j < kT; ++j) put(g.plain.mds[i][j]);
    char *out = hex[g.params_set == 1 ? 1 : 0];
    host::sha256_hex(buf, o, out);
    return out;
}

size_t pg_workspace_bytes(const pg_tree *trees, size_t n_trees) {
    if (!trees) return kWorkspaceBytes;
    uint64_t counters = 0;
    for (size_t k = 0; k < n_trees; ++k) {
        if (!is_pow2(trees[k].n_leaves)) return 0;
        dev::TreePlan tp;
        std::memset(&tp, 0, sizeof tp);
        uint32_t nc = 0;
        plan_tree(tp, trees[k].rows, trees[k].n_leaves, trees[k].width ? trees[k].width : 1, trees[k].nodes, 0, 0, nc);
        counters += nc;
    }
    return kPlanBytes + sizeof(uint32_t) * (1 + (size_t)counters);
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

pg_status pg_params_select(const char *name) {
    std::lock_guard<std::mutex> lk(g_mu);
    int want = 0;
    if (name == nullptr || std::strcmp(name, "pg12_v1") == 0) want = 0;
    else if (std::strcmp(name, "pg12_small") == 0) want = 1;
    else return fail(PG_ERR_PARAMS, "unknown parameter set '%s' (built-in: pg12_v1, pg12_small)", name);
    if (want != g.params_set) {
        g.params_set = want;
        g.params_ready = false;
        ++g.params_gen;
    }
    pg_status s = ensure_params();
    if (s != PG_OK) return s;
    if (g.init) {
        PG_CUDA(cudaSetDevice(g.device));
        s = upload_tables();
        if (s != PG_OK) return s;
    }
    return PG_OK;
}

const char *pg_params_name(void) { return g.params_set == 1 ? "pg12_small" : "pg12_v1"; }

size_t pg_tc_tables_export(void *out, size_t bytes) {
    if (out == nullptr) return sizeof(TcTables);
    if (bytes < sizeof(TcTables)) return 0;
    std::lock_guard<std::mutex> lk(g_mu);
    if (ensure_params() != PG_OK) return 0;
    host::build_tc_tables(g.opt, *static_cast<TcTables *>(out));
    return sizeof(TcTables);
}

pg_status pg_params_export_chain(uint64_t *vp, uint64_t *beta, uint64_t *w) {
    std::lock_guard<std::mutex> lk(g_mu);
    pg_status s = ensure_params();
    if (s != PG_OK) return s;
    ChainParams cp;
    host::derive_chain(g.opt, cp);
    if (vp) std::memcpy(vp, cp.vp, sizeof cp.vp);
    if (beta) std::memcpy(beta, cp.beta, sizeof cp.beta);
    if (w) std::memcpy(w, cp.w, sizeof cp.w);
    return PG_OK;
}

pg_status pg_set_engine(int engine) {
    if (engine != PG_ENGINE_INT && engine != PG_ENGINE_TENSOR)
        return fail(PG_ERR_INVALID_ARG, "unknown engine %d (0: integer pipes, 1: tensor-core dense layers)", engine);
    std::lock_guard<std::mutex> lk(g_mu);
    g.engine = engine;
    return PG_OK;
}

int pg_get_engine(void) { return g.engine; }

pg_status pg_device_faults(uint32_t *faults) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    if (!faults) return fail(PG_ERR_INVALID_ARG, "faults is NULL");
    int v = 0;
    const int zero = 0;
    PG_CUDA(cudaMemcpyFromSymbol(&v, dev::g_tc_fault, sizeof v));
    PG_CUDA(cudaMemcpyToSymbol(dev::g_tc_fault, &zero, sizeof zero));
    *faults = (uint32_t)v;
    return PG_OK;
}

pg_status pg_init(int device, const char *params_path) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g.init && g.device != device) return fail(PG_ERR_INVALID_ARG, "already initialised on device %d", g.device);
    }
    pg_status s = pg_params_select(params_path);
    if (s != PG_OK) return s;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g.init) return PG_OK;  // constants of the selected set already loaded
    int ndev = 0;
    PG_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(PG_ERR_INVALID_ARG, "device %d out of range (%d)", device, ndev);
    PG_CUDA(cudaSetDevice(device));
    s = upload_tables();
    if (s != PG_OK) return s;
    PG_CUDA(cudaFuncSetAttribute(dev::k_tc_permute, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dev::TcL::kBytes));
    PG_CUDA(cudaFuncSetAttribute(dev::k_tc_sponge<dev::kTcGroups, dev::kTcChain>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dev::TcL::kBytes));
    PG_CUDA(cudaFuncSetAttribute(dev::k_tc_sponge<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)dev::TcL1::kBytes));
    PG_CUDA(cudaFuncSetAttribute(dev::k_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dev::TcL::kBytes));
    PG_CUDA(cudaFuncSetAttribute(dev::k_tc_leaves_stream<dev::kTcGroups, dev::kTcChain>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dev::TcL::kBytes));
    PG_CUDA(cudaFuncSetAttribute(dev::k_tc_leaves_stream<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)dev::TcL1::kBytes));
    {
        const int ns = ntt_upload_constants();
        if (ns != PG_OK) return (pg_status)ns;
    }
    PG_CUDA(cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, device));
    {
        int a = 0, b = 0, c = 0, d = 0, e = 0, f = 0, za = 0, zb = 0;
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, dev::k_merkle<256, dev::kMdsFull>, 256, 0));
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, dev::k_merkle<256, dev::kMdsSmall>, 256, 0));
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&za, dev::k_merkle<256, dev::kMdsFull, true>, 256, 0));
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&zb, dev::k_merkle<256, dev::kMdsSmall, true>, 256, 0));
        a = a < za ? a : za;
        b = b < zb ? b : zb;
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, dev::k_merkle<128, dev::kMdsFull>, 128, 0));
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, dev::k_merkle<128, dev::kMdsSmall>, 128, 0));
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e, dev::k_permute<dev::kMdsFull>, dev::kSmallBlock, 0));
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f, dev::k_permute<dev::kMdsSmall>, dev::kSmallBlock, 0));
        int la = 0, lb = 0;
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&la, dev::k_merkle_leaves<dev::kMdsFull>, dev::kBlock, 0));
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lb, dev::k_merkle_leaves<dev::kMdsSmall>, dev::kBlock, 0));
        g.leaves_blocks_per_sm = la < lb ? la : lb;
        g.merkle_blocks_per_sm = a < b ? a : b;
        g.merkle128_blocks_per_sm = c < d ? c : d;
        g.permute_blocks_per_sm = e < f ? e : f;
    }
    if (g.merkle_blocks_per_sm < 1 || g.merkle128_blocks_per_sm < 1 || g.permute_blocks_per_sm < 1 ||
        g.leaves_blocks_per_sm < 1)
        return fail(PG_ERR_CUDA, "kernels cannot be resident (occupancy 0)");
    void *ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, kWorkspaceBytes);
    if (e != cudaSuccess) return fail(PG_ERR_OOM, "workspace cudaMalloc(%zu): %s", kWorkspaceBytes, cudaGetErrorString(e));
    g.ws = static_cast<uint8_t *>(ws);
    g.ws_bytes = kWorkspaceBytes;
    PG_CUDA(cudaStreamCreateWithFlags(&g.copy_st, cudaStreamNonBlocking));
    for (auto &ev : g.host_ev) PG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PG_CUDA(cudaMalloc(&g.d_ready, 256));
    PG_CUDA(cudaMemset(g.d_ready, 0, 256));
    PG_CUDA(cudaHostAlloc(&g.ready_vals, kReadyVals * sizeof(uint32_t), cudaHostAllocDefault));
    for (uint32_t v = 0; v < kReadyVals; ++v) g.ready_vals[v] = v;
    g.ready_base = 0;
    PG_CUDA(cudaEventCreateWithFlags(&g.ready_ev, cudaEventDisableTiming));
    {
        int engines = 0;
        PG_CUDA(cudaDeviceGetAttribute(&engines, cudaDevAttrAsyncEngineCount, device));
        const char *env = std::getenv("PG12_HOST_STREAM");
        g.host_stream = PG12_HOST_STREAM && engines > 0 && !(env && std::strcmp(env, "0") == 0);
    }
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
    if (g.copy_st) cudaStreamDestroy(g.copy_st);
    g.copy_st = nullptr;
    for (auto &ev : g.host_ev) {
        if (ev) cudaEventDestroy(ev);
        ev = nullptr;
    }
    if (g.d_ready) cudaFree(g.d_ready);
    g.d_ready = nullptr;
    if (g.ready_vals) cudaFreeHost(g.ready_vals);
    g.ready_vals = nullptr;
    if (g.ready_ev) cudaEventDestroy(g.ready_ev);
    g.ready_ev = nullptr;
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
    if (g.engine == 1) {
        ProfScope prof(kIdTcPermute, as_stream(stream), (uint64_t)n);
        dev::k_tc_permute<<<tc_grid(n), dev::kTcThreads, dev::TcL::kBytes, as_stream(stream)>>>(states, (uint64_t)n, vec16);
        PG_CUDA(cudaGetLastError());
        return PG_OK;
    }
    const uint64_t want = (n + 127) / 128;
    const uint64_t cap = (uint64_t)g.sms * g.permute_blocks_per_sm * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    ProfScope prof(kIdPermute, as_stream(stream), (uint64_t)n);
    if (g.params_set == 1) dev::k_permute<dev::kMdsSmall><<<grid, 128, 0, as_stream(stream)>>>(states, (uint64_t)n, vec16);
    else dev::k_permute<dev::kMdsFull><<<grid, 128, 0, as_stream(stream)>>>(states, (uint64_t)n, vec16);
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
    if (g.engine == 1) return launch_tc_sponge(rows, n_rows, width, digests, as_stream(stream), false, kIdTcRows);
    const int vec16 = (width % 2 == 0) && (reinterpret_cast<uintptr_t>(rows) % 16) == 0;
    const uint64_t want = (n_rows + 127) / 128;
    const uint64_t cap = (uint64_t)g.sms * g.permute_blocks_per_sm * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    ProfScope prof(kIdHashRows, as_stream(stream), (uint64_t)n_rows * ((width + kRate - 1) / kRate));
    if (g.params_set == 1)
        dev::k_hash_rows<dev::kMdsSmall><<<grid, 128, 0, as_stream(stream)>>>(rows, (uint64_t)n_rows, (uint64_t)width, vec16, digests);
    else
        dev::k_hash_rows<dev::kMdsFull><<<grid, 128, 0, as_stream(stream)>>>(rows, (uint64_t)n_rows, (uint64_t)width, vec16, digests);
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
    if (n_leaves > (1ull << 34)) return fail(PG_ERR_INVALID_ARG, "n_leaves=%zu above 2^34", n_leaves);
    if (reinterpret_cast<uintptr_t>(rows) % 8) return fail(PG_ERR_INVALID_ARG, "rows not 8-byte aligned");
    if (reinterpret_cast<uintptr_t>(nodes) % 16) return fail(PG_ERR_INVALID_ARG, "nodes not 16-byte aligned");
    if (overlaps(rows, (size_t)n_leaves * width * 8, nodes, ((size_t)2 * n_leaves - 1) * 32))
        return fail(PG_ERR_INVALID_ARG, "rows and nodes overlap");
    cudaStream_t st = as_stream(stream);
    // the leaves in one launch, then one launch per level (launch_levels);
    // nothing but rows and nodes is read or written, so concurrent builds on
    // different streams are independent
    const uint32_t first_top = 1;
    if ((uint64_t)n_leaves <= (g.engine == 1 ? kTcSmallTree : kSmallTree)) {  // whole tree in the 16-lane form
        const uint64_t threads = (uint64_t)n_leaves * 16;
        const unsigned grid = (unsigned)((threads + dev::kTopBlock - 1) / dev::kTopBlock);
        ProfScope prof(kIdMerkleTopLeaf, st, (uint64_t)n_leaves * ((width + kRate - 1) / kRate));
        dev::k_merkle_top_leaf<<<grid, dev::kTopBlock, 0, st>>>(rows, (uint64_t)n_leaves, (uint64_t)width, nodes);
        PG_CUDA(cudaGetLastError());
    } else if (g.engine == 1) {
        s = launch_tc_sponge(rows, n_leaves, width, nodes, st, false, kIdTcLeaves);
        if (s != PG_OK) return s;
    } else {
        dev::TreePlan tp;
        std::memset(&tp, 0, sizeof tp);
        uint32_t n_counters = 0;
        const uint32_t tasks = plan_tree(tp, rows, n_leaves, width, nodes, 0, 0, n_counters);
        const uint32_t want = (tasks + dev::kBlock / 32 - 1) / (dev::kBlock / 32);
        const uint32_t cap = (uint32_t)(g.sms * g.leaves_blocks_per_sm);
        const unsigned grid = want < cap ? want : cap;
        ProfScope prof(kIdMerkle, st, (uint64_t)n_leaves * ((width + kRate - 1) / kRate));
        if (g.params_set == 1) dev::k_merkle_leaves<dev::kMdsSmall><<<grid, dev::kBlock, 0, st>>>(tp, tasks);
        else dev::k_merkle_leaves<dev::kMdsFull><<<grid, dev::kBlock, 0, st>>>(tp, tasks);
        PG_CUDA(cudaGetLastError());
    }
    s = launch_levels(nodes, n_leaves, first_top, st);
    if (s != PG_OK) return s;
    if (root_out) {
        PG_CUDA(cudaMemcpyAsync(root_out, nodes + 4 * (2 * n_leaves - 2), 32, cudaMemcpyDeviceToHost, st));
        PG_CUDA(cudaStreamSynchronize(st));
    }
    return PG_OK;
}

// Host-row builds: the copied chunks' ends (at most 16).  The first chunk
// holds n / FIRST_DIV rows, each next one twice as many, up to n / MAX_DIV;
// once at most two of those are left, each chunk takes half of the rest (not
// below n / FIRST_DIV).  When the host link is faster than the hashing, the
// copies run ahead and the sizes hardly matter; when it is slower, the
// hashing keeps pace with the copies and what is left after the last copy
// lands is one small chunk.
#ifndef PG12_HOST_CHUNK_FIRST_DIV
#define PG12_HOST_CHUNK_FIRST_DIV 64
#endif
#ifndef PG12_HOST_CHUNK_MAX_DIV
#define PG12_HOST_CHUNK_MAX_DIV 8
#endif
static_assert(PG12_HOST_CHUNK_FIRST_DIV >= PG12_HOST_CHUNK_MAX_DIV, "host chunks: the first is the smallest");

uint32_t host_chunks(uint64_t n, uint64_t (&end)[16]) {
    const uint64_t lo = n / PG12_HOST_CHUNK_FIRST_DIV > 0 ? n / PG12_HOST_CHUNK_FIRST_DIV : 1;
    const uint64_t hi = n / PG12_HOST_CHUNK_MAX_DIV > lo ? n / PG12_HOST_CHUNK_MAX_DIV : lo;
    uint64_t grow = lo, first = 0;
    uint32_t c = 0;
    while (first < n) {
        const uint64_t rem = n - first;
        uint64_t rows = rem <= 2 * hi ? rem / 2 : grow;
        if (rows < lo) rows = lo;
        if (rows >= rem || rem - rows < lo || c == 15) rows = rem;
        first += rows;
        end[c++] = first;
        if (grow < hi) grow <<= 1;
    }
    return c;
}

pg_status pg_merkle_build_host(const uint64_t *rows_host, size_t n_leaves, size_t width, uint64_t *rows_dev,
                               uint64_t *nodes, uint64_t *root_out, void *stream) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    if (!rows_host || !rows_dev || !nodes) return fail(PG_ERR_INVALID_ARG, "rows_host, rows_dev or nodes is NULL");
    if (width == 0) return fail(PG_ERR_INVALID_ARG, "width must be >= 1");
    if (!is_pow2(n_leaves)) return fail(PG_ERR_NOT_POW2, "n_leaves=%zu is not a power of two", n_leaves);
    if (n_leaves > (1ull << 34)) return fail(PG_ERR_INVALID_ARG, "n_leaves=%zu above 2^34", n_leaves);
    if (reinterpret_cast<uintptr_t>(rows_dev) % 8) return fail(PG_ERR_INVALID_ARG, "rows_dev not 8-byte aligned");
    if (reinterpret_cast<uintptr_t>(nodes) % 16) return fail(PG_ERR_INVALID_ARG, "nodes not 16-byte aligned");
    if (overlaps(rows_dev, (size_t)n_leaves * width * 8, nodes, ((size_t)2 * n_leaves - 1) * 32))
        return fail(PG_ERR_INVALID_ARG, "rows_dev and nodes overlap");
    cudaStream_t st = as_stream(stream);
    const uint64_t n = n_leaves, bytes_per_row = 8 * (uint64_t)width;
    // below 64 MiB of rows the copy takes less than the extra launches would
    // save: one copy, then the device-rows build
    if (n <= kSmallTree || n * bytes_per_row < (64ull << 20)) {
        PG_CUDA(cudaMemcpyAsync(rows_dev, rows_host, n * bytes_per_row, cudaMemcpyHostToDevice, st));
        return pg_merkle_build(rows_dev, n_leaves, width, nodes, root_out, stream);
    }
    // The chunks (host_chunks): small first so hashing starts early, then
    // n / 8 rows, halving again toward the end.  The copies into rows_dev wait
    // for work already queued on `st` (an earlier build may still read it).
    PG_CUDA(cudaEventRecord(g.host_ev[16], st));
    PG_CUDA(cudaStreamWaitEvent(g.copy_st, g.host_ev[16], 0));
    uint64_t ends[16];
    const uint32_t nchunks = host_chunks(n, ends);
    if (g.engine == 1 && g.host_stream) {
        // Tensor engine: one leaf launch for all chunks.  After each chunk's
        // rows the copy stream copies the arrival value base + c + 1 into
        // d_ready (a copy-engine write; the waiting kernel needs no other
        // kernel to run), and the launch's groups wait for the chunk of each
        // unit before reading it.  Every build takes 16 fresh values; when
        // they run out, the counter restarts at 0 once the last streaming
        // launch has finished (no launch can then be waiting on it).
        if (g.ready_base + 16 >= kReadyVals) {
            PG_CUDA(cudaEventSynchronize(g.ready_ev));
            PG_CUDA(cudaMemcpyAsync(g.d_ready, g.ready_vals, sizeof(uint32_t), cudaMemcpyHostToDevice, g.copy_st));
            // this build's launch must not see the old, larger value
            PG_CUDA(cudaEventRecord(g.host_ev[15], g.copy_st));
            PG_CUDA(cudaStreamWaitEvent(st, g.host_ev[15], 0));
            g.ready_base = 0;
        }
        dev::ChunkMap cm = {};
        cm.base = g.ready_base;
        for (uint32_t c = 0; c < nchunks; ++c) {
            const uint64_t first = c ? ends[c - 1] : 0, rows_c = ends[c] - first;
            PG_CUDA(cudaMemcpyAsync(rows_dev + first * width, rows_host + first * width, rows_c * bytes_per_row,
                                    cudaMemcpyHostToDevice, g.copy_st));
            PG_CUDA(cudaMemcpyAsync(g.d_ready, g.ready_vals + cm.base + c + 1, sizeof(uint32_t),
                                    cudaMemcpyHostToDevice, g.copy_st));
            cm.end[c] = ends[c];
            cm.count = c + 1;
        }
        g.ready_base += 16;
        // every copy is queued before the launch, so that they run even where
        // launches block the host until they finish (CUDA_LAUNCH_BLOCKING)
        s = launch_leaves_stream(rows_dev, n, width, nodes, g.d_ready, cm, st);
        if (s != PG_OK) return s;
        PG_CUDA(cudaEventRecord(g.ready_ev, st));
        s = launch_levels(nodes, n, 1, st);
        if (s != PG_OK) return s;
        if (root_out) {
            PG_CUDA(cudaMemcpyAsync(root_out, nodes + 4 * (2 * n - 2), 32, cudaMemcpyDeviceToHost, st));
            PG_CUDA(cudaStreamSynchronize(st));
        }
        return PG_OK;
    }
    for (uint32_t c = 0; c < nchunks; ++c) {
        const uint64_t first = c ? ends[c - 1] : 0, rows_c = ends[c] - first;
        PG_CUDA(cudaMemcpyAsync(rows_dev + first * width, rows_host + first * width, rows_c * bytes_per_row,
                                cudaMemcpyHostToDevice, g.copy_st));
        PG_CUDA(cudaEventRecord(g.host_ev[c], g.copy_st));
        PG_CUDA(cudaStreamWaitEvent(st, g.host_ev[c], 0));
        s = launch_leaves(rows_dev + first * width, rows_c, width, nodes + 4 * first, st);
        if (s != PG_OK) return s;
    }
    s = launch_levels(nodes, n, 1, st);
    if (s != PG_OK) return s;
    if (root_out) {
        PG_CUDA(cudaMemcpyAsync(root_out, nodes + 4 * (2 * n - 2), 32, cudaMemcpyDeviceToHost, st));
        PG_CUDA(cudaStreamSynchronize(st));
    }
    return PG_OK;
}

pg_status pg_merkle_build_batch(const pg_tree *trees, size_t n_trees, const pg_schedule *sched, void *stream) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    std::vector<dev::TreePlan> plans;
    uint32_t tasks = 0;
    uint64_t counters = 0;
    pg_schedule rs;
    s = plan_batch(trees, n_trees, sched, plans, tasks, counters, rs);
    if (s != PG_OK) return s;
    const size_t plan_bytes = plans.size() * sizeof(dev::TreePlan);
    const size_t counter_bytes = sizeof(uint32_t) * (1 + (size_t)counters);
    if (plan_bytes > kPlanBytes || counter_bytes > g.ws_bytes - kPlanBytes)
        return fail(PG_ERR_OOM, "batch needs %zu plan bytes and %zu counter bytes; workspace holds %zu and %zu", plan_bytes,
                    counter_bytes, kPlanBytes, g.ws_bytes - kPlanBytes);
    cudaStream_t st = as_stream(stream);
    auto *d_plan = reinterpret_cast<dev::TreePlan *>(g.ws);
    auto *d_counters = reinterpret_cast<uint32_t *>(g.ws + kPlanBytes);
    PG_CUDA(cudaMemcpyAsync(d_plan, plans.data(), plan_bytes, cudaMemcpyHostToDevice, st));
    PG_CUDA(cudaMemsetAsync(d_counters, 0, counter_bytes, st));
    return launch_batch(&rs, d_plan, (uint32_t)plans.size(), tasks, d_counters, st, batch_perms(trees, n_trees),
                        top_perms_of(plans.data(), plans.size()));
}

pg_status pg_batch_graph_create(const pg_tree *trees, size_t n_trees, const pg_schedule *sched,
                                pg_batch_graph **out) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    if (!out) return fail(PG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::vector<dev::TreePlan> plans;
    uint32_t tasks = 0;
    uint64_t counters = 0;
    pg_schedule rs;
    s = plan_batch(trees, n_trees, sched, plans, tasks, counters, rs);
    if (s != PG_OK) return s;
    auto *h = new (std::nothrow) pg_batch_graph();
    if (!h) return fail(PG_ERR_OOM, "host allocation failed");
    h->device = g.device;
    h->sched = rs;
    h->plan_bytes = plans.size() * sizeof(dev::TreePlan);
    h->n_trees = (uint32_t)plans.size();
    h->tasks = tasks;
    h->counters = counters;
    h->perms = batch_perms(trees, n_trees);
    h->top_perms = top_perms_of(plans.data(), plans.size());
    const size_t plan_bytes_aligned = (h->plan_bytes + 255) & ~(size_t)255;
    const size_t total = plan_bytes_aligned + sizeof(uint32_t) * (1 + (size_t)counters);
    cudaError_t e = cudaMalloc(&h->dmem, total);
    if (e != cudaSuccess) {
        delete h;
        return fail(PG_ERR_OOM, "batch graph cudaMalloc(%zu): %s", total, cudaGetErrorString(e));
    }
    auto cleanup = [&](pg_status st_) {
        if (h->exec) cudaGraphExecDestroy(h->exec);
        if (h->graph) cudaGraphDestroy(h->graph);
        if (h->capture) cudaStreamDestroy(h->capture);
        cudaFree(h->dmem);
        delete h;
        return st_;
    };
    auto *d_plan = static_cast<dev::TreePlan *>(h->dmem);
    auto *d_counters = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(h->dmem) + plan_bytes_aligned);
    e = cudaMemcpy(d_plan, plans.data(), h->plan_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cleanup(fail(PG_ERR_CUDA, "plan upload: %s", cudaGetErrorString(e)));
    e = cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail(PG_ERR_CUDA, "stream create: %s", cudaGetErrorString(e)));
    e = cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cleanup(fail(PG_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e)));
    cudaError_t e_memset = cudaMemsetAsync(d_counters, 0, sizeof(uint32_t) * (1 + (size_t)counters), h->capture);
    pg_status sl = launch_batch(&h->sched, d_plan, h->n_trees, tasks, d_counters, h->capture, h->perms, h->top_perms);
    e = cudaStreamEndCapture(h->capture, &h->graph);
    if (e_memset != cudaSuccess || sl != PG_OK || e != cudaSuccess)
        return cleanup(sl != PG_OK ? sl : fail(PG_ERR_CUDA, "capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e_memset)));
    e = cudaGraphInstantiate(&h->exec, h->graph, 0);
    if (e != cudaSuccess) return cleanup(fail(PG_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)));
    *out = h;
    return PG_OK;
}

pg_status pg_batch_graph_launch(pg_batch_graph *graph, void *stream) {
    if (!graph) return fail(PG_ERR_INVALID_ARG, "graph is NULL");
    pg12::ProfScope prof(pg12::kIdGraph, as_stream(stream), graph->perms);
    PG_CUDA(cudaGraphLaunch(graph->exec, as_stream(stream)));
    return PG_OK;
}

pg_status pg_batch_graph_destroy(pg_batch_graph *graph) {
    if (!graph) return PG_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    if (graph->capture) cudaStreamDestroy(graph->capture);
    cudaFree(graph->dmem);
    delete graph;
    if (e != cudaSuccess) return fail(PG_ERR_CUDA, "destroy: %s", cudaGetErrorString(e));
    return PG_OK;
}

pg_status pg_batch_autotune(const pg_tree *trees, size_t n_trees, void *stream, pg_schedule *best,
                            float *best_ms) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    if (!best) return fail(PG_ERR_INVALID_ARG, "best is NULL");
    cudaStream_t st = as_stream(stream);
    std::vector<pg_schedule> cands;
    for (uint32_t order = 0; order <= 1; ++order)
        for (uint32_t top : {1u, 16u}) {
            for (uint32_t fuse = 0; fuse <= 2; ++fuse) {
                pg_schedule c{};
                c.engine = PG_BATCH_ENGINE_TENSOR;
                c.order = order;
                c.fuse_levels = fuse;
                c.top_lanes = top;
                cands.push_back(c);
            }
            for (uint32_t b : {256u, 128u}) {
                pg_schedule c{};
                c.engine = PG_BATCH_ENGINE_INT;
                c.block = b;
                c.order = order;
                c.top_lanes = top;
                cands.push_back(c);
            }
        }
    cudaEvent_t e0, e1;
    PG_CUDA(cudaEventCreate(&e0));
    PG_CUDA(cudaEventCreate(&e1));
    float top_ms = -1.f;
    pg_schedule win{};
    for (const pg_schedule &c : cands) {
        s = pg_merkle_build_batch(trees, n_trees, &c, stream);  // warm-up
        if (s != PG_OK) break;
        float tot = 0.f;
        const int reps = 3;
        for (int r = 0; r < reps && s == PG_OK; ++r) {
            cudaEventRecord(e0, st);
            s = pg_merkle_build_batch(trees, n_trees, &c, stream);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            tot += ms;
        }
        if (s != PG_OK) break;
        const float avg = tot / reps;
        if (top_ms < 0.f || avg < top_ms) {
            top_ms = avg;
            win = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != PG_OK) return s;
    *best = win;
    if (best_ms) *best_ms = top_ms;
    return PG_OK;
}

pg_status pg_server_create(const pg_server_config *cfg, pg_server **out) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    if (!out) return fail(PG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    auto *srv = new (std::nothrow) pg_server();
    if (!srv) return fail(PG_ERR_OOM, "host allocation failed");
    if (cfg) srv->cfg = *cfg;
    if (srv->cfg.pool_bytes == 0) srv->cfg.pool_bytes = (size_t)4 << 30;
    if (srv->cfg.max_batch == 0) srv->cfg.max_batch = 256;
    if (srv->cfg.max_inflight == 0) srv->cfg.max_inflight = 2;
    if (srv->cfg.max_inflight > 8) srv->cfg.max_inflight = 8;
    srv->device = g.device;
    srv->t0 = std::chrono::steady_clock::now();
    auto cleanup = [&](pg_status st_) {
        for (auto &sl : srv->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.d_plans) cudaFree(sl.d_plans);
            if (sl.d_counters) cudaFree(sl.d_counters);
            if (sl.h_plans) cudaFreeHost(sl.h_plans);
            if (sl.h_flags) cudaFreeHost(sl.h_flags);
        }
        if (srv->pool) cudaFree(srv->pool);
        delete srv;
        return st_;
    };
    cudaError_t e = cudaMalloc(&srv->pool, srv->cfg.pool_bytes);
    if (e != cudaSuccess) return cleanup(fail(PG_ERR_OOM, "server pool cudaMalloc(%zu): %s", srv->cfg.pool_bytes, cudaGetErrorString(e)));
    srv->alloc.init(srv->cfg.pool_bytes);
    srv->slots.resize(srv->cfg.max_inflight);
    for (auto &sl : srv->slots) {
        sl.counter_words = srv->cfg.pool_bytes / 512 + 1024 + 2 * (size_t)srv->cfg.max_batch;
        const size_t plan_bytes = sizeof(dev::TreePlan) * srv->cfg.max_batch;
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_plans, plan_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_counters, sizeof(uint32_t) * sl.counter_words);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_plans, plan_bytes);
        if (e == cudaSuccess)
            e = cudaHostAlloc(&sl.h_flags, sizeof(uint32_t) * srv->cfg.max_batch, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&sl.d_flags, sl.h_flags, 0);
        if (e != cudaSuccess) return cleanup(fail(PG_ERR_OOM, "server stream buffers: %s", cudaGetErrorString(e)));
    }
    srv->worker = std::thread(server_loop, srv);
    *out = srv;
    return PG_OK;
}

pg_status pg_server_submit(pg_server *srv, const uint64_t *rows, uint64_t n_leaves, uint64_t width, uint64_t *id_out) {
    if (!srv || !rows || !id_out) return fail(PG_ERR_INVALID_ARG, "NULL argument");
    if (width == 0) return fail(PG_ERR_INVALID_ARG, "width must be >= 1");
    if (!is_pow2(n_leaves)) return fail(PG_ERR_NOT_POW2, "n_leaves=%llu is not a power of two", (unsigned long long)n_leaves);
    if (reinterpret_cast<uintptr_t>(rows) % 8) return fail(PG_ERR_INVALID_ARG, "rows not 8-byte aligned");
    const size_t bytes = (size_t)(2 * n_leaves - 1) * 32;
    if (PoolAlloc::round(bytes) > srv->alloc.total())
        return fail(PG_ERR_OOM, "request needs %zu node bytes, the pool holds %zu", bytes, srv->alloc.total());
    if ((n_leaves + dev::kWarpNodes - 1) / dev::kWarpNodes + 2 > srv->slots[0].counter_words)
        return fail(PG_ERR_OOM, "request needs more arrival counters than a stream holds");
    std::lock_guard<std::mutex> lk(srv->mu);
    const uint64_t id = srv->next_id++;
    ServerReq r;
    r.rows = rows;
    r.n = n_leaves;
    r.w = width;
    r.bytes = bytes;
    r.t_submit = srv->now();
    srv->reqs.emplace(id, r);
    srv->queue.push_back(id);
    ++srv->outstanding;
    *id_out = id;
    srv->cv.notify_all();
    return PG_OK;
}

pg_status pg_server_query(pg_server *srv, uint64_t id, pg_request_info *info) {
    if (!srv || !info) return fail(PG_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(PG_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)id);
    const auto &r = it->second;
    info->state = r.state;
    info->batch_size = r.batch;
    info->submit_s = r.t_submit;
    info->launch_s = r.t_launch;
    info->done_s = r.t_done;
    info->nodes = r.admitted ? reinterpret_cast<const uint64_t *>(srv->pool + r.off) : nullptr;
    return PG_OK;
}

pg_status pg_server_release(pg_server *srv, uint64_t id) {
    if (!srv) return fail(PG_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(PG_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)id);
    if (it->second.state != PG_REQ_DONE && it->second.state != PG_REQ_FAILED)
        return fail(PG_ERR_INVALID_ARG, "request %llu is still in flight", (unsigned long long)id);
    if (it->second.admitted) srv->alloc.release(it->second.off, it->second.bytes);
    srv->reqs.erase(it);
    srv->cv.notify_all();
    return PG_OK;
}

pg_status pg_server_drain(pg_server *srv, double timeout_s) {
    if (!srv) return fail(PG_ERR_INVALID_ARG, "NULL server");
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (srv->outstanding > 0) {
        if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout && srv->outstanding > 0)
            return fail(PG_ERR_TIMEOUT, "drain: %zu requests still outstanding after %.3f s", srv->outstanding, timeout_s);
    }
    return PG_OK;
}

pg_status pg_server_destroy(pg_server *srv) {
    if (!srv) return PG_OK;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    cudaError_t e = cudaSuccess;
    for (auto &sl : srv->slots) {
        if (sl.stream) {
            cudaError_t e2 = cudaStreamSynchronize(sl.stream);
            if (e == cudaSuccess) e = e2;
            cudaStreamDestroy(sl.stream);
        }
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.d_plans) cudaFree(sl.d_plans);
        if (sl.d_counters) cudaFree(sl.d_counters);
        if (sl.h_plans) cudaFreeHost(sl.h_plans);
        if (sl.h_flags) cudaFreeHost(sl.h_flags);
    }
    if (srv->pool) cudaFree(srv->pool);
    delete srv;
    if (e != cudaSuccess) return fail(PG_ERR_CUDA, "server destroy: %s", cudaGetErrorString(e));
    return PG_OK;
}

pg_status pg_merkle_open(const uint64_t *nodes, size_t n_leaves, const uint64_t *indices, size_t k,
                         uint64_t *paths, void *stream) {
    if (!is_pow2(n_leaves)) return fail(PG_ERR_NOT_POW2, "n_leaves=%zu is not a power of two", n_leaves);
    if (k == 0) return PG_OK;
    if (!nodes || !indices || !paths) return fail(PG_ERR_INVALID_ARG, "NULL buffer");
    const uint32_t depth = log2u(n_leaves);
    if (depth == 0) return PG_OK;  // a one-leaf tree has empty paths
    const uint64_t threads = (uint64_t)k * depth;
    const unsigned grid = (unsigned)((threads + 255) / 256);
    pg12::ProfScope prof(pg12::kIdOpen, as_stream(stream), 0);
    dev::k_merkle_open<<<grid, 256, 0, as_stream(stream)>>>(nodes, (uint64_t)n_leaves, depth, indices, (uint64_t)k, paths);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

pg_status pg_merkle_verify(const uint64_t *root, size_t n_leaves, const uint64_t *leaves, const uint64_t *indices,
                           size_t k, const uint64_t *paths, uint8_t *ok, void *stream) {
    pg_status s = require_init();
    if (s != PG_OK) return s;
    if (!is_pow2(n_leaves)) return fail(PG_ERR_NOT_POW2, "n_leaves=%zu is not a power of two", n_leaves);
    if (k == 0) return PG_OK;
    if (!root || !leaves || !indices || !ok || (!paths && n_leaves > 1)) return fail(PG_ERR_INVALID_ARG, "NULL buffer");
    const uint32_t depth = log2u(n_leaves);
    const unsigned grid = (unsigned)((k + dev::kVerifyBlock - 1) / dev::kVerifyBlock);
    ProfScope prof(kIdVerify, as_stream(stream), (uint64_t)k * depth);
    if (g.params_set == 1)
        dev::k_merkle_verify<dev::kMdsSmall><<<grid, dev::kVerifyBlock, 0, as_stream(stream)>>>(root, depth, (uint64_t)n_leaves,
                                                                                             leaves, indices, (uint64_t)k, paths, ok);
    else
        dev::k_merkle_verify<dev::kMdsFull><<<grid, dev::kVerifyBlock, 0, as_stream(stream)>>>(root, depth, (uint64_t)n_leaves,
                                                                                            leaves, indices, (uint64_t)k, paths, ok);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

// Allocation-free variant of pg_merkle_build (declared in include/pg12.h).
// Its first call on a device, and its first call on that device after the
// active parameter set has changed, does the set-up with the device current:
// it uploads the constant tables (cudaMemcpyToSymbol, synchronous) and
// resolves the device address of g_noalloc_scratch with
// cudaGetSymbolAddress -- in host code the array's name is only a host-side
// stand-in and must never be handed to a kernel.  Make those calls before
// any stream capture.
pg_status pg_merkle_build_noalloc(const uint64_t *rows, size_t n_leaves, size_t width, uint64_t *nodes,
                                  void *stream) {
    constexpr int kMaxDevices = 64;
    static uint32_t *scratch_ptr[kMaxDevices];
    static int blocks_per_sm[kMaxDevices];
    static int sm_count[kMaxDevices];
    static int consts_gen[kMaxDevices];  // parameter-set generation loaded on each device
    if (!rows || !nodes) return fail(PG_ERR_INVALID_ARG, "rows or nodes is NULL");
    if (width == 0) return fail(PG_ERR_INVALID_ARG, "width must be >= 1");
    if (!is_pow2(n_leaves)) return fail(PG_ERR_NOT_POW2, "n_leaves=%zu is not a power of two", n_leaves);
    if (n_leaves > dev::kNoAllocMaxLeaves)
        return fail(PG_ERR_INVALID_ARG, "n_leaves=%zu exceeds the allocation-free limit of %llu leaves", n_leaves,
                    (unsigned long long)dev::kNoAllocMaxLeaves);
    if (reinterpret_cast<uintptr_t>(rows) % 8) return fail(PG_ERR_INVALID_ARG, "rows not 8-byte aligned");
    if (reinterpret_cast<uintptr_t>(nodes) % 16) return fail(PG_ERR_INVALID_ARG, "nodes not 16-byte aligned");
    if (overlaps(rows, (size_t)n_leaves * width * 8, nodes, ((size_t)2 * n_leaves - 1) * 32))
        return fail(PG_ERR_INVALID_ARG, "rows and nodes overlap");
    int device = 0;
    PG_CUDA(cudaGetDevice(&device));
    if (device < 0 || device >= kMaxDevices) return fail(PG_ERR_INVALID_ARG, "device %d out of range", device);
    int params_set = 0;  // the set whose constants this call's kernel uses, read with them
    {
        std::lock_guard<std::mutex> lk(g_mu);
        params_set = g.params_set;
        if (scratch_ptr[device] == nullptr || consts_gen[device] != g.params_gen) {
            pg_status s = ensure_params();
            if (s != PG_OK) return s;
            dev::DevConsts dc;
            dev::make_dev_consts(g.opt, dc);
            PG_CUDA(cudaMemcpyToSymbol(dev::c_dev, &dc, sizeof(dc)));
            consts_gen[device] = g.params_gen;
            PG_CUDA(cudaDeviceGetAttribute(&sm_count[device], cudaDevAttrMultiProcessorCount, device));
            int oa = 0, ob = 0;
            PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oa, dev::k_merkle_single<dev::kMdsFull>, dev::kBlock, 0));
            PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, dev::k_merkle_single<dev::kMdsSmall>, dev::kBlock, 0));
            blocks_per_sm[device] = oa < ob ? oa : ob;
            if (blocks_per_sm[device] < 1) return fail(PG_ERR_CUDA, "k_merkle_single cannot be resident");
            void *p = nullptr;
            PG_CUDA(cudaGetSymbolAddress(&p, dev::g_noalloc_scratch));
            scratch_ptr[device] = static_cast<uint32_t *>(p);
        }
    }
    uint32_t *scratch = scratch_ptr[device];
    dev::TreePlan tp;
    std::memset(&tp, 0, sizeof tp);
    uint32_t n_counters = 0;
    const uint32_t tasks = plan_tree(tp, rows, n_leaves, width, nodes, 0, 0, n_counters);
    if (1 + (size_t)n_counters > dev::kNoAllocWords)
        return fail(PG_ERR_INVALID_ARG, "n_leaves=%zu needs more scratch than the allocation-free limit", n_leaves);
    cudaStream_t st = as_stream(stream);
    // the array keeps the previous call's counts: clear what this call uses
    PG_CUDA(cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * (1 + (size_t)n_counters), st));
    const uint32_t warps_per_block = dev::kBlock / 32;
    const uint32_t want = (tasks + warps_per_block - 1) / warps_per_block;
    const uint32_t cap = (uint32_t)(sm_count[device] * blocks_per_sm[device]);
    const unsigned grid = want < cap ? want : cap;
    ProfScope prof(kIdSingle, st, tree_perms(n_leaves, width));
    if (params_set == 1) dev::k_merkle_single<dev::kMdsSmall><<<grid, dev::kBlock, 0, st>>>(tp, tasks, scratch + 1, scratch);
    else dev::k_merkle_single<dev::kMdsFull><<<grid, dev::kBlock, 0, st>>>(tp, tasks, scratch + 1, scratch);
    PG_CUDA(cudaGetLastError());
    return PG_OK;
}

pg_status pg_profile_enable(int on) {
    std::vector<pg12::ProfRecord> old;
    {
        std::lock_guard<std::mutex> lk(pg12::g_prof.mu);
        pg12::g_prof.on.store(on != 0);
        old.swap(pg12::g_prof.recs);
        pg12::g_prof.dropped = 0;
    }
    // events of discarded records go back to the spare list once they have completed
    for (auto &r : old) cudaEventSynchronize(r.b);
    std::lock_guard<std::mutex> lk(pg12::g_prof.mu);
    for (auto &r : old) {
        pg12::g_prof.spare.emplace_back(r.device, r.a);
        pg12::g_prof.spare.emplace_back(r.device, r.b);
    }
    return PG_OK;
}

pg_status pg_profile_read(pg_kernel_time *out, size_t cap, size_t *n_out, uint64_t *dropped) {
    std::vector<pg12::ProfRecord> recs;
    uint64_t drop = 0;
    {
        std::lock_guard<std::mutex> lk(pg12::g_prof.mu);
        recs.swap(pg12::g_prof.recs);
        drop = pg12::g_prof.dropped;
        pg12::g_prof.dropped = 0;
    }
    pg_kernel_time acc[pg12::kIdCount];
    std::memset(acc, 0, sizeof acc);
    cudaError_t err = cudaSuccess;
    for (auto &r : recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        acc[r.kid].launches += 1;
        acc[r.kid].perms += r.perms;
        acc[r.kid].total_ms += ms;
    }
    {
        std::lock_guard<std::mutex> lk(pg12::g_prof.mu);
        for (auto &r : recs) {
            pg12::g_prof.spare.emplace_back(r.device, r.a);
            pg12::g_prof.spare.emplace_back(r.device, r.b);
        }
    }
    size_t n = 0;
    for (int kid = 0; kid < pg12::kIdCount; ++kid) {
        if (acc[kid].launches == 0) continue;
        if (out && n < cap) {
            out[n] = acc[kid];
            std::snprintf(out[n].name, sizeof out[n].name, "%s", pg12::kKernelNames[kid]);
        }
        ++n;
    }
    if (n_out) *n_out = n;
    if (dropped) *dropped = drop;
    if (err != cudaSuccess) return fail(PG_ERR_CUDA, "profile events: %s", cudaGetErrorString(err));
    if (out && n > cap) return fail(PG_ERR_INVALID_ARG, "profile has %zu kernels, cap is %zu", n, cap);
    return PG_OK;
}

}  // extern "C"
