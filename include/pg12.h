/*
 * pg12.h -- C ABI of the GB300 Poseidon-12 / Goldilocks Merkle library.
 *
 * Everything here follows arXiv 2506.09505:
 *   field        Eq. 1: p = 2^64 - 2^32 + 1; an element is canonical when
 *                0 <= e < p (Sec. 2.4).
 *   permutation  Alg. 1 and Sec. 2.4: width 12, S-box x^7, 4 + 22 + 4 rounds
 *                (HALF_FULL_ROUNDS = 4, PARTIAL_ROUNDS = 22), 12x12 MDS layer.
 *   sponge       Sec. 2.4: rate 8 (chunks of eight elements), capacity 4,
 *                4-element digest; overwrite mode, short last chunk
 *                zero-filled.
 *   Merkle tree  Sec. 2.4 and Sec. 4.2: leaves are hashes of the data rows,
 *                each parent hashes the concatenation of its two children,
 *                level by level up to the root.
 *
 * Conventions shared by every call
 *   - Elements are uint64_t, little-endian words.  Any 64-bit input word is
 *     accepted and taken mod p; every output word is canonical (< p).
 *   - "dev" pointers are CUDA device pointers on the device given to
 *     pg_init(); the caller allocates and owns every buffer.  The library
 *     owns only its constant tables and a small workspace it allocates in
 *     pg_init() (released by pg_shutdown()).
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream) unless stated otherwise.  Argument
 *     errors are detected on the host and returned before anything is
 *     launched.  CUDA errors map to PG_ERR_CUDA; pg_last_error() gives the
 *     text.  Device-side waits (on the tensor cores' completion barriers and
 *     on pg_merkle_build_host's chunk arrival counter) give up after about
 *     2 s and report through pg_device_faults; nothing else waits on the
 *     device.
 *   - Not thread-safe: calls that share one pg_init() context must be
 *     serialised by the caller.
 */
#ifndef PG12_H
#define PG12_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PG_OK = 0,
    PG_ERR_INVALID_ARG = 1, /* null pointer, zero width, bad sizes            */
    PG_ERR_NOT_POW2 = 2,    /* leaf count is not a power of two               */
    PG_ERR_OOM = 3,         /* workspace or host allocation failed            */
    PG_ERR_CUDA = 4,        /* a CUDA runtime call failed                     */
    PG_ERR_TIMEOUT = 5,     /* a bounded host wait expired                    */
    PG_ERR_PARAMS = 6,      /* parameter set missing, malformed or inconsistent */
    PG_ERR_NOT_INIT = 7     /* pg_init() has not succeeded on this process    */
} pg_status;

/* One tree of a batch (Sec. 4.2 workload, any size/width mix). */
typedef struct {
    const uint64_t *rows; /* dev, n_leaves*width words, row-major            */
    uint64_t n_leaves;    /* power of two >= 1                                */
    uint64_t width;       /* elements per row, >= 1                           */
    uint64_t *nodes;      /* dev, (2*n_leaves-1)*4 words, level-major output  */
} pg_tree;

/* Launch schedule of a batch (pg_merkle_build_batch, pg_batch_graph_create,
 * the server).  Zero fields take the defaults.  Three knobs shape the work:
 *   engine       the persistent kernel: tensor-core groups (128 threads
 *                own 128 states; tasks are units of 128 nodes of one level)
 *                or integer pipes (one thread per state; tasks are 32 nodes
 *                hashed by one warp).
 *   fuse_levels  tensor engine: levels a task builds on its own.  A task is
 *                2^f consecutive leaf units (2^f * 128 leaves); its group
 *                also builds the f levels above them before it meets other
 *                tasks through arrival counters (the second of two sibling
 *                units to finish builds their parent unit).
 *   top_lanes    threads per state of a tree's top levels: 1 = the
 *                persistent kernel climbs every tree to its root; 16 = it
 *                stops below the first level of at most 64 nodes, and a
 *                second launch builds every tree's remaining levels with 16
 *                lanes per node (one block per tree, latency form).
 * plus, for the integer engine, the block size and persistent blocks per
 * SM, and for both the order in which trees hand out their leaf tasks. */
#define PG_BATCH_ENGINE_DEFAULT 0 /* the process's engine (pg_get_engine) */
#define PG_BATCH_ENGINE_INT 1
#define PG_BATCH_ENGINE_TENSOR 2
typedef struct {
    uint32_t block;         /* integer engine: threads per block, 128 or 256 (default 256)  */
    uint32_t blocks_per_sm; /* integer engine: persistent blocks per SM, capped by occupancy */
    uint32_t order;         /* 0 = trees as given, 1 = most work first (default 0)          */
    uint32_t engine;        /* PG_BATCH_ENGINE_*                                           */
    uint32_t fuse_levels;   /* tensor engine: 0..3 (default 0)                             */
    uint32_t top_lanes;     /* 0 or 1 = climb to the roots (default), 16 = hand off         */
    uint32_t reserved[2];   /* must be 0                                                   */
} pg_schedule;

/* Opaque handle of a captured batch (see pg_batch_graph_create). */
typedef struct pg_batch_graph pg_batch_graph;

/* Serving runtime (continuous batching of tree builds); see pg_server_create. */
typedef struct pg_server pg_server;

typedef struct {
    size_t pool_bytes;     /* device memory for node buffers (admission budget); 0 = 4 GiB */
    uint32_t max_batch;    /* requests per launch (0 = 256)                               */
    uint32_t max_inflight; /* batches on the device at once, one stream each (0 = 2, <= 8) */
    pg_schedule sched;     /* launch schedule of every batch (zeros = defaults)          */
} pg_server_config;

/* Request states reported by pg_server_query. */
enum { PG_REQ_QUEUED = 0, PG_REQ_RUNNING = 1, PG_REQ_DONE = 2, PG_REQ_FAILED = 3 };

typedef struct {
    int32_t state;          /* PG_REQ_*                                                  */
    int32_t batch_size;     /* requests in the launch that built it (0 until launched)   */
    double submit_s;        /* host clock (s since pg_server_create) at submission        */
    double launch_s;        /* ... when its batch was launched                           */
    double done_s;          /* ... when the server saw its batch complete                */
    const uint64_t *nodes;  /* dev, (2N-1)*4 words in the server's pool, once admitted   */
} pg_request_info;

/* Element-wise field operations (pg_field_eval / pg_field_bench), the GPU
 * counterparts of Table 1's basic functions. */
enum {
    PG_OP_ADD = 1,       /* a + b                          (Alg. 4, add)            */
    PG_OP_SUB = 2,       /* a - b                          (Alg. 6, sub)            */
    PG_OP_MUL = 3,       /* a * b                          (mult_128)               */
    PG_OP_SQR = 4,       /* a * a                          (square_128)             */
    PG_OP_REDUCE = 5,    /* (b * 2^64 + a) mod p           (Alg. 2, reduce_128_64)  */
    PG_OP_MUL_SMALL = 6, /* a * (b mod 2^8)                (mult_72)                */
    PG_OP_SBOX = 7,      /* a^7                            (Alg. 1 SBox)            */
    PG_OP_DOT12 = 8,     /* 12-term dot product, bench only (spmv/mmult rows)       */
    PG_OP_PIPE_IMAD = 9,       /* bench only: raw mad.lo.u32 throughput (IMAD)      */
    PG_OP_PIPE_IMAD_WIDE = 10, /* bench only: raw mad.wide.u32 throughput           */
    PG_OP_PIPE_IADD = 11,      /* bench only: raw 32-bit add throughput             */
    PG_OP_LAT_MUL = 12,        /* bench only: latency of a dependent chain of a * b */
    PG_OP_LAT_SBOX = 13,       /* bench only: latency of x^7                        */
    PG_OP_LAT_DOT12 = 14,      /* bench only: latency of a 12-term dot product      */
    PG_OP_LAT_PERM = 15,       /* bench only: latency of one permutation, one thread per state */
    PG_OP_LAT_PERM_WIDE = 16   /* bench only: latency of one permutation, 16 lanes per state   */
};

/* Library version, e.g. "pg12 1.0 sm_103a". */
const char *pg_version(void);

/* Text of the most recent error of this process ("" if none). */
const char *pg_last_error(void);

/*
 * pg_init -- select `device`, build the parameter set on the host and upload
 * the optimised-form constants (Alg. 1) to the device.
 *   device       CUDA ordinal.
 *   params_path  name of a built-in parameter set: NULL or "pg12_v1" (Cauchy
 *                MDS, the default) or "pg12_small" (circulant MDS with 8-bit
 *                entries, Table 1's mult_72 / mmult_4x12_8 shape); anything
 *                else returns PG_ERR_PARAMS.
 * Idempotent for the same device (a different set name switches the active
 * set, see pg_params_select).  Synchronous.  Allocates the workspace used by
 * pg_merkle_build / pg_merkle_build_batch.
 */
pg_status pg_init(int device, const char *params_path);

/*
 * pg_params_select -- make a built-in parameter set ("pg12_v1" or NULL,
 * "pg12_small") the active one for every later call of this process.  Works
 * without a GPU (host generation only); after pg_init it also reloads the
 * device constants.  Device work in flight keeps the constants it started
 * with only if the caller synchronises before switching.
 */
pg_status pg_params_select(const char *name);

/* Name of the active parameter set. */
const char *pg_params_name(void);

/*
 * Permutation engines (the computed function is the same; results are
 * bit-identical):
 *   PG_ENGINE_INT     every step on the integer pipes (Alg. 1 with the
 *                     special-prime reduction of Alg. 2, one thread per state);
 *   PG_ENGINE_TENSOR  the same function, with every linear layer of 128
 *                     states at a time as an exact tensor-core contraction of
 *                     byte limbs (fp16 operands, fp32 sums of integers below
 *                     2^24): the eight full rounds' 12x12 MDS products (Alg. 1,
 *                     MDS) and the 22 partial rounds' layers in their unrolled
 *                     form (pg_params_export_chain), the S-boxes and a scalar
 *                     chain on the integer pipes -- used by pg_permute_batch,
 *                     pg_hash_rows, the leaves of pg_merkle_build /
 *                     pg_merkle_build_host and their tree levels of at least
 *                     2^13 nodes.  The default.
 * pg_set_engine applies to launches made after it returns; PG_ERR_INVALID_ARG
 * for any other value.  Host-only.
 */

#define PG_ENGINE_INT 0
#define PG_ENGINE_TENSOR 1
pg_status pg_set_engine(int engine);
int pg_get_engine(void);

/*
 * pg_tc_tables_export -- host copy of the tensor-core digit tables of the
 * active parameter set, for inspection and CPU tests: with out == NULL
 * returns the table size in bytes; else writes it to `out` (host, `bytes`
 * long) and returns it, or returns 0 if `bytes` is too small.  Layout (all
 * little-endian fp16 bit patterns, K-major 8x8 core matrices of 128 bytes;
 * a table of n output rows and k input words holds row 8i+b, column 8j+a =
 * balanced base-256 digit b of 2^(8a) mat[i][j] mod p, core matrix (row
 * group g, column chunk c) at byte (g k + c) * 128, row r at 16 r):
 *   m    [96 x 96]  M of the full rounds
 *   pre  [96 x 96]  the transition matrix of full round 3
 *   b_bias [2 core matrices]  row b, column 0 = 4 u_b (the bias digits)
 *   a_bias [2 core matrices]  2^-13 at column 0 of every row
 *   a_zcap [4 core matrices]  bytes of (c_0[j])^7, j = 8..11, every row
 *   vpa  [80 x 96]  rows 0..9 of the chain's vp (pg_params_export_chain)
 *   vpb  [96 x 96]  rows 10..21 of vp
 *   bs   [96 x 96]  row i: beta[10 + i][r] for inputs r = 0..10; row 11
 *                   and input 11 zero
 *   w1   [96 x 96]  the chain's w, inputs s_0 .. s_10 (input 11 zero)
 *   w2   [96 x 96]  w, inputs s_11 .. s_21 (input 11 zero)
 * Host-only; works without a GPU.
 */
size_t pg_tc_tables_export(void *out, size_t bytes);

/*
 * pg_params_export_chain -- host copy of the unrolled form of the 22 partial
 * rounds (Alg. 1, MDSPartial) that the tensor-core kernels compute.  With
 * x^(0) the state entering partial round 0, y3 the S-box outputs of full
 * round 3 (so x^(0) = pre * y3), c_q cell 0 before partial round q and
 * s_q = (c_q + part_rc[q])^7:
 *   c_0 = x^(0)_0;  c_(q+1) = sum_j vp[q*12 + j] y3_j + sum_(r<=q) beta[q*22 + r] s_r;
 *   after round 21: cell 0 = c_22 = sum_j vp[21*12 + j] y3_j + sum_r w[0*22 + r] s_r,
 *                   cell i = x^(0)_i + sum_r w[i*22 + r] s_r  (i = 1..11).
 *   vp    host, 22*12 words;  beta  host, 22*22 words (r <= q used);
 *   w     host, 12*22 words (row 0 = beta row 21).
 * Any pointer may be NULL.  Host-only; works without a GPU.
 */
pg_status pg_params_export_chain(uint64_t *vp, uint64_t *beta, uint64_t *w);

/*
 * pg_device_faults -- *faults = 1 if a tensor-core kernel launched since the
 * last call gave up waiting for its tensor cores (each such wait is bounded,
 * about two seconds; the kernel then stops and frees its tensor memory, and
 * its outputs are not valid), else 0; the flag is cleared.  Synchronous (it
 * reads a device word).  PG_ERR_NOT_INIT before pg_init.
 */
pg_status pg_device_faults(uint32_t *faults);

/* Release the workspace.  Safe to call when not initialised. */
pg_status pg_shutdown(void);

/*
 * pg_params_export -- host copy of the plain parameter set this library
 * generated (Sec. 2.4: round constants C and MDS matrix M of Alg. 1, before
 * the optimised rewrite):
 *   rc   host, 30*12 words, rc[r*12 + i] = constant of round r, cell i;
 *   mds  host, 12*12 words, row-major, new_i = sum_j mds[i*12+j] * x_j.
 * Either pointer may be NULL.  Host-only; works without a GPU.
 */
pg_status pg_params_export(uint64_t *rc, uint64_t *mds);

/*
 * pg_params_sha256 -- fingerprint of the active plain parameter set: the
 * SHA-256 (FIPS 180-4) of rc[30][12] followed by mds[12][12], each word as
 * 8 little-endian bytes, as 64 lowercase hex digits.  The returned string is
 * owned by the library and stays valid until the process exits.  NULL if the
 * set could not be generated.  Host-only; works without a GPU.
 */
const char *pg_params_sha256(void);

/*
 * pg_workspace_bytes -- device bytes of the library workspace that a batch of
 * these trees needs (tree plans and arrival counters of pg_merkle_build_batch;
 * the batch fails with PG_ERR_OOM above the workspace pg_init allocates).
 * With trees == NULL: the size of that workspace.  0 if a tree's n_leaves is
 * not a power of two.  Host-only.
 */
size_t pg_workspace_bytes(const pg_tree *trees, size_t n_trees);

/*
 * pg_params_export_optimized -- host copy of the optimised-form constants
 * that the kernels use (Alg. 1's C, M, S after the sparse rewrite):
 *   full_rc   8*12 words: constants added before the S-box of full rounds
 *             0..3 and 26..29 (in that order);
 *   mds       12*12 words: dense matrix of full rounds 0,1,2,26..29;
 *   pre       12*12 words: dense matrix of full round 3 (transition matrix);
 *   part_rc   22 words: scalar added to cell 0 before the S-box of partial
 *             round r (r = 0..21);
 *   part_v    22*12 words: first row of the sparse matrix of partial round r
 *             (new_0 = sum_j v[j] x_j);
 *   part_w    22*11 words: first column below the diagonal
 *             (new_i = x_i + w[i-1] x_0 for i >= 1).
 * Any pointer may be NULL.  Host-only; works without a GPU.
 */
pg_status pg_params_export_optimized(uint64_t *full_rc, uint64_t *mds, uint64_t *pre,
                                     uint64_t *part_rc, uint64_t *part_v, uint64_t *part_w);

/*
 * pg_permute_batch -- Alg. 1: one Poseidon-12 permutation of each of `n`
 * independent states, in place.
 *   states  dev, n*12 words, state k at states[12k .. 12k+11]; 8-byte aligned.
 *   n       number of states; 0 is a no-op.
 */
pg_status pg_permute_batch(uint64_t *states, size_t n, void *stream);

/*
 * pg_hash_rows -- Sec. 2.4 sponge over every row of a row-major matrix.
 *   rows     dev, n_rows*width words, row r at rows[r*width ..]; 8-byte aligned.
 *   n_rows   number of rows (0 = no-op).
 *   width    elements per row, >= 1 (0 -> PG_ERR_INVALID_ARG).  Rows use
 *            ceil(width/8) permutations; a short last chunk is zero-filled.
 *   digests  dev, n_rows*4 words, digest r at digests[4r ..].
 */
pg_status pg_hash_rows(const uint64_t *rows, size_t n_rows, size_t width, uint64_t *digests,
                       void *stream);

/*
 * pg_merkle_build -- Sec. 4.2: whole Merkle tree over n_leaves rows.
 *   rows      dev, n_leaves*width words, row-major.
 *   n_leaves  power of two >= 1 (otherwise PG_ERR_NOT_POW2).
 *   width     elements per row, >= 1.
 *   nodes     dev, (2*n_leaves-1)*4 words, level-major: level 0 (the
 *             n_leaves leaf digests), then level 1 (n_leaves/2 nodes), ...,
 *             the root in the last 4 words.  Node k of level l is the hash
 *             of nodes 2k and 2k+1 of level l-1.
 *   root_out  host, 4 words, or NULL.  When non-NULL the call synchronises
 *             `stream` and copies the root there.
 * Launches: the leaf sponges in one launch (the tensor-core kernel, or the
 * integer-pipe kernel under PG_ENGINE_INT; trees of at most 8,192 leaves:
 * the 16-lanes-per-state form), then one launch per level of more than 64
 * nodes and one launch of an 8-block cluster for all levels of at most 64
 * nodes up to the root.  Level launches use programmatic
 * dependent launch: each may be scheduled while the previous one finishes,
 * and reads its input only once that one has completed.
 * Reads and writes nothing but rows and nodes (no library workspace), so
 * builds of different trees on different streams may run concurrently.
 * rows and nodes must not overlap (PG_ERR_INVALID_ARG).
 */
pg_status pg_merkle_build(const uint64_t *rows, size_t n_leaves, size_t width, uint64_t *nodes,
                          uint64_t *root_out, void *stream);

/*
 * pg_merkle_build_host -- pg_merkle_build with the rows in host memory: the
 * same nodes, with the host-to-device copy of the rows overlapped with leaf
 * hashing.  The rows are copied in at most 16 chunks on a library stream
 * (small first, then n/8 rows, halving again toward the end, so that on a
 * host link slower than the hashing little work is left once the last copy
 * lands).  Tensor engine: one leaf launch on `stream` hashes them as they
 * arrive (after each chunk the copy stream writes an arrival counter that
 * the launch waits on, each wait bounded by about 2 s, then the fault shows
 * in pg_device_faults); integer engine: one leaf launch per chunk once its
 * copy has finished.  The streamed form needs the copies to run while the
 * launch does: tools that hold copies back during a kernel (profilers that
 * replay kernels) make its waits run out; PG12_HOST_STREAM=0 in the
 * environment (read by pg_init) selects the per-chunk form.
 *   rows_host  host, n_leaves*width words, row-major; page-locked memory
 *              lets the copies overlap (pageable memory works, serialised).
 *   rows_dev   dev, n_leaves*width words: caller-owned staging buffer the
 *              rows are copied into (holds them on return).
 *   n_leaves, width, nodes, root_out, stream  as for pg_merkle_build.
 * Rows of less than 64 MiB are copied in one piece before the build.
 * The copies start once the work already queued on `stream` has finished.
 * Allocates nothing.  Calls from several host threads at once are not
 * supported (they share the library's copy stream, events and counter).
 */
pg_status pg_merkle_build_host(const uint64_t *rows_host, size_t n_leaves, size_t width, uint64_t *rows_dev,
                               uint64_t *nodes, uint64_t *root_out, void *stream);

/*
 * pg_merkle_build_batch -- Sec. 4.2 trees of mixed sizes and widths built
 * in ONE persistent launch: leaf tasks of all trees come from one counter
 * and each tree's upper levels are built by the group (tensor engine) or
 * warp (integer engine) that completes the second of two sibling tasks, so
 * small trees' top levels overlap with other trees' leaf work; with
 * top_lanes = 16 a second launch builds the levels of at most 64 nodes.
 * Results are identical to pg_merkle_build on each tree alone.
 *   trees    host array of n_trees descriptors (device buffers, caller-owned;
 *            node buffers of different trees must not overlap).
 *   n_trees  >= 1.
 *   sched    NULL = defaults.
 * Uses the pg_init workspace (plans + counters); a batch too large for it
 * returns PG_ERR_OOM (use pg_batch_graph_create, which sizes its own).
 */
pg_status pg_merkle_build_batch(const pg_tree *trees, size_t n_trees, const pg_schedule *sched, void *stream);

/*
 * pg_batch_graph_create -- capture a batch into a CUDA graph: the plans are
 * uploaded once into device memory owned by the handle, and the graph holds
 * the counter reset and the persistent kernel.  Synchronous.  The handle
 * reads the trees' row buffers and writes their node buffers at every
 * launch; they must stay valid until pg_batch_graph_destroy.
 */
pg_status pg_batch_graph_create(const pg_tree *trees, size_t n_trees, const pg_schedule *sched,
                                pg_batch_graph **out);

/* Replay a captured batch on `stream` (asynchronous). */
pg_status pg_batch_graph_launch(pg_batch_graph *graph, void *stream);

/* Release a captured batch (synchronises with its last launch). */
pg_status pg_batch_graph_destroy(pg_batch_graph *graph);

/*
 * pg_batch_autotune -- time each candidate schedule on the real batch with
 * CUDA events and return the fastest in *best (and its time in *best_ms if
 * non-NULL).  Candidates: tensor engine x tree order {given, most work
 * first} x levels fused per task {0, 1, 2} x top-level lanes {1, 16}, and
 * integer engine x order x block {256, 128} x top-level lanes {1, 16}.
 * Runs the batch several times on `stream` (outputs are overwritten with the
 * same values); synchronous.
 */
pg_status pg_batch_autotune(const pg_tree *trees, size_t n_trees, void *stream, pg_schedule *best,
                            float *best_ms);

/*
 * Serving runtime: a host thread admits tree-build requests into node
 * buffers carved from a device memory pool (admission by free HBM: a
 * request waits while its (2N-1)*32-byte node buffer does not fit), and
 * launches every admitted request that is waiting as one batch
 * (pg_merkle_build_batch's kernel) on one of max_inflight streams, so
 * requests that arrive while earlier batches run join the next launch and
 * their work overlaps on the device.  Results equal pg_merkle_build on each
 * tree alone.  Row buffers stay caller-owned and must remain valid until the
 * request is done.  All calls are thread-safe.
 *   pg_server_create   needs pg_init(); allocates the pool and per-stream
 *                      plan/counter buffers.
 *   pg_server_submit   queue a build (rows dev, n_leaves pow2, width >= 1);
 *                      a request larger than the whole pool fails with
 *                      PG_ERR_OOM.  Returns its id.
 *   pg_server_query    state, timestamps and node pointer of a request.
 *   pg_server_release  give a finished request's node buffer back to the pool.
 *   pg_server_drain    wait (bounded by timeout_s, else PG_ERR_TIMEOUT) until
 *                      every submitted request is done or failed.
 *   pg_server_destroy  stop the thread, wait for the device, free everything.
 */
pg_status pg_server_create(const pg_server_config *cfg, pg_server **out);
pg_status pg_server_submit(pg_server *srv, const uint64_t *rows, uint64_t n_leaves, uint64_t width, uint64_t *id_out);
pg_status pg_server_query(pg_server *srv, uint64_t id, pg_request_info *info);
pg_status pg_server_release(pg_server *srv, uint64_t id);
pg_status pg_server_drain(pg_server *srv, double timeout_s);
pg_status pg_server_destroy(pg_server *srv);

/*
 * pg_field_eval -- out[i] = op(a[i], b[i]) mod p, canonical, for the ops
 * PG_OP_ADD .. PG_OP_SBOX (b may be NULL for one-operand ops; it is read as
 * 0).  a, b, out: dev, n words each; any 64-bit input words.  Asynchronous.
 */
pg_status pg_field_eval(int op, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n, void *stream);

/*
 * pg_field_bench -- throughput of one operation on the current device
 * (twelve independent chains per thread, grid = SMs x occupancy): results
 * per second and per SM clock (clock64-timed).  For the PG_OP_LAT_* ops, the
 * latency instead: one warp runs one dependent chain of the operation;
 * ops_per_clk_sm receives the SM cycles per operation and ops_per_s the
 * operations per second of that chain.  Synchronous; allocates and frees two
 * small device buffers.
 */
pg_status pg_field_bench(int op, double *ops_per_s, double *ops_per_clk_sm);

/*
 * pg_merkle_open -- authentication paths of k leaves from a built tree
 * (Sec. 2.4: the root commits to every leaf; a path is the sibling of each
 * ancestor, from the leaf level up).
 *   nodes     dev, level-major node array of a tree of n_leaves leaves.
 *   indices   dev, k leaf indices (uint64, each < n_leaves, else the path is
 *             filled with all-ones words).
 *   paths     dev, k * log2(n_leaves) * 4 words; path q at
 *             paths[q * log2(n_leaves) * 4 ..], level 0 sibling first.
 * Asynchronous; pure gathers (no hashing).
 */
pg_status pg_merkle_open(const uint64_t *nodes, size_t n_leaves, const uint64_t *indices, size_t k,
                         uint64_t *paths, void *stream);

/*
 * pg_merkle_verify -- recompute the root from each (leaf digest, index,
 * path) with the permutation and compare it with `root`.
 *   root       dev, 4 words.
 *   leaves     dev, k * 4 words (leaf digests, level 0 of the tree).
 *   indices    dev, k leaf indices.
 *   paths      dev, as written by pg_merkle_open.
 *   ok         dev, k bytes: 1 if the path reproduces the root, else 0.
 * Needs pg_init().  Asynchronous.
 */
pg_status pg_merkle_verify(const uint64_t *root, size_t n_leaves, const uint64_t *leaves, const uint64_t *indices,
                           size_t k, const uint64_t *paths, uint8_t *ok, void *stream);

/*
 * pg_merkle_build_noalloc -- the same tree as pg_merkle_build (identical
 * output), for callers that cannot allocate device memory: code whose
 * allocator forbids cudaMalloc, or a host process that may only use the
 * buffers it was handed.  The paper has no counterpart; it is a property of
 * this library's interface, not of the method.
 *   rows, n_leaves, width, nodes  as for pg_merkle_build (caller-owned);
 *                                 n_leaves must be at most 2^22, otherwise
 *                                 PG_ERR_INVALID_ARG with a message naming
 *                                 the limit.
 *   stream                        cudaStream_t as void* (NULL = default).
 * Allocates nothing and does not need pg_init().  Its scratch (the arrival
 * counters of the build, 512 KiB) is a file-scope __device__ array that every
 * GPU loading the library holds until process exit, one copy per device.
 * The first call on a device, and the first call on it after the active
 * parameter set changed (pg_params_select, pg_init with another set),
 * performs that device's set-up (a synchronous upload of the constant
 * tables, and the lookup of the array's device address) with the device
 * current; make those calls before any stream capture.  All calls on one
 * device share that device's array, which keeps the previous call's contents
 * (each call clears what it uses): calls that overlap on the same GPU race
 * and must be serialised by the caller.  rows and nodes must not overlap
 * (PG_ERR_INVALID_ARG).
 * Asynchronous on `stream`; no root is returned (read it from nodes).
 */
pg_status pg_merkle_build_noalloc(const uint64_t *rows, size_t n_leaves, size_t width, uint64_t *nodes,
                                  void *stream);

/*
 * Goldilocks NTT and low-degree extension (Sec. 2.3 names the NTT as
 * zkProver's Goldilocks hotspot after Merkle building; Sec. 2.4 commits to
 * polynomial evaluations).  The paper gives no definition; these are the
 * textbook ones: 7 generates the multiplicative group of Eq. 1's field, the
 * primitive 2^k-th root of unity is w_k = 7^((p - 1) / 2^k).
 * Data is row-major with `ncols` columns: element (row r, column c) at
 * r * ncols + c; every column is transformed on its own.  Inputs may hold
 * any 64-bit words (read mod p); outputs are canonical.
 *
 * pg_ntt -- in place: X_i = sum_j x_j w^(i j) with w = w_k, n = 2^k rows;
 * with inverse != 0, x_j = n^-1 sum_i X_i w^(-i j).  Natural row order in
 * and out.
 *   data   dev, n * ncols words, caller-owned, 8-byte aligned.
 *   n      power of two, at most 2^30 (PG_ERR_NOT_POW2 / PG_ERR_INVALID_ARG).
 * Needs pg_init().  Asynchronous on `stream`.
 */
pg_status pg_ntt(uint64_t *data, size_t n, size_t ncols, int inverse, void *stream);

/*
 * pg_lde -- low-degree extension with blowup 2^log_blowup on the coset
 * shifted by 7: column c of `evals` holds P_c(w_k^j), j < n = 2^k, for the
 * unique P_c of degree < n; row i of `out` receives P_c(7 * w_{k+b}^i),
 * i < N = n * 2^b.  The rows of `out` are the leaves a Merkle commitment
 * hashes (pg_merkle_build with width = ncols).
 *   evals    dev, n * ncols words (read only unless it is also `scratch`).
 *   out      dev, N * ncols words; must not overlap evals or scratch.
 *   scratch  dev, n * ncols words of working space; may be `evals` itself
 *            (then evals is overwritten).  On return it holds c_j 7^j (the
 *            coefficients of P_c(7 x)) in bit-reversed row order.
 *   log_blowup  0..16; N at most 2^30 rows.
 * Needs pg_init().  Asynchronous on `stream`; PG_ERR_INVALID_ARG on bad
 * sizes or overlapping buffers, PG_ERR_NOT_POW2 if n is not a power of two.
 */
pg_status pg_lde(const uint64_t *evals, size_t n, size_t ncols, uint32_t log_blowup, uint64_t *out,
                 uint64_t *scratch, void *stream);

/*
 * Launch timing (the cudaEvent side of the paper's hardware-counter
 * measurements, Sec. 4.1-4.2): when enabled, every kernel launch the library
 * makes (and every pg_batch_graph_launch) is bracketed by a pair of CUDA
 * events recorded on the launching stream.  Launches made while a stream is
 * being captured are not recorded.  At most 65,536 launches are held;
 * further ones are counted as dropped.
 *
 * pg_profile_enable -- on != 0 starts recording, 0 stops it; either way the
 * records held so far are discarded.  Host-synchronous with those records'
 * events.  Never fails.
 */
typedef struct pg_kernel_time {
    char name[32];     /* kernel name: "k_merkle", "k_merkle_top", ..., "batch_graph" */
    uint64_t launches; /* launches recorded */
    uint64_t perms;    /* permutations those launches performed */
    double total_ms;   /* sum of their event-timed durations */
} pg_kernel_time;

pg_status pg_profile_enable(int on);

/*
 * pg_profile_read -- waits for the recorded launches to finish, sums them
 * per kernel into out[0 .. *n_out) (kernels with no launch are left out) and
 * clears the records (recording stays as it was).
 *   out      host array of cap entries, or NULL to only count.
 *   n_out    host, receives the number of kernels with launches.
 *   dropped  host or NULL, receives the launches not recorded since the
 *            last enable/read because the record store was full.
 * PG_ERR_INVALID_ARG if out is non-NULL and cap < *n_out (the first cap
 * entries are still written); PG_ERR_CUDA if an event could not be read.
 */
pg_status pg_profile_read(pg_kernel_time *out, size_t cap, size_t *n_out, uint64_t *dropped);

#ifdef __cplusplus
}
#endif

#endif /* PG12_H */
