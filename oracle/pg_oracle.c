/*
 * pg_oracle.c -- plain, slow, obviously-correct CPU reference for the
 * Poseidon-12 / Goldilocks Merkle-tree path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; it exists so that tests, the smoke check and the timed
 * CPU baseline have an independent answer to compare against.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * What it follows (arXiv 2506.09505):
 *   - the field: Eq. 1, p = 2^64 - 2^32 + 1, canonical elements 0 <= e < p
 *     (Sec. 2.4).  All arithmetic is done on unsigned __int128 followed by
 *     "% p": the plain definition, none of Alg. 2/4/6's tricks.
 *   - the permutation: Sec. 2.4 ("Poseidon Hash") and Alg. 1: width 12,
 *     S-box x^7, HALF_FULL_ROUNDS = 4 (so 8 full rounds) and
 *     PARTIAL_ROUNDS = 22.  The oracle uses the plain round form of the
 *     Poseidon paper that Sec. 2.4 cites: every round adds its 12 round
 *     constants, applies the S-box (all 12 cells in a full round, cell 0 in a
 *     partial round), then multiplies by the 12x12 MDS matrix M, column
 *     convention new_i = sum_j M[i][j] * x_j.  Alg. 1 is the sparse
 *     "optimised" rewrite of exactly this map; the oracle does not use it.
 *   - the sponge: Sec. 2.4 -- the state absorbs the input in chunks of eight
 *     elements, permuting once per chunk; rate 8, capacity 4, digest = the
 *     first four state elements.  Overwrite mode: a chunk replaces state[0..7]
 *     and state[8..11] is carried; a short last chunk is zero-filled.
 *   - the Merkle tree: Sec. 2.4 ("Merkle Tree") and Sec. 4.2: leaves are the
 *     hashes of the data rows; each parent is the hash of the concatenation of
 *     its two children (8 elements, one permutation); level by level to the
 *     root.  Nodes are returned level-major: level 0 (N leaf digests), then
 *     level 1, ..., the root last.
 *   - the parameters: the paper prints no constants (Alg. 1 only names
 *     C, M, S).  They are generated with the Poseidon paper's procedure: a
 *     Grain LFSR seeded with (prime field, x^alpha S-box, n = 64, t = 12,
 *     R_F = 8, R_P = 22), 160 warm-up clocks, bit pairs filtered so that the
 *     second bit is kept only when the first is 1, 64-bit big-endian words
 *     rejected when >= p; first the 30 x 12 round constants, then 2t field
 *     elements x_0..x_11, y_0..y_11 for a Cauchy matrix M[i][j] = 1/(x_i+y_j)
 *     (all 24 distinct, no x_i + y_j = 0; otherwise the 24 are drawn again).
 *     This is the project's parameter set "pg12_v1".
 *     parity unpinned: identity of these constants with any external
 *     implementation's constants (none is available to compare with).
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#include <pthread.h>

typedef unsigned __int128 u128;

#define ORC_P 0xFFFFFFFF00000001ULL /* Eq. 1 */
#define ORC_T 12
#define ORC_RF 8
#define ORC_RP 22
#define ORC_ROUNDS (ORC_RF + ORC_RP)

/* ------------------------------------------------------------------ field */

uint64_t orc_canon(uint64_t x) { return x % ORC_P; }
uint64_t orc_add(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a + b) % ORC_P); }
uint64_t orc_sub(uint64_t a, uint64_t b) {
    return (uint64_t)(((u128)(a % ORC_P) + ORC_P - (b % ORC_P)) % ORC_P);
}
uint64_t orc_mul(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * b) % ORC_P); }

uint64_t orc_pow(uint64_t a, uint64_t e) {
    uint64_t r = 1 % ORC_P, b = a % ORC_P;
    while (e) {
        if (e & 1) r = orc_mul(r, b);
        b = orc_mul(b, b);
        e >>= 1;
    }
    return r;
}

/* Fermat inverse, a^(p-2); 0 maps to 0. */
uint64_t orc_inv(uint64_t a) { return orc_pow(a, ORC_P - 2); }

/* S-box of Alg. 1: x^7. */
static uint64_t orc_sbox(uint64_t x) { return orc_pow(x, 7); }

/* Element-wise field operation over n pairs (Eq. 1), canonical results:
 * op 1 a+b, 2 a-b, 3 a*b, 4 a^2, 5 a^7.  b is ignored for ops 4 and 5.
 * Returns 0, or -1 for an unknown op. */
int orc_field_many(int op, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t n) {
    size_t i;
    switch (op) {
    case 1: for (i = 0; i < n; ++i) out[i] = orc_add(a[i], b[i]); return 0;
    case 2: for (i = 0; i < n; ++i) out[i] = orc_sub(a[i], b[i]); return 0;
    case 3: for (i = 0; i < n; ++i) out[i] = orc_mul(a[i], b[i]); return 0;
    case 4: for (i = 0; i < n; ++i) out[i] = orc_mul(a[i], a[i]); return 0;
    case 5: for (i = 0; i < n; ++i) out[i] = orc_sbox(a[i]); return 0;
    default: return -1;
    }
}

/* d with 7*d = 1 mod (p-1), so (x^7)^d = x: extended Euclid on (7, p-1). */
uint64_t orc_sbox_inverse_exponent(void) {
    __int128 r0 = (__int128)(ORC_P - 1), r1 = 7, s0 = 0, s1 = 1;
    while (r1 != 0) {
        __int128 q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    /* r0 == gcd == 1, s0 * 7 == 1 mod (p-1) */
    __int128 m = (__int128)(ORC_P - 1);
    s0 %= m;
    if (s0 < 0) s0 += m;
    return (uint64_t)s0;
}

/* ------------------------------------------------------- matrix helpers */

/* y = M x, column convention y_i = sum_j M[i][j] x_j. */
static void orc_matvec(const uint64_t *m, const uint64_t *x, uint64_t *y) {
    for (int i = 0; i < ORC_T; i++) {
        uint64_t acc = 0;
        for (int j = 0; j < ORC_T; j++) acc = orc_add(acc, orc_mul(m[i * ORC_T + j], x[j]));
        y[i] = acc;
    }
}

/* Inverse of an n x n matrix over F_p by Gauss-Jordan elimination.
 * Returns 0 on success, -1 if singular. */
int orc_mat_inverse(const uint64_t *a_in, uint64_t *inv, int n) {
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n * n);
    if (!a) return -2;
    memcpy(a, a_in, sizeof(uint64_t) * (size_t)n * n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) inv[i * n + j] = (i == j);
    for (int c = 0; c < n; c++) {
        int piv = -1;
        for (int r = c; r < n; r++)
            if (a[r * n + c] % ORC_P) { piv = r; break; }
        if (piv < 0) { free(a); return -1; }
        if (piv != c)
            for (int j = 0; j < n; j++) {
                uint64_t t = a[c * n + j]; a[c * n + j] = a[piv * n + j]; a[piv * n + j] = t;
                t = inv[c * n + j]; inv[c * n + j] = inv[piv * n + j]; inv[piv * n + j] = t;
            }
        uint64_t s = orc_inv(a[c * n + c]);
        for (int j = 0; j < n; j++) {
            a[c * n + j] = orc_mul(a[c * n + j], s);
            inv[c * n + j] = orc_mul(inv[c * n + j], s);
        }
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            uint64_t f = a[r * n + c];
            if (!f) continue;
            for (int j = 0; j < n; j++) {
                a[r * n + j] = orc_sub(a[r * n + j], orc_mul(f, a[c * n + j]));
                inv[r * n + j] = orc_sub(inv[r * n + j], orc_mul(f, inv[c * n + j]));
            }
        }
    }
    free(a);
    return 0;
}

/* Determinant of an n x n matrix over F_p (Gaussian elimination). */
uint64_t orc_mat_det(const uint64_t *a_in, int n) {
    uint64_t *a = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n * n);
    if (!a) return 0;
    memcpy(a, a_in, sizeof(uint64_t) * (size_t)n * n);
    uint64_t det = 1;
    for (int c = 0; c < n; c++) {
        int piv = -1;
        for (int r = c; r < n; r++)
            if (a[r * n + c] % ORC_P) { piv = r; break; }
        if (piv < 0) { free(a); return 0; }
        if (piv != c) {
            for (int j = 0; j < n; j++) {
                uint64_t t = a[c * n + j]; a[c * n + j] = a[piv * n + j]; a[piv * n + j] = t;
            }
            det = orc_sub(0, det);
        }
        det = orc_mul(det, a[c * n + c]);
        uint64_t s = orc_inv(a[c * n + c]);
        for (int r = c + 1; r < n; r++) {
            uint64_t f = orc_mul(a[r * n + c], s);
            if (!f) continue;
            for (int j = c; j < n; j++) a[r * n + j] = orc_sub(a[r * n + j], orc_mul(f, a[c * n + j]));
        }
    }
    free(a);
    return det;
}

/* ------------------------------------------------ Grain LFSR parameters */

typedef struct { uint8_t b[80]; } orc_grain;

/* One LFSR clock: b_{i+80} = b_{i+62} ^ b_{i+51} ^ b_{i+38} ^ b_{i+23} ^ b_{i+13} ^ b_i. */
static int orc_grain_clock(orc_grain *g) {
    int nb = g->b[62] ^ g->b[51] ^ g->b[38] ^ g->b[23] ^ g->b[13] ^ g->b[0];
    memmove(g->b, g->b + 1, 79);
    g->b[79] = (uint8_t)nb;
    return nb;
}

static void orc_grain_put(orc_grain *g, int *pos, uint64_t v, int nbits) {
    for (int k = nbits - 1; k >= 0; k--) g->b[(*pos)++] = (uint8_t)((v >> k) & 1);
}

static void orc_grain_init(orc_grain *g, int field, int sbox, int n, int t, int rf, int rp) {
    int pos = 0;
    orc_grain_put(g, &pos, (uint64_t)field, 2);
    orc_grain_put(g, &pos, (uint64_t)sbox, 4);
    orc_grain_put(g, &pos, (uint64_t)n, 12);
    orc_grain_put(g, &pos, (uint64_t)t, 12);
    orc_grain_put(g, &pos, (uint64_t)rf, 10);
    orc_grain_put(g, &pos, (uint64_t)rp, 10);
    orc_grain_put(g, &pos, (1ULL << 30) - 1, 30);
    for (int i = 0; i < 160; i++) orc_grain_clock(g);
}

/* Output bit: clock pairs; keep the second bit only if the first is 1. */
static int orc_grain_bit(orc_grain *g) {
    for (;;) {
        int keep = orc_grain_clock(g);
        int bit = orc_grain_clock(g);
        if (keep) return bit;
    }
}

/* n-bit big-endian word (n <= 64). */
static uint64_t orc_grain_word(orc_grain *g, int n) {
    uint64_t v = 0;
    for (int i = 0; i < n; i++) v = (v << 1) | (uint64_t)orc_grain_bit(g);
    return v;
}

/* Field element by rejection: draw 64 bits until the word is < p. */
static uint64_t orc_grain_field(orc_grain *g) {
    for (;;) {
        uint64_t v = orc_grain_word(g, 64);
        if (v < ORC_P) return v;
    }
}

/* Raw Grain output words for tests of the generator itself. */
void orc_grain_words(int field, int sbox, int n, int t, int rf, int rp, int nbits,
                     uint64_t *out, size_t count) {
    orc_grain g;
    orc_grain_init(&g, field, sbox, n, t, rf, rp);
    for (size_t i = 0; i < count; i++) out[i] = orc_grain_word(&g, nbits);
}

/* Generate parameter set pg12_v1: rc[30*12] (round r, cell i at rc[r*12+i])
 * and mds[12*12] (row-major, column convention).  Also returns the Cauchy
 * points xs[12], ys[12] if non-NULL.  Returns the number of Cauchy redraws. */
int orc_params_generate(uint64_t *rc, uint64_t *mds, uint64_t *xs_out, uint64_t *ys_out) {
    orc_grain g;
    orc_grain_init(&g, 1, 0, 64, ORC_T, ORC_RF, ORC_RP);
    for (int k = 0; k < ORC_ROUNDS * ORC_T; k++) rc[k] = orc_grain_field(&g);
    int redraws = 0;
    for (;;) {
        uint64_t v[2 * ORC_T];
        for (int k = 0; k < 2 * ORC_T; k++) v[k] = orc_grain_field(&g);
        int ok = 1;
        for (int a = 0; a < 2 * ORC_T && ok; a++)
            for (int b = a + 1; b < 2 * ORC_T; b++)
                if (v[a] == v[b]) { ok = 0; break; }
        for (int i = 0; i < ORC_T && ok; i++)
            for (int j = 0; j < ORC_T; j++)
                if (orc_add(v[i], v[ORC_T + j]) == 0) { ok = 0; break; }
        if (!ok) { redraws++; continue; }
        for (int i = 0; i < ORC_T; i++)
            for (int j = 0; j < ORC_T; j++) mds[i * ORC_T + j] = orc_inv(orc_add(v[i], v[ORC_T + j]));
        if (xs_out) memcpy(xs_out, v, sizeof(uint64_t) * ORC_T);
        if (ys_out) memcpy(ys_out, v + ORC_T, sizeof(uint64_t) * ORC_T);
        return redraws;
    }
}

/* ------------------------------------------------------------ permutation */

/* Round r (0-based) is full for r < 4 and r >= 26, partial otherwise. */
static int orc_is_full(int r) { return r < ORC_RF / 2 || r >= ORC_RF / 2 + ORC_RP; }

/* Plain round form: per round, add constants, S-box, multiply by M. */
void orc_permute(const uint64_t *rc, const uint64_t *mds, uint64_t *st) {
    uint64_t x[ORC_T], y[ORC_T];
    for (int i = 0; i < ORC_T; i++) x[i] = st[i] % ORC_P;
    for (int r = 0; r < ORC_ROUNDS; r++) {
        for (int i = 0; i < ORC_T; i++) x[i] = orc_add(x[i], rc[r * ORC_T + i]);
        if (orc_is_full(r)) {
            for (int i = 0; i < ORC_T; i++) x[i] = orc_sbox(x[i]);
        } else {
            x[0] = orc_sbox(x[0]);
        }
        orc_matvec(mds, x, y);
        memcpy(x, y, sizeof x);
    }
    memcpy(st, x, sizeof x);
}

/* Inverse of orc_permute: rounds in reverse, M^-1, x^d, subtract constants.
 * mds_inv must be the inverse of the MDS matrix (orc_mat_inverse). */
void orc_permute_inverse(const uint64_t *rc, const uint64_t *mds_inv, uint64_t *st) {
    uint64_t x[ORC_T], y[ORC_T];
    uint64_t d = orc_sbox_inverse_exponent();
    for (int i = 0; i < ORC_T; i++) x[i] = st[i] % ORC_P;
    for (int r = ORC_ROUNDS - 1; r >= 0; r--) {
        orc_matvec(mds_inv, x, y);
        memcpy(x, y, sizeof x);
        if (orc_is_full(r)) {
            for (int i = 0; i < ORC_T; i++) x[i] = orc_pow(x[i], d);
        } else {
            x[0] = orc_pow(x[0], d);
        }
        for (int i = 0; i < ORC_T; i++) x[i] = orc_sub(x[i], rc[r * ORC_T + i]);
    }
    memcpy(st, x, sizeof x);
}

/* Permute n independent states in place (state k at st[12k..12k+11]). */
void orc_permute_many(const uint64_t *rc, const uint64_t *mds, uint64_t *st, size_t n) {
    for (size_t k = 0; k < n; k++) orc_permute(rc, mds, st + ORC_T * k);
}

typedef struct {
    const uint64_t *rc, *mds;
    uint64_t *st;
    size_t lo, hi;
} orc_perm_job;

static void *orc_perm_worker(void *arg) {
    orc_perm_job *j = (orc_perm_job *)arg;
    for (size_t k = j->lo; k < j->hi; k++) orc_permute(j->rc, j->mds, j->st + ORC_T * k);
    return NULL;
}

/* The same over nthreads threads, each taking a contiguous range of states
 * (the timed all-core CPU baseline; the result equals orc_permute_many). */
void orc_permute_many_mt(const uint64_t *rc, const uint64_t *mds, uint64_t *st, size_t n, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((size_t)nthreads > n) nthreads = (int)(n ? n : 1);
    pthread_t th[256];
    orc_perm_job jobs[256];
    for (int t = 0; t < nthreads; t++) {
        jobs[t].rc = rc;
        jobs[t].mds = mds;
        jobs[t].st = st;
        jobs[t].lo = n * (size_t)t / (size_t)nthreads;
        jobs[t].hi = n * (size_t)(t + 1) / (size_t)nthreads;
    }
    if (nthreads == 1) {
        orc_perm_worker(&jobs[0]);
        return;
    }
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, orc_perm_worker, &jobs[t]);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
}

/* ----------------------------------------------------------------- sponge */

/* Overwrite-mode sponge, rate 8 / capacity 4, digest = state[0..3].
 * Every element is reduced mod p on input.  A row of width w uses
 * ceil(w/8) permutations (at least one: the empty row hashes one zero
 * chunk). */
void orc_hash_row(const uint64_t *rc, const uint64_t *mds, const uint64_t *row, size_t w,
                  uint64_t *digest) {
    uint64_t st[ORC_T] = {0};
    size_t chunks = w == 0 ? 1 : (w + 7) / 8;
    for (size_t c = 0; c < chunks; c++) {
        for (int i = 0; i < 8; i++) {
            size_t k = c * 8 + (size_t)i;
            st[i] = k < w ? row[k] % ORC_P : 0;
        }
        orc_permute(rc, mds, st);
    }
    memcpy(digest, st, 4 * sizeof(uint64_t));
}

/* Two-to-one compression: perm([L(4), R(4), 0,0,0,0])[0..3]. */
void orc_hash_pair(const uint64_t *rc, const uint64_t *mds, const uint64_t *left,
                   const uint64_t *right, uint64_t *out) {
    uint64_t st[ORC_T] = {0};
    for (int i = 0; i < 4; i++) { st[i] = left[i] % ORC_P; st[4 + i] = right[i] % ORC_P; }
    orc_permute(rc, mds, st);
    memcpy(out, st, 4 * sizeof(uint64_t));
}

/* ------------------------------------------------------------ Merkle tree */

typedef struct {
    const uint64_t *rc, *mds, *rows, *below;
    uint64_t *out;
    size_t w, lo, hi;
    int leaves;
} orc_job;

static void *orc_worker(void *arg) {
    orc_job *j = (orc_job *)arg;
    for (size_t i = j->lo; i < j->hi; i++) {
        if (j->leaves)
            orc_hash_row(j->rc, j->mds, j->rows + i * j->w, j->w, j->out + 4 * i);
        else
            orc_hash_pair(j->rc, j->mds, j->below + 8 * i, j->below + 8 * i + 4, j->out + 4 * i);
    }
    return NULL;
}

static void orc_level(orc_job base, size_t count, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if ((size_t)nthreads > count) nthreads = (int)(count ? count : 1);
    pthread_t th[256];
    orc_job jobs[256];
    if (nthreads > 256) nthreads = 256;
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = base;
        jobs[t].lo = count * (size_t)t / (size_t)nthreads;
        jobs[t].hi = count * (size_t)(t + 1) / (size_t)nthreads;
    }
    if (nthreads == 1) { orc_worker(&jobs[0]); return; }
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
}

/* Build the whole tree over n_leaves rows (n_leaves a power of two, >= 1),
 * row-major rows[n_leaves][w].  nodes receives (2*n_leaves - 1) * 4 words,
 * level-major, root last.  Each level is split over nthreads threads, with a
 * join between levels (the scheme of Sec. 4.2).  Returns 0, or -1 when
 * n_leaves is not a power of two. */
int orc_merkle_build(const uint64_t *rc, const uint64_t *mds, const uint64_t *rows,
                     size_t n_leaves, size_t w, uint64_t *nodes, int nthreads) {
    if (n_leaves == 0 || (n_leaves & (n_leaves - 1))) return -1;
    orc_job base = {rc, mds, rows, NULL, nodes, w, 0, 0, 1};
    orc_level(base, n_leaves, nthreads);
    size_t below = 0, cnt = n_leaves;
    while (cnt > 1) {
        size_t here = below + cnt;
        orc_job j = {rc, mds, NULL, nodes + 4 * below, nodes + 4 * here, w, 0, 0, 0};
        orc_level(j, cnt / 2, nthreads);
        below = here;
        cnt /= 2;
    }
    return 0;
}

/* Authentication path of leaf `index`: the sibling digest at every level
 * from the leaves up (log2(n_leaves) entries of 4 words). */
int orc_auth_path(const uint64_t *nodes, size_t n_leaves, size_t index, uint64_t *path) {
    if (n_leaves == 0 || (n_leaves & (n_leaves - 1)) || index >= n_leaves) return -1;
    size_t base = 0, cnt = n_leaves, k = 0;
    while (cnt > 1) {
        size_t sib = index ^ 1;
        memcpy(path + 4 * k, nodes + 4 * (base + sib), 4 * sizeof(uint64_t));
        base += cnt;
        cnt /= 2;
        index /= 2;
        k++;
    }
    return 0;
}

/* Root recomputed from a leaf digest and its authentication path. */
void orc_root_from_path(const uint64_t *rc, const uint64_t *mds, const uint64_t *leaf_digest,
                        size_t index, const uint64_t *path, size_t depth, uint64_t *root) {
    uint64_t cur[4], nxt[4];
    memcpy(cur, leaf_digest, sizeof cur);
    for (size_t k = 0; k < depth; k++) {
        if (index & 1) orc_hash_pair(rc, mds, path + 4 * k, cur, nxt);
        else orc_hash_pair(rc, mds, cur, path + 4 * k, nxt);
        memcpy(cur, nxt, sizeof cur);
        index >>= 1;
    }
    memcpy(root, cur, sizeof cur);
}

/* --------------------------------------------------------- MDS property */

/* Determinant of a k x k matrix (k <= 12) held in a[12*12], row stride 12. */
static uint64_t orc_small_det(uint64_t a[12 * 12], int k) {
    uint64_t det = 1;
    for (int c = 0; c < k; c++) {
        int piv = -1;
        for (int r = c; r < k; r++)
            if (a[r * 12 + c]) { piv = r; break; }
        if (piv < 0) return 0;
        if (piv != c) {
            for (int j = 0; j < k; j++) {
                uint64_t t = a[c * 12 + j]; a[c * 12 + j] = a[piv * 12 + j]; a[piv * 12 + j] = t;
            }
            det = orc_sub(0, det);
        }
        det = orc_mul(det, a[c * 12 + c]);
        uint64_t s = orc_inv(a[c * 12 + c]);
        for (int r = c + 1; r < k; r++) {
            uint64_t f = orc_mul(a[r * 12 + c], s);
            if (!f) continue;
            for (int j = c; j < k; j++) a[r * 12 + j] = orc_sub(a[r * 12 + j], orc_mul(f, a[c * 12 + j]));
        }
    }
    return det;
}

/* Brute force over every square submatrix of the 12x12 matrix m
 * (C(24,12) - 1 = 2,704,155 of them).  Returns how many are singular; a
 * matrix is MDS exactly when this is 0.  *checked receives the number of
 * minors examined. */
long orc_count_singular_minors(const uint64_t *m, long *checked) {
    long bad = 0, total = 0;
    uint64_t a[12 * 12];
    for (int rs = 1; rs < (1 << 12); rs++) {
        int k = __builtin_popcount((unsigned)rs);
        int rows[12], nr = 0;
        for (int i = 0; i < 12; i++)
            if (rs >> i & 1) rows[nr++] = i;
        for (int cs = 1; cs < (1 << 12); cs++) {
            if (__builtin_popcount((unsigned)cs) != k) continue;
            int cols[12], nc = 0;
            for (int j = 0; j < 12; j++)
                if (cs >> j & 1) cols[nc++] = j;
            for (int i = 0; i < k; i++)
                for (int j = 0; j < k; j++) a[i * 12 + j] = m[rows[i] * 12 + cols[j]];
            total++;
            if (orc_small_det(a, k) == 0) bad++;
        }
    }
    if (checked) *checked = total;
    return bad;
}

/* ------------------------------------------- small-entry parameter set */

/* Same as orc_count_singular_minors but stops at the first singular minor,
 * visiting minors by increasing size.  Returns 1 if every minor is
 * nonsingular (the matrix is MDS), else 0. */
int orc_is_mds(const uint64_t *m) {
    uint64_t a[12 * 12];
    for (int k = 1; k <= 12; k++) {
        for (int rs = 1; rs < (1 << 12); rs++) {
            if (__builtin_popcount((unsigned)rs) != k) continue;
            int rows[12], nr = 0;
            for (int i = 0; i < 12; i++)
                if (rs >> i & 1) rows[nr++] = i;
            for (int cs = 1; cs < (1 << 12); cs++) {
                if (__builtin_popcount((unsigned)cs) != k) continue;
                int cols[12], nc = 0;
                for (int j = 0; j < 12; j++)
                    if (cs >> j & 1) cols[nc++] = j;
                for (int i = 0; i < k; i++)
                    for (int j = 0; j < k; j++) a[i * 12 + j] = m[rows[i] * 12 + cols[j]];
                if (orc_small_det(a, k) == 0) return 0;
            }
        }
    }
    return 1;
}

/* Parameter set pg12_small: the round constants of pg12_v1 (the first 360
 * field elements of the same Grain stream), and a circulant MDS matrix with
 * 8-bit entries -- the matrix shape whose products Table 1's mult_72 and
 * mmult_4x12_8 serve.  After the round constants the stream yields
 * candidates of twelve 64-bit words each; entry c_i = 1 + (word mod 255)
 * (so 1..255) and M[i][j] = c[(j - i) mod 12].  The first candidate whose
 * matrix is MDS is taken.  Writes rc[360], mds[144], row[12]; returns the
 * index of the accepted candidate. */
int orc_params_generate_small(uint64_t *rc, uint64_t *mds, uint64_t *row) {
    orc_grain g;
    orc_grain_init(&g, 1, 0, 64, ORC_T, ORC_RF, ORC_RP);
    for (int k = 0; k < ORC_ROUNDS * ORC_T; k++) rc[k] = orc_grain_field(&g);
    for (int cand = 0;; cand++) {
        uint64_t c[12];
        for (int i = 0; i < 12; i++) c[i] = 1 + orc_grain_word(&g, 64) % 255;
        for (int i = 0; i < 12; i++)
            for (int j = 0; j < 12; j++) mds[i * 12 + j] = c[((j - i) % 12 + 12) % 12];
        if (orc_is_mds(mds)) {
            memcpy(row, c, sizeof c);
            return cand;
        }
    }
}
