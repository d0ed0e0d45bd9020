// Internal declarations shared by the host and device translation units of
// the library (not part of the public ABI in include/pg12.h).
#pragma once

#include <cstddef>
#include <cstdint>

namespace pg12 {

constexpr uint64_t kP = 0xFFFFFFFF00000001ull;  // Eq. 1
constexpr uint64_t kEps = 0xFFFFFFFFull;        // 2^64 mod p = 2^32 - 1
constexpr int kT = 12;                          // state width (Sec. 2.4)
constexpr int kRF = 8;                          // full rounds, 2 x HALF_FULL_ROUNDS
constexpr int kRP = 22;                         // PARTIAL_ROUNDS (Alg. 1)
constexpr int kRounds = kRF + kRP;
constexpr int kRate = 8;                        // sponge chunk (Sec. 2.4)
constexpr int kDigest = 4;

// Plain-form parameter set: x <- M * S(x + rc[r]) for r = 0..29.
struct PlainParams {
    uint64_t rc[kRounds][kT];
    uint64_t mds[kT][kT];
};

// Optimised form (Alg. 1 with MDSPartial), as the device consumes it.
struct OptParams {
    uint64_t full_rc[kRF][kT];    // rounds 0..3 then 26..29
    uint64_t mds[kT][kT];         // dense matrix of full rounds 0..2, 26..29
    uint64_t pre[kT][kT];         // dense transition matrix of full round 3
    uint64_t part_rc[kRP];        // scalar into cell 0, per partial round
    uint64_t part_v[kRP][kT];     // new_0 = sum_j v[j] x_j
    uint64_t part_w[kRP][kT - 1]; // new_i = x_i + w[i-1] x_0
};

// The partial rounds (Alg. 1, MDSPartial) unrolled.  With x^(0) the state
// entering partial round 0, c_q its cell 0 before round q and
// s_q = S(c_q + k_q), round q adds w_q[i] s_q to cell i >= 1 and sets cell 0
// to <v_q, x>, so
//   x_i^(q) = x_i^(0) + sum_(r<q) w_r[i] s_r                       (i >= 1)
//   c_(q+1) = U_q + sum_(r<=q) beta[q][r] s_r,  U_q = sum_(i>=1) v_q[i] x_i^(0),
//   beta[q][r] = sum_(i>=1) v_q[i] w_r[i] (r < q),  beta[q][q] = v_q[0],
// and after round 21 cell 0 is c_22 and cell i >= 1 is
// x_i^(0) + sum_r w_r[i] s_r.  Since x^(0) = P y3 (y3 the S-box outputs of
// full round 3, P its transition matrix), U = (V' P) y3 with V'[q][i] = v_q[i]
// for i >= 1 and 0 for i = 0.  Only the chain c_q -> s_q -> c_(q+1) is
// sequential; U and the final updates are two contractions per state.
struct ChainParams {
    uint64_t vp[kRP][kT];    // U_q = sum_j vp[q][j] y3_j
    uint64_t beta[kRP][kRP]; // beta[q][r], r <= q
    uint64_t w[kT][kRP];     // row 0: beta[21][r]; row i >= 1: w_r[i]
};

// Tensor-core form of the dense contractions.  Each operand word y_j (a weak
// 64-bit word) is split into its eight bytes y_ja (a = 0..7), each an fp16
// operand; each constant (2^(8a) m_ij mod p), taken in [-128 G, 127 G] with
// G = (2^64 - 1) / 255, is split into eight balanced base-256 digits
// d_ijab in [-128, 127].  Then
//   (M y)_i = sum_b 2^(8b) Z_ib  (mod p),   Z_ib = sum_(j,a) y_ja d_ijab,
// a 128 x 8K x 8N product per 128 states whose fp32 sums are exact
// integers.  A bias block adds magic_b to column (i, b) so that every sum
// lies in [2^23, 2^24) (times 2^-24), where its fp32 bits are an integer
// offset of its value, and the magics are chosen so that the offsets cancel
// mod p: (M y)_i = sum_b 2^(8b) bits(i, b) (mod p).
//
// Operands are stored in the tensor cores' K-major, unswizzled layout: 8 x 8
// fp16 "core matrices" of 128 contiguous bytes, row r at 16 r.  A table of
// N = 8 n rows (outputs) and K = 8 k columns (input words) holds core matrix
// (row group g, column chunk c) at halfs (g k + c) * 64.
constexpr int kTcN = kT * 8;   // output columns (i, b) of a 12-row table
constexpr int kTcK = kT * 8;   // K of a 12-word input
// The chain runs in two halves: s_0 .. s_10, then s_11 .. s_21; between them
// the first half's contributions to the second half's chain values are one
// contraction (the bs table).
constexpr int kTcSplit = 11;       // S-box outputs of the first half
constexpr int kTcUa = kTcSplit - 1;  // rows of the first U table (U_0 .. U_9)
static_assert(kRP - kTcUa == kT && kRP - kTcSplit < kT, "each table has at most 12 rows and 12 input words");
struct TcTables {
    // the part every tensor-core kernel copies (full rounds)
    uint16_t m[kTcN * kTcK];          // M of the full rounds
    uint16_t pre[kTcN * kTcK];        // transition matrix of full round 3
    // B operand of the bias: 8 rows b (the same for every row group: read with
    // a zero row-group stride), column 0 = 4 u_b, the rest 0; two core matrices
    uint16_t b_bias[2 * 64];
    // A operand of the bias: 8 identical rows, 2^-13 at column 0
    uint16_t a_bias[2 * 64];
    // A operand of cells 8..11 in round 0 of a state whose capacity enters as
    // zero: the bytes of (c_0[j])^7 as fp16 subnormals, 8 identical rows per
    // core matrix, one core matrix per cell
    uint16_t a_zcap[4 * 64];
    // the partial rounds' contractions (ChainParams); input word 11 of bs, w1
    // and w2 has zero digits (that A column holds a stale word)
    uint16_t vpa[kTcUa * 8 * kTcK];   // U_0 .. U_9 from y3 (80 rows)
    uint16_t vpb[kTcN * kTcK];        // U_10 .. U_21 from y3
    uint16_t bs[kTcN * kTcK];         // rows q = 10 .. 21: beta[q][r], r = 0 .. 10 (row 21 zero)
    uint16_t w1[kTcN * kTcK];         // final cells from s_0 .. s_10
    uint16_t w2[kTcN * kTcK];         // final cells from s_11 .. s_21
};
static_assert(sizeof(TcTables) % 16 == 0, "tables are copied in 16-byte pieces");

// Records the text returned by pg_last_error() and passes `status` through.
int set_error(int status, const char *fmt, ...);

// Launch timing (pg_profile_enable / pg_profile_read): a ProfScope around a
// launch records CUDA events on `stream` before and after it while timing is
// on.  Defined in pg12.cu; the stream and events are held as opaque pointers.
enum KernelId {
    kIdMerkle, kIdMerkleTop, kIdMerkleTopLeaf, kIdPermute, kIdHashRows, kIdOpen, kIdVerify, kIdSingle,
    kIdGraph, kIdNttPass, kIdNttBitrev, kIdMerkleLevel, kIdMerkleTopTail,
    kIdTcPermute, kIdTcLeaves, kIdTcLevel, kIdTcRows, kIdTcBatch, kIdBatchTop, kIdCount
};

class ProfScope {
  public:
    ProfScope(int kid, void *stream, uint64_t perms);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

  private:
    void *st_ = nullptr;
    void *a_ = nullptr, *b_ = nullptr;
    int kid_ = 0, device_ = 0;
    uint64_t perms_ = 0;
    bool active_ = false;
};

// Uploads the NTT root and coset tables to the current device (ntt.cu);
// pg_init calls it.
int ntt_upload_constants();
// PG_OK once pg_init has succeeded, else PG_ERR_NOT_INIT (pg12.cu).
int ntt_require_init();

namespace host {
uint64_t fp_add(uint64_t a, uint64_t b);
uint64_t fp_sub(uint64_t a, uint64_t b);
uint64_t fp_mul(uint64_t a, uint64_t b);
uint64_t fp_pow(uint64_t a, uint64_t e);
uint64_t fp_inv(uint64_t a);
void generate_plain(PlainParams &pp);
// pg12_small: pg12_v1's round constants and a circulant MDS matrix with
// 8-bit entries; `row` receives its first row.  Returns the accepted
// candidate's index.
int generate_small(PlainParams &pp, uint32_t row[kT]);
bool derive_optimized(const PlainParams &pp, OptParams &op);
// Chain form of the partial rounds of an optimised set.
void derive_chain(const OptParams &op, ChainParams &cp);
// Digit tables of the tensor-core contractions for an optimised set; false if
// a sum could leave the exact window (every table is checked).
bool build_tc_tables(const OptParams &op, TcTables &tt);
// The bias blocks every tensor-core contraction adds (TcTables::a_bias and
// b_bias) and their digits u_b.
void tc_bias_blocks(uint16_t a_bias[128], uint16_t b_bias[128], int u[8]);
// FIPS 180-4 SHA-256 of `len` bytes as 64 lowercase hex digits.
void sha256_hex(const uint8_t *data, size_t len, char out[65]);
}  // namespace host

}  // namespace pg12
