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

// Tensor-core form of the full rounds' dense layers (Alg. 1, MDS).  Each
// S-box output x_j is split into its eight bytes x_ja (a = 0..7), each an
// fp16 operand; each constant (2^(8a) m_ij mod p), taken in (-2^63, 2^63),
// is split into eight balanced base-256 digits d_ijab in [-128, 127].  Then
//   y_i = sum_b 2^(8b) Z_ib  (mod p),   Z_ib = sum_(j,a) x_ja d_ijab,
// a 128 x 96 x 96 product per 128 states whose fp32 sums are exact integers
// (|Z| <= 96 * 255 * 128 < 2^22).  A bias row adds magic_b to column (i, b)
// so that every sum lies in [2^23, 2^24), where its fp32 bits are an
// integer offset of its value, and the magics are chosen so that the offsets
// cancel mod p: y_i = sum_b 2^(8b) bits(i, b) (mod p).
//
// The operands are stored in the tensor cores' K-major, unswizzled layout:
// 8 x 8 fp16 "core matrices" of 128 contiguous bytes, row r at 16 r.
constexpr int kTcN = kT * 8;       // output columns (i, b)
constexpr int kTcK = kT * 8;       // data K (j, a)
constexpr int kTcKC = kTcK / 8 + 2;  // core-matrix columns of a B table: 12 data + 2 bias
struct TcTables {
    // B operand of matrix m (0: M of the full rounds, 1: the transition matrix
    // of round 3): row n = 8 i + b, column k = 8 j + a (12 data chunks), then
    // the bias chunks (column 96 = 4 u_b, the rest 0); core matrix (n/8, c)
    // at halfs (n/8 * kTcKC + c) * 64.
    uint16_t b[2][kTcN * kTcKC * 8];
    // A operand of the bias: 8 identical rows (read with a zero row-group
    // stride), 2^-13 at column 0; two core matrices.
    uint16_t a_bias[2 * 64];
    // A operand of cells 8..11 in round 0 of a state whose capacity enters as
    // zero: the bytes of (c_0[j])^7 as fp16 subnormals, 8 identical rows per
    // core matrix, one core matrix per cell.
    uint16_t a_zcap[4 * 64];
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
// Digit tables of the tensor-core dense layers for an optimised set.
void build_tc_tables(const OptParams &op, TcTables &tt);
// FIPS 180-4 SHA-256 of `len` bytes as 64 lowercase hex digits.
void sha256_hex(const uint8_t *data, size_t len, char out[65]);
}  // namespace host

}  // namespace pg12
