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

// Records the text returned by pg_last_error() and passes `status` through.
int set_error(int status, const char *fmt, ...);

// Launch timing (pg_profile_enable / pg_profile_read): a ProfScope around a
// launch records CUDA events on `stream` before and after it while timing is
// on.  Defined in pg12.cu; the stream and events are held as opaque pointers.
enum KernelId {
    kIdMerkle, kIdMerkleTop, kIdMerkleTopLeaf, kIdPermute, kIdHashRows, kIdOpen, kIdVerify, kIdSingle,
    kIdGraph, kIdNttPass, kIdNttBitrev, kIdMerkleLevel, kIdMerkleTopTail, kIdCount
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
// FIPS 180-4 SHA-256 of `len` bytes as 64 lowercase hex digits.
void sha256_hex(const uint8_t *data, size_t len, char out[65]);
}  // namespace host

}  // namespace pg12
