// Host-side parameter construction for the device permutation.
//
// 1. Parameter set pg12_v1 (the paper prints none of the constants C, M, S
//    that Alg. 1 names): the Poseidon paper's Grain-LFSR procedure seeded
//    with (prime field, x^alpha S-box, n = 64, t = 12, R_F = 8, R_P = 22) --
//    80-bit register, 160 discarded clocks, self-shrinking output (a bit is
//    emitted only when the clock before it produced a 1), 64-bit big-endian
//    words rejected when >= p.  360 round constants come first, then 24
//    points x_0..x_11, y_0..y_11 for the Cauchy matrix M[i][j] = 1/(x_i+y_j);
//    the 24 are drawn again if any two coincide or some x_i + y_j = 0.
// 2. The sparse rewrite of the 22 partial rounds that Alg. 1 uses
//    (MDSPartial with its vec[2][12] per round), derived here from (C, M):
//    - constants: a partial round's S-box touches cell 0 only, so cells
//      1..11 of its constant are carried through the S-box and the matrix
//      into the next round's constant; each partial round keeps one scalar
//      and the remainder lands in the constant of the first full round of
//      the second half;
//    - matrices: going backwards from the last partial round, the round's
//      matrix N is factored as N = A * B with B = diag(1, N_hat) (which
//      commutes with a cell-0 S-box and with cell-0 constants) and A sparse,
//      A = [[n00, v^T], [n_col, I]] with v = N_hat^-T n_row; B is pushed
//      into the previous round, so full round 3 ends with the dense
//      "transition" matrix B_first * M.
#include "pg12_internal.h"

#include <cstring>
#include <vector>

namespace pg12 {
namespace host {

static inline uint64_t fp_reduce(unsigned __int128 v) { return (uint64_t)(v % kP); }
uint64_t fp_add(uint64_t a, uint64_t b) { return fp_reduce((unsigned __int128)a + b); }
uint64_t fp_sub(uint64_t a, uint64_t b) { return fp_add(a, b == 0 ? 0 : kP - (b % kP)); }
uint64_t fp_mul(uint64_t a, uint64_t b) { return fp_reduce((unsigned __int128)a * b); }
uint64_t fp_pow(uint64_t a, uint64_t e) {
    uint64_t acc = 1, base = a % kP;
    for (; e; e >>= 1, base = fp_mul(base, base))
        if (e & 1) acc = fp_mul(acc, base);
    return acc;
}
uint64_t fp_inv(uint64_t a) { return fp_pow(a, kP - 2); }

// ---------------------------------------------------------------- Grain LFSR
namespace {
class Grain {
  public:
    Grain(unsigned field, unsigned sbox, unsigned n, unsigned t, unsigned rf, unsigned rp) {
        // register bits s[0] (oldest) .. s[79]; packed as a bit queue
        int k = 0;
        auto push = [&](uint64_t v, int bits) {
            for (int b = bits - 1; b >= 0; --b) s_[k++] = (uint8_t)((v >> b) & 1u);
        };
        push(field, 2);
        push(sbox, 4);
        push(n, 12);
        push(t, 12);
        push(rf, 10);
        push(rp, 10);
        push(0x3FFFFFFFull, 30);
        head_ = 0;
        for (int i = 0; i < 160; ++i) step();
    }
    // One register clock; the taps are s[0], s[13], s[23], s[38], s[51], s[62].
    int step() {
        auto at = [&](int i) { return (int)s_[(head_ + i) % 80]; };
        int nb = at(0) ^ at(13) ^ at(23) ^ at(38) ^ at(51) ^ at(62);
        s_[head_] = (uint8_t)nb;  // the oldest slot becomes the newest bit
        head_ = (head_ + 1) % 80;
        return nb;
    }
    int bit() {
        for (;;) {
            int gate = step();
            int out = step();
            if (gate) return out;
        }
    }
    uint64_t word64() {
        uint64_t w = 0;
        for (int i = 0; i < 64; ++i) w = (w << 1) | (uint64_t)bit();
        return w;
    }
    uint64_t element() {
        uint64_t w;
        do { w = word64(); } while (w >= kP);
        return w;
    }

  private:
    uint8_t s_[80];
    int head_;
};
}  // namespace

void generate_plain(PlainParams &pp) {
    Grain g(1, 0, 64, kT, kRF, kRP);
    for (int r = 0; r < kRounds; ++r)
        for (int i = 0; i < kT; ++i) pp.rc[r][i] = g.element();
    for (;;) {
        uint64_t pts[2 * kT];
        for (auto &p : pts) p = g.element();
        bool good = true;
        for (int a = 0; a < 2 * kT && good; ++a)
            for (int b = 0; b < a; ++b)
                if (pts[a] == pts[b]) { good = false; break; }
        for (int i = 0; i < kT && good; ++i)
            for (int j = 0; j < kT; ++j)
                if (fp_add(pts[i], pts[kT + j]) == 0) { good = false; break; }
        if (!good) continue;
        for (int i = 0; i < kT; ++i)
            for (int j = 0; j < kT; ++j) pp.mds[i][j] = fp_inv(fp_add(pts[i], pts[kT + j]));
        return;
    }
}

// --------------------------------------------- small-entry parameter set
namespace {
// Goldilocks product without a division: 2^64 = 2^32 - 1, 2^96 = -1.
inline uint64_t fast_mul(uint64_t a, uint64_t b) {
    const unsigned __int128 r = (unsigned __int128)a * b;
    const uint64_t lo = (uint64_t)r, hi = (uint64_t)(r >> 64);
    const uint64_t hl = hi & 0xFFFFFFFFull, hh = hi >> 32;
    uint64_t t = lo - hh;
    if (lo < hh) t -= 0xFFFFFFFFull;
    const uint64_t u = (hl << 32) - hl;
    uint64_t v = t + u;
    if (v < u) v += 0xFFFFFFFFull;
    return v >= kP ? v - kP : v;
}
inline uint64_t fast_sub(uint64_t a, uint64_t b) { return a >= b ? a - b : a + (kP - b); }

// Nonsingular k x k submatrix?  Elimination by cross-multiplication
// (row_j <- p * row_j - f * row_pivot), so no inverses are needed.
bool minor_nonsingular(uint64_t (&a)[kT][kT], int k) {
    for (int c = 0; c < k; ++c) {
        int piv = -1;
        for (int r = c; r < k; ++r)
            if (a[r][c]) { piv = r; break; }
        if (piv < 0) return false;
        if (piv != c)
            for (int j = c; j < k; ++j) std::swap(a[piv][j], a[c][j]);
        const uint64_t p = a[c][c];
        for (int r = c + 1; r < k; ++r) {
            const uint64_t f = a[r][c];
            if (!f) continue;
            for (int j = c; j < k; ++j) a[r][j] = fast_sub(fast_mul(p, a[r][j]), fast_mul(f, a[c][j]));
        }
    }
    return true;
}

// MDS test of a circulant matrix: every square submatrix nonsingular.  A
// submatrix and its copy shifted by s along both axes are equal, so only row
// sets that contain row 0 are visited.
bool circulant_is_mds(const uint64_t (&m)[kT][kT]) {
    uint64_t a[kT][kT];
    for (int k = 1; k <= kT; ++k) {
        for (int rs = 1; rs < (1 << kT); rs += 2) {  // row 0 always present
            if (__builtin_popcount((unsigned)rs) != k) continue;
            int rows[kT], nr = 0;
            for (int i = 0; i < kT; ++i)
                if (rs >> i & 1) rows[nr++] = i;
            for (int cs = 1; cs < (1 << kT); ++cs) {
                if (__builtin_popcount((unsigned)cs) != k) continue;
                int cols[kT], nc = 0;
                for (int j = 0; j < kT; ++j)
                    if (cs >> j & 1) cols[nc++] = j;
                for (int i = 0; i < k; ++i)
                    for (int j = 0; j < k; ++j) a[i][j] = m[rows[i]][cols[j]];
                if (!minor_nonsingular(a, k)) return false;
            }
        }
    }
    return true;
}
}  // namespace

int generate_small(PlainParams &pp, uint32_t row[kT]) {
    Grain g(1, 0, 64, kT, kRF, kRP);
    for (int r = 0; r < kRounds; ++r)
        for (int i = 0; i < kT; ++i) pp.rc[r][i] = g.element();
    for (int cand = 0;; ++cand) {
        uint32_t c[kT];
        for (auto &v : c) v = (uint32_t)(1 + g.word64() % 255);
        for (int i = 0; i < kT; ++i)
            for (int j = 0; j < kT; ++j) pp.mds[i][j] = c[((j - i) % kT + kT) % kT];
        if (circulant_is_mds(pp.mds)) {
            for (int i = 0; i < kT; ++i) row[i] = c[i];
            return cand;
        }
    }
}

// ------------------------------------------------------- sparse rewrite
namespace {
using Mat = std::vector<std::vector<uint64_t>>;

Mat matmul(const Mat &a, const Mat &b) {
    size_t n = a.size(), m = b[0].size(), k = b.size();
    Mat c(n, std::vector<uint64_t>(m, 0));
    for (size_t i = 0; i < n; ++i)
        for (size_t j = 0; j < m; ++j) {
            uint64_t s = 0;
            for (size_t l = 0; l < k; ++l) s = fp_add(s, fp_mul(a[i][l], b[l][j]));
            c[i][j] = s;
        }
    return c;
}

// Solve A x = b over F_p (A square, invertible); returns false if singular.
bool solve(Mat a, std::vector<uint64_t> b, std::vector<uint64_t> &x) {
    const size_t n = a.size();
    for (size_t col = 0; col < n; ++col) {
        size_t piv = col;
        while (piv < n && a[piv][col] == 0) ++piv;
        if (piv == n) return false;
        std::swap(a[piv], a[col]);
        std::swap(b[piv], b[col]);
        uint64_t inv = fp_inv(a[col][col]);
        for (size_t j = col; j < n; ++j) a[col][j] = fp_mul(a[col][j], inv);
        b[col] = fp_mul(b[col], inv);
        for (size_t r = 0; r < n; ++r) {
            if (r == col || a[r][col] == 0) continue;
            uint64_t f = a[r][col];
            for (size_t j = col; j < n; ++j) a[r][j] = fp_sub(a[r][j], fp_mul(f, a[col][j]));
            b[r] = fp_sub(b[r], fp_mul(f, b[col]));
        }
    }
    x = b;
    return true;
}
}  // namespace

bool derive_optimized(const PlainParams &pp, OptParams &op) {
    const int first_part = kRF / 2, last_part = kRF / 2 + kRP - 1;
    Mat M(kT, std::vector<uint64_t>(kT));
    for (int i = 0; i < kT; ++i)
        for (int j = 0; j < kT; ++j) M[i][j] = pp.mds[i][j];

    // constants: forward carry of cells 1..11 through each partial round
    std::vector<uint64_t> carry(kT, 0);  // constant still to be added before the next S-box
    for (int i = 0; i < kT; ++i) carry[i] = pp.rc[first_part][i];
    for (int r = first_part; r <= last_part; ++r) {
        op.part_rc[r - first_part] = carry[0];
        std::vector<uint64_t> rest(kT, 0);
        for (int i = 1; i < kT; ++i) rest[i] = carry[i];
        std::vector<uint64_t> next(kT, 0);
        for (int i = 0; i < kT; ++i) {
            uint64_t s = 0;
            for (int j = 1; j < kT; ++j) s = fp_add(s, fp_mul(M[i][j], rest[j]));
            next[i] = s;
        }
        for (int i = 0; i < kT; ++i) carry[i] = fp_add(next[i], pp.rc[r + 1][i]);
    }
    // full-round constants: rounds 0..3, then 26 (with the carried remainder), 27..29
    for (int r = 0; r < first_part; ++r)
        for (int i = 0; i < kT; ++i) op.full_rc[r][i] = pp.rc[r][i];
    for (int i = 0; i < kT; ++i) op.full_rc[first_part][i] = carry[i];
    for (int r = last_part + 2; r < kRounds; ++r)
        for (int i = 0; i < kT; ++i) op.full_rc[r - kRP][i] = pp.rc[r][i];

    // matrices: backwards factorisation N = A * diag(1, N_hat)
    Mat N = M;
    for (int r = last_part; r >= first_part; --r) {
        const int q = r - first_part;
        Mat Nhat_T(kT - 1, std::vector<uint64_t>(kT - 1));
        for (int i = 1; i < kT; ++i)
            for (int j = 1; j < kT; ++j) Nhat_T[j - 1][i - 1] = N[i][j];
        std::vector<uint64_t> nrow(kT - 1), v;
        for (int j = 1; j < kT; ++j) nrow[j - 1] = N[0][j];
        if (!solve(Nhat_T, nrow, v)) return false;
        op.part_v[q][0] = N[0][0];
        for (int j = 1; j < kT; ++j) op.part_v[q][j] = v[j - 1];
        for (int i = 1; i < kT; ++i) op.part_w[q][i - 1] = N[i][0];
        Mat B(kT, std::vector<uint64_t>(kT, 0));
        B[0][0] = 1;
        for (int i = 1; i < kT; ++i)
            for (int j = 1; j < kT; ++j) B[i][j] = N[i][j];
        N = matmul(B, M);  // the previous round's matrix absorbs B
    }
    for (int i = 0; i < kT; ++i)
        for (int j = 0; j < kT; ++j) {
            op.mds[i][j] = pp.mds[i][j];
            op.pre[i][j] = N[i][j];
        }
    return true;
}

// ------------------------------------------------------------ tensor-core digit tables
namespace {

// fp16 bits of a nonzero integer below 2^16 with at most 11 significant bits
// (exactly representable).
uint16_t half_of_int(int v) {
    if (v == 0) return 0;
    const uint16_t sign = v < 0 ? 0x8000u : 0u;
    uint32_t m = (uint32_t)(v < 0 ? -v : v);
    int e = 0;
    while ((m >> e) > 1) ++e;  // 2^e <= m < 2^(e+1)
    const uint32_t frac = (e <= 10 ? m << (10 - e) : m >> (e - 10)) & 0x3FFu;  // 10 fraction bits
    return (uint16_t)(sign | ((uint32_t)(e + 15) << 10) | frac);
}

// Eight balanced base-256 digits of a residue: the representative v in
// [-128 (2^64-1)/255, 127 (2^64-1)/255] (an interval of 2^64 - 1 > p
// integers) written as sum_b d_b 256^b with d_b in [-128, 127].
void balanced_digits(uint64_t r, int d[8]) {
    const unsigned __int128 hi = (unsigned __int128)127 * 0x0101010101010101ull;
    __int128 v = (unsigned __int128)r <= hi ? (__int128)r : (__int128)r - (__int128)kP;
    for (int b = 0; b < 8; ++b) {
        __int128 q = v >= 0 ? v / 256 : -((-v + 255) / 256);  // floor(v / 256)
        int rem = (int)(v - q * 256);                          // in [0, 256)
        if (rem >= 128) {
            rem -= 256;
            ++q;
        }
        d[b] = rem;
        v = q;
    }
}

}  // namespace

void derive_chain(const OptParams &op, ChainParams &cp) {
    std::memset(&cp, 0, sizeof cp);
    // v_q[i] and w_r[i] for i = 0..11 (w_r[0] unused)
    auto v = [&](int q, int i) { return op.part_v[q][i] % kP; };
    auto w = [&](int r, int i) { return op.part_w[r][i - 1] % kP; };
    for (int q = 0; q < kRP; ++q)
        for (int j = 0; j < kT; ++j) {
            uint64_t acc = 0;
            for (int i = 1; i < kT; ++i) acc = fp_add(acc, fp_mul(v(q, i), op.pre[i][j] % kP));
            cp.vp[q][j] = acc;
        }
    for (int q = 0; q < kRP; ++q) {
        for (int r = 0; r < q; ++r) {
            uint64_t acc = 0;
            for (int i = 1; i < kT; ++i) acc = fp_add(acc, fp_mul(v(q, i), w(r, i)));
            cp.beta[q][r] = acc;
        }
        cp.beta[q][q] = v(q, 0);
    }
    for (int r = 0; r < kRP; ++r) {
        cp.w[0][r] = cp.beta[kRP - 1][r];
        for (int i = 1; i < kT; ++i) cp.w[i][r] = w(r, i);
    }
}

namespace {

// Digit table of an (n x k) matrix mat (row-major, canonical words): output
// row i, input word j; B operand row 8 i + b, column 8 j + a holds digit b of
// 2^(8a) mat[i][j].  Records, per output column, the largest positive and
// negative sums of digits over the table (for the exactness check).
void digit_table(const uint64_t *mat, int n, int k, uint16_t *dst, long *pos, long *neg) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < k; ++j)
            for (int a = 0; a < 8; ++a) {
                int d[8];
                balanced_digits(fp_mul(mat[i * k + j] % kP, fp_pow(2, 8 * (uint64_t)a)), d);
                for (int b = 0; b < 8; ++b) {
                    const int row = 8 * i + b;
                    dst[(row / 8 * k + j) * 64 + (row % 8) * 8 + a] = half_of_int(d[b]);
                    if (d[b] > 0) pos[row] += d[b];
                    else neg[row] -= d[b];
                }
            }
}

}  // namespace

void tc_bias_blocks(uint16_t a_bias[128], uint16_t b_bias[128], int u[8]) {
    // Bias digits u_b: column (i, b) reads back bits = 0x3E800000 + magic_b + Z
    // with magic_b = 8192 u_b (A bias 2^-13 times B bias 4 u_b, values scaled by
    // 2^-24), and sum_b 2^(8b) (0x3E800000 + 8192 u_b) = 0 (mod p) is solved for
    // u_b in [1407, 1665], the range that keeps magic_b + Z in [2^23, 2^24) for
    // |Z| <= 3133440 (96 products of a byte and a digit).  The sums
    // sum_b u_b 2^(8b) cover every integer from 1407 G to 1665 G (G = sum_b
    // 2^(8b); 259 digit values for radix 256), an interval longer than p, so a
    // solution exists.
    typedef unsigned __int128 u128;
    const uint64_t G = 0x0101010101010101ull;
    const uint64_t Gp = G % kP;
    const uint64_t c0 = fp_mul(0x3E800000ull, Gp);              // sum_b 2^(8b) 0x3E800000 mod p
    const uint64_t t = fp_mul(fp_sub(0, c0), fp_inv(8192));     // wanted sum_b u_b 2^(8b) mod p
    const u128 umin = (u128)1407 * G;
    const uint64_t umin_p = (uint64_t)(umin % kP);
    u128 rest = fp_sub(t, umin_p);                               // U - umin, in [0, p)
    for (int b = 7; b >= 0; --b) {
        const u128 wgt = (u128)1 << (8 * b);
        u128 e = rest / wgt;
        if (e > 258) e = 258;
        rest -= e * wgt;
        u[b] = 1407 + (int)e;
    }
    std::memset(a_bias, 0, 128 * sizeof(uint16_t));
    std::memset(b_bias, 0, 128 * sizeof(uint16_t));
    for (int b = 0; b < 8; ++b) b_bias[b * 8] = half_of_int(4 * u[b]);
    for (int r = 0; r < 8; ++r) a_bias[r * 8] = 0x0800;  // 2^-13
}

bool build_tc_tables(const OptParams &op, TcTables &tt) {
    std::memset(&tt, 0, sizeof tt);
    int u[8];
    tc_bias_blocks(tt.a_bias, tt.b_bias, u);

    ChainParams cp;
    derive_chain(op, cp);
    static uint64_t m[kT * kT], pre[kT * kT], vpa[kTcUa * kT], vpb[kT * kT], bs[kT * kT], w1[kT * kT], w2[kT * kT];
    for (int i = 0; i < kT; ++i)
        for (int j = 0; j < kT; ++j) {
            m[i * kT + j] = op.mds[i][j] % kP;
            pre[i * kT + j] = op.pre[i][j] % kP;
            if (i < kTcUa) vpa[i * kT + j] = cp.vp[i][j];
            vpb[i * kT + j] = cp.vp[kTcUa + i][j];
            const int q = kTcUa + i;  // bs: the first half's s_r in c_(q+1), q = 10 .. 20
            bs[i * kT + j] = (q < kRP - 1 && j < kTcSplit) ? cp.beta[q][j] : 0;
            w1[i * kT + j] = j < kTcSplit ? cp.w[i][j] : 0;
            w2[i * kT + j] = j < kRP - kTcSplit ? cp.w[i][kTcSplit + j] : 0;
        }
    // every accumulation's worst sums: magic_b - 255 neg >= 2^23 and
    // magic_b + 255 pos < 2^24 for each column; the second half's chain values
    // accumulate vpb and bs into one sum, the final cells w1 and w2
    bool ok = true;
    auto check = [&](const long *pos, const long *neg, int rows) {
        for (int r = 0; r < rows; ++r) {
            const long magic = 8192L * u[r % 8];
            ok = ok && magic - 255 * neg[r] >= (1L << 23) && magic + 255 * pos[r] < (1L << 24);
        }
    };
    {
        long pos[kTcN] = {}, neg[kTcN] = {};
        digit_table(m, kT, kT, tt.m, pos, neg);
        check(pos, neg, kTcN);
    }
    {
        long pos[kTcN] = {}, neg[kTcN] = {};
        digit_table(pre, kT, kT, tt.pre, pos, neg);
        check(pos, neg, kTcN);
    }
    {
        long pos[kTcN] = {}, neg[kTcN] = {};
        digit_table(vpa, kTcUa, kT, tt.vpa, pos, neg);
        check(pos, neg, kTcUa * 8);
    }
    {
        long pos[kTcN] = {}, neg[kTcN] = {};
        digit_table(vpb, kT, kT, tt.vpb, pos, neg);
        digit_table(bs, kT, kT, tt.bs, pos, neg);
        check(pos, neg, kTcN);
    }
    {
        long pos[kTcN] = {}, neg[kTcN] = {};
        digit_table(w1, kT, kT, tt.w1, pos, neg);
        digit_table(w2, kT, kT, tt.w2, pos, neg);
        check(pos, neg, kTcN);
    }
    for (int j = kRate; j < kT; ++j) {
        const uint64_t c = op.full_rc[0][j] % kP;
        const uint64_t c7 = fp_pow(c, 7);
        for (int r = 0; r < 8; ++r)
            for (int a = 0; a < 8; ++a) tt.a_zcap[(j - kRate) * 64 + r * 8 + a] = (uint16_t)((c7 >> (8 * a)) & 0xFF);
    }
    return ok;
}

// ------------------------------------------------------------ SHA-256
// FIPS 180-4 SHA-256 of a byte string, used to fingerprint a parameter set.
// Its constants are computed from their definition rather than tabulated:
// the initial hash words are the first 32 fractional bits of the square
// roots of the first 8 primes, the round constants those of the cube roots
// of the first 64 primes (integer roots of p * 2^64 and p * 2^96).
namespace {

typedef unsigned __int128 u128;

// Both roots below are under 2^36 (primes up to 311, scaled by 2^64 / 2^96),
// so the searches run over [0, 2^40], where mid^3 cannot overflow.
uint64_t isqrt128(u128 v) {  // floor(sqrt(v)) for v < 2^80
    uint64_t lo = 0, hi = 1ull << 40;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo + 1) / 2;
        if ((u128)mid * mid <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

uint64_t icbrt128(u128 v) {  // floor(cbrt(v)) for v < 2^120
    uint64_t lo = 0, hi = 1ull << 40;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo + 1) / 2;
        if ((u128)mid * mid * mid <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct ShaConsts {
    uint32_t h0[8], k[64];
    ShaConsts() {
        int found = 0;
        for (uint32_t n = 2; found < 64; ++n) {
            bool prime = true;
            for (uint32_t d = 2; d * d <= n; ++d)
                if (n % d == 0) prime = false;
            if (!prime) continue;
            if (found < 8) h0[found] = (uint32_t)isqrt128((u128)n << 64);
            k[found] = (uint32_t)icbrt128((u128)n << 96);
            ++found;
        }
    }
};

inline uint32_t rotr(uint32_t x, int r) { return (x >> r) | (x << (32 - r)); }

void sha_block(uint32_t h[8], const uint8_t *blk, const ShaConsts &c) {
    uint32_t w[64];
    for (int i = 0; i < 16; ++i)
        w[i] = ((uint32_t)blk[4 * i] << 24) | ((uint32_t)blk[4 * i + 1] << 16) | ((uint32_t)blk[4 * i + 2] << 8) |
               (uint32_t)blk[4 * i + 3];
    for (int i = 16; i < 64; ++i) {
        const uint32_t s0 = rotr(w[i - 15], 7) ^ rotr(w[i - 15], 18) ^ (w[i - 15] >> 3);
        const uint32_t s1 = rotr(w[i - 2], 17) ^ rotr(w[i - 2], 19) ^ (w[i - 2] >> 10);
        w[i] = w[i - 16] + s0 + w[i - 7] + s1;
    }
    uint32_t a = h[0], b = h[1], cc = h[2], d = h[3], e = h[4], f = h[5], g = h[6], hh = h[7];
    for (int i = 0; i < 64; ++i) {
        const uint32_t t1 = hh + (rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25)) + ((e & f) ^ (~e & g)) + c.k[i] + w[i];
        const uint32_t t2 = (rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22)) + ((a & b) ^ (a & cc) ^ (b & cc));
        hh = g;
        g = f;
        f = e;
        e = d + t1;
        d = cc;
        cc = b;
        b = a;
        a = t1 + t2;
    }
    h[0] += a; h[1] += b; h[2] += cc; h[3] += d; h[4] += e; h[5] += f; h[6] += g; h[7] += hh;
}

}  // namespace

void sha256_hex(const uint8_t *data, size_t len, char out[65]) {
    static const ShaConsts c;
    uint32_t h[8];
    std::memcpy(h, c.h0, sizeof h);
    size_t off = 0;
    for (; off + 64 <= len; off += 64) sha_block(h, data + off, c);
    uint8_t tail[128] = {0};
    const size_t rem = len - off;
    std::memcpy(tail, data + off, rem);
    tail[rem] = 0x80;
    const size_t tlen = rem + 9 <= 64 ? 64 : 128;
    const uint64_t bits = (uint64_t)len * 8;
    for (int i = 0; i < 8; ++i) tail[tlen - 1 - i] = (uint8_t)(bits >> (8 * i));
    for (size_t o = 0; o < tlen; o += 64) sha_block(h, tail + o, c);
    static const char hex[] = "0123456789abcdef";
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) out[8 * i + j] = hex[(h[i] >> (28 - 4 * j)) & 15];
    out[64] = 0;
}

}  // namespace host
}  // namespace pg12
