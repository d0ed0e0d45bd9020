/*
 * ntt_oracle.c -- plain CPU reference for the Goldilocks number-theoretic
 * transform and the low-degree extension that feeds a Merkle commitment.
 *
 * TEST INFRASTRUCTURE ONLY, like pg_oracle.c (whose field functions it uses
 * and with which it is linked into liboracle.so).  Nothing in the product
 * path may call it; it shares no code or table with the CUDA library.
 *
 * Sec. 2.3 names the NTT as zkProver's second Goldilocks hotspot (10% of its
 * time, after Merkle building) and Sec. 2.4 says the committed Merkle leaves
 * are polynomial evaluations, but the paper defines neither transform.  So
 * this file writes out the textbook definitions:
 *   - roots: g = 7 generates the multiplicative group of the field of Eq. 1
 *     (checked by the tests against the factorisation of p - 1); the
 *     primitive 2^k-th root of unity is w_k = g^((p - 1) / 2^k), k <= 32.
 *   - NTT of length n = 2^k: X_i = sum_j x_j w_k^(i j); the inverse is
 *     x_j = n^-1 sum_i X_i w_k^(-i j).  Natural order in and out.
 *   - LDE with blowup 2^b and coset shift s: the n values of a column are the
 *     evaluations of the unique polynomial P of degree < n on the subgroup
 *     {w_k^j}; the output holds P(s * w_{k+b}^i) for i < n * 2^b.
 * Data with several columns is row-major: element (row r, column c) at
 * r * ncols + c, every column transformed on its own.
 *
 * Two evaluations of the NTT are given: the definition as a double sum
 * (orc_dft_naive) and a recursive radix-2 split (orc_fft: X_i = E_i + w^i O_i,
 * X_{i+n/2} = E_i - w^i O_i, with E and O the transforms of the even- and
 * odd-indexed halves), which the tests pin to the definition on small sizes.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define ORC_P 0xFFFFFFFF00000001ULL
#define ORC_GENERATOR 7ULL

uint64_t orc_add(uint64_t a, uint64_t b);
uint64_t orc_sub(uint64_t a, uint64_t b);
uint64_t orc_mul(uint64_t a, uint64_t b);
uint64_t orc_pow(uint64_t a, uint64_t e);
uint64_t orc_inv(uint64_t a);

/* primitive 2^log_n-th root of unity (or its inverse); 0 if log_n > 32 */
uint64_t orc_two_adic_root(int log_n, int inverse) {
    if (log_n < 0 || log_n > 32) return 0;
    uint64_t w = orc_pow(ORC_GENERATOR, (ORC_P - 1) >> log_n);
    return inverse ? orc_inv(w) : w;
}

static int orc_log2(size_t n) {
    int k = 0;
    while (((size_t)1 << k) < n) ++k;
    return k;
}

/* the definition: y_i = sum_j x_j w^(i j) (inverse: w^-1 and a factor n^-1) */
int orc_dft_naive(const uint64_t *x, uint64_t *y, size_t n, int inverse) {
    if (n == 0 || (n & (n - 1))) return -1;
    const uint64_t w = orc_two_adic_root(orc_log2(n), inverse);
    for (size_t i = 0; i < n; ++i) {
        const uint64_t wi = orc_pow(w, (uint64_t)i);
        uint64_t acc = 0, wij = 1;
        for (size_t j = 0; j < n; ++j) {
            acc = orc_add(acc, orc_mul(x[j], wij));
            wij = orc_mul(wij, wi);
        }
        y[i] = acc;
    }
    if (inverse) {
        const uint64_t ninv = orc_inv((uint64_t)n % ORC_P);
        for (size_t i = 0; i < n; ++i) y[i] = orc_mul(y[i], ninv);
    }
    return 0;
}

/* recursive radix-2 transform with root w (unnormalised), in place */
static void orc_fft_rec(uint64_t *x, size_t n, uint64_t w, uint64_t *tmp) {
    if (n == 1) return;
    const size_t h = n / 2;
    uint64_t *even = tmp, *odd = tmp + h;
    for (size_t j = 0; j < h; ++j) {
        even[j] = x[2 * j];
        odd[j] = x[2 * j + 1];
    }
    memcpy(x, tmp, n * sizeof(uint64_t));  /* x = [even | odd], tmp free again */
    const uint64_t w2 = orc_mul(w, w);
    orc_fft_rec(x, h, w2, tmp);
    orc_fft_rec(x + h, h, w2, tmp);
    uint64_t wi = 1;
    for (size_t i = 0; i < h; ++i) {
        const uint64_t e = x[i], t = orc_mul(wi, x[h + i]);
        tmp[i] = orc_add(e, t);
        tmp[h + i] = orc_sub(e, t);
        wi = orc_mul(wi, w);
    }
    memcpy(x, tmp, n * sizeof(uint64_t));
}

/* same result as orc_dft_naive, in place */
int orc_fft(uint64_t *x, size_t n, int inverse) {
    if (n == 0 || (n & (n - 1))) return -1;
    uint64_t *tmp = (uint64_t *)malloc(n * sizeof(uint64_t));
    if (!tmp) return -2;
    orc_fft_rec(x, n, orc_two_adic_root(orc_log2(n), inverse), tmp);
    free(tmp);
    if (inverse) {
        const uint64_t ninv = orc_inv((uint64_t)n % ORC_P);
        for (size_t i = 0; i < n; ++i) x[i] = orc_mul(x[i], ninv);
    }
    return 0;
}

/* every column of a row-major n x ncols array, in place */
int orc_ntt_columns(uint64_t *data, size_t n, size_t ncols, int inverse) {
    if (n == 0 || (n & (n - 1)) || ncols == 0) return -1;
    uint64_t *col = (uint64_t *)malloc(n * sizeof(uint64_t));
    if (!col) return -2;
    for (size_t c = 0; c < ncols; ++c) {
        for (size_t r = 0; r < n; ++r) col[r] = data[r * ncols + c] % ORC_P;
        int e = orc_fft(col, n, inverse);
        if (e) {
            free(col);
            return e;
        }
        for (size_t r = 0; r < n; ++r) data[r * ncols + c] = col[r];
    }
    free(col);
    return 0;
}

/* Horner evaluation of sum_j c_j x^j */
uint64_t orc_poly_eval(const uint64_t *coeffs, size_t n, uint64_t x) {
    uint64_t acc = 0;
    for (size_t j = n; j-- > 0;) acc = orc_add(orc_mul(acc, x), coeffs[j] % ORC_P);
    return acc;
}

/* coefficients of each column's interpolant: the inverse NTT, row-major */
int orc_interpolate_columns(const uint64_t *evals, size_t n, size_t ncols, uint64_t *coeffs) {
    memcpy(coeffs, evals, n * ncols * sizeof(uint64_t));
    return orc_ntt_columns(coeffs, n, ncols, 1);
}

/* LDE: out[i][c] = P_c(shift * w_{k+b}^i), i < n 2^b, P_c the interpolant of column c */
int orc_lde_columns(const uint64_t *evals, size_t n, size_t ncols, int log_blowup, uint64_t shift,
                    uint64_t *out) {
    if (n == 0 || (n & (n - 1)) || ncols == 0 || log_blowup < 0 || log_blowup > 16) return -1;
    const size_t big = n << log_blowup;
    uint64_t *col = (uint64_t *)malloc(big * sizeof(uint64_t));
    if (!col) return -2;
    for (size_t c = 0; c < ncols; ++c) {
        for (size_t r = 0; r < n; ++r) col[r] = evals[r * ncols + c] % ORC_P;
        int e = orc_fft(col, n, 1); /* coefficients c_j */
        if (!e) {
            uint64_t sj = 1; /* c_j s^j: P(s x) = sum_j (c_j s^j) x^j */
            for (size_t j = 0; j < n; ++j) {
                col[j] = orc_mul(col[j], sj);
                sj = orc_mul(sj, shift % ORC_P);
            }
            for (size_t j = n; j < big; ++j) col[j] = 0;
            e = orc_fft(col, big, 0);
        }
        if (e) {
            free(col);
            return e;
        }
        for (size_t r = 0; r < big; ++r) out[r * ncols + c] = col[r];
    }
    free(col);
    return 0;
}
