"""Pins of the NTT / LDE oracle against facts that do not come from it.

The transform is the textbook one (the paper names the NTT as a zkProver
hotspot in Sec. 2.3 without defining it).  Each check below uses Python's
own big integers: the factorisation of p - 1 and the order of the generator,
the defining properties of the roots, closed-form transforms of unit
vectors, brute-force cyclic convolution, and low-degree extensions evaluated
point by point from random coefficients.  A wrong root, a transposed index,
a dropped factor n^-1 or a wrong coset power fails at least one of them.
"""
import numpy as np
import pytest

import oracle
import pg_synth

P = oracle.P


def _is_prime(q: int) -> bool:
    if q < 2:
        return False
    d = 2
    while d * d <= q:
        if q % d == 0:
            return False
        d += 1
    return True


def test_generator_has_full_order():
    factors = [2, 3, 5, 17, 257, 65537]
    assert (1 << 32) * 3 * 5 * 17 * 257 * 65537 == P - 1
    assert all(_is_prime(q) for q in factors)
    for q in factors:
        assert pow(oracle.GENERATOR, (P - 1) // q, P) != 1


@pytest.mark.parametrize("k", list(range(0, 33)))
def test_two_adic_roots_are_primitive(k):
    w = oracle.two_adic_root(k)
    assert pow(w, 1 << k, P) == 1
    if k >= 1:
        assert pow(w, 1 << (k - 1), P) == P - 1
        assert oracle.two_adic_root(k - 1) == w * w % P
    assert w * oracle.two_adic_root(k, inverse=True) % P == 1
    assert w == pow(oracle.GENERATOR, (P - 1) >> k, P)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 32])
def test_dft_of_unit_vectors_closed_form(n):
    k = n.bit_length() - 1
    w = oracle.two_adic_root(k)
    for m in sorted({0, min(1, n - 1), n // 2, n - 1}):
        x = np.zeros(n, dtype=np.uint64)
        x[m] = 1
        want = [pow(w, m * i, P) for i in range(n)]
        assert [int(v) for v in oracle.dft_naive(x)] == want
        winv = pow(w, P - 2, P)
        ninv = pow(n, P - 2, P)
        want_inv = [pow(winv, m * i, P) * ninv % P for i in range(n)]
        assert [int(v) for v in oracle.dft_naive(x, inverse=True)] == want_inv
    ones = np.ones(n, dtype=np.uint64)
    assert [int(v) for v in oracle.dft_naive(ones)] == [n % P] + [0] * (n - 1)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256])
def test_fft_matches_definition(n):
    x = pg_synth.words(0x4E54 + n, n)
    assert (oracle.fft(x) == oracle.dft_naive(x)).all()
    assert (oracle.fft(x, inverse=True) == oracle.dft_naive(x, inverse=True)).all()


@pytest.mark.parametrize("n", [2, 1024, 1 << 14])
def test_fft_round_trip(n):
    x = pg_synth.words(0x4E55 + n, n)
    assert (oracle.fft(oracle.fft(x), inverse=True) == x).all()


def test_convolution_theorem_against_brute_force():
    n = 32
    a = [int(v) for v in pg_synth.words(0x4E56, n)]
    b = [int(v) for v in pg_synth.words(0x4E57, n)]
    conv = [sum(a[j] * b[(i - j) % n] for j in range(n)) % P for i in range(n)]
    fa = oracle.fft(np.array(a, dtype=np.uint64))
    fb = oracle.fft(np.array(b, dtype=np.uint64))
    prod = np.array([int(x) * int(y) % P for x, y in zip(fa, fb)], dtype=np.uint64)
    assert [int(v) for v in oracle.fft(prod, inverse=True)] == conv


def test_columns_are_independent_and_row_major():
    n, c = 64, 5
    d = pg_synth.matrix(0x4E58, n, c)
    got = oracle.ntt_columns(d)
    for j in range(c):
        assert (got[:, j] == oracle.fft(np.ascontiguousarray(d[:, j]))).all()
    assert (oracle.ntt_columns(got, inverse=True) == d).all()


def test_non_canonical_words_are_reduced():
    n = 8
    x = np.array([P, P + 1, (1 << 64) - 1, 0, 1, 2, 3, P - 1], dtype=np.uint64)
    xc = np.array([int(v) % P for v in x], dtype=np.uint64)
    d = x.reshape(n, 1)
    assert (oracle.ntt_columns(d)[:, 0] == oracle.dft_naive(xc)).all()


def test_horner():
    c = [int(v) for v in pg_synth.words(0x4E59, 17)]
    x = 0x123456789
    assert oracle.poly_eval(np.array(c, dtype=np.uint64), x) == sum(cj * pow(x, j, P) for j, cj in enumerate(c)) % P


def _evals_of(coeffs, n):
    w = oracle.two_adic_root(n.bit_length() - 1)
    return [[sum(int(coeffs[j][c]) * pow(w, i * j, P) for j in range(n)) % P
             for c in range(coeffs.shape[1])] for i in range(n)]


def test_interpolation_recovers_coefficients():
    n, cols = 16, 3
    coeffs = pg_synth.matrix(0x4E5A, n, cols)
    evals = np.array(_evals_of(coeffs, n), dtype=np.uint64)
    assert (oracle.interpolate_columns(evals) == coeffs).all()


@pytest.mark.parametrize("log_n,log_b,shift", [(4, 2, 7), (3, 1, 7), (0, 3, 7), (4, 0, 7), (2, 2, 1), (5, 3, 12345)])
def test_lde_is_evaluation_on_the_shifted_coset(log_n, log_b, shift):
    n, cols = 1 << log_n, 3
    coeffs = pg_synth.matrix(0x4E5B + log_n, n, cols)
    evals = np.array(_evals_of(coeffs, n), dtype=np.uint64).reshape(n, cols)
    got = oracle.lde_columns(evals, log_b, shift=shift)
    big = n << log_b
    wb = oracle.two_adic_root(log_n + log_b)
    for i in range(big):
        x = shift * pow(wb, i, P) % P
        for c in range(cols):
            assert int(got[i, c]) == sum(int(coeffs[j][c]) * pow(x, j, P) for j in range(n)) % P


def test_lde_without_shift_contains_the_input():
    n, cols, b = 32, 4, 3
    evals = pg_synth.matrix(0x4E5C, n, cols)
    got = oracle.lde_columns(evals, b, shift=1)
    assert (got[:: 1 << b] == evals).all()
    assert (oracle.lde_columns(evals, 0, shift=1) == evals).all()
