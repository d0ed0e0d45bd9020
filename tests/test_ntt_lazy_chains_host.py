"""Host model of the NTT kernel's lazy sums (csrc/ntt.cu, struct Lz).

The radix-8 steps keep their sums as l0 + l1 2^32 + t 2^64 (t a signed
32-bit word) and reduce once per output; the 8-point DFTs' twiddles are the
shifts 2^24, 2^48 and 2^72 (mod p = 2^64 - 2^32 + 1).  This file restates each
of those PTX carry chains on 32-bit words with an explicit carry flag
(add.cc / addc write and read the carry; sub.cc / subc the borrow) and checks,
on random and extreme words, that every chain gives the exact value mod p and
that the ranges the kernel relies on hold: the top word of the 96-bit value
handed to the final correction is -1, 0 or 1, and that correction never
wraps.  The GPU parity tests check the kernel itself; this pins the arithmetic
the kernel was written from.
"""
import random

P = 2**64 - 2**32 + 1
M = 0xFFFFFFFF


class Carry:
    def __init__(self):
        self.cf = 0

    def add_cc(self, a, b):
        r = a + b
        self.cf = r >> 32
        return r & M

    def addc_cc(self, a, b):
        r = a + b + self.cf
        self.cf = r >> 32
        return r & M

    def addc(self, a, b):
        return (a + b + self.cf) & M

    def sub_cc(self, a, b):
        r = a - b
        self.cf = 1 if r < 0 else 0
        return r & M

    def subc_cc(self, a, b):
        r = a - b - self.cf
        self.cf = 1 if r < 0 else 0
        return r & M

    def subc(self, a, b):
        return (a - b - self.cf) & M


def s32(x):
    x &= M
    return x - (1 << 32) if x >> 31 else x


def sar(x, n):
    return (s32(x) >> n) & M


def value(a):
    l0, l1, t = a
    return l0 + (l1 << 32) + s32(t) * 2**64


def lz(w):
    return (w & M, w >> 32, 0)


def lz_add(a, b):
    c = Carry()
    return c.add_cc(a[0], b[0]), c.addc_cc(a[1], b[1]), c.addc(a[2], b[2])


def lz_sub(a, b):
    c = Carry()
    return c.sub_cc(a[0], b[0]), c.subc_cc(a[1], b[1]), c.subc(a[2], b[2])


def fix_top(w0, w1, tp):
    """(w1:w0) + tp (2^32 - 1); asserts the preconditions the kernel relies on."""
    assert s32(tp) in (-1, 0, 1)
    exact = w0 + (w1 << 32) + s32(tp) * (2**32 - 1)
    assert 0 <= exact < 2**64
    c = Carry()
    r0 = c.sub_cc(w0, tp)
    r1 = c.subc(w1, sar(tp, 31))
    r1 = (r1 + tp) & M
    assert r0 + (r1 << 32) == exact
    return exact


def lz_reduce(a):
    l0, l1, t = a
    sh = sar(t, 31)
    c = Carry()
    w1 = c.add_cc(l1, t)
    w2 = c.addc(sh, 0)
    c = Carry()
    w0 = c.sub_cc(l0, t)
    w1 = c.subc_cc(w1, sh)
    w2 = c.subc(w2, sh)
    return fix_top(w0, w1, w2)


def lz_m24(a):
    l0, l1, t = a
    assert -2**7 < s32(t) < 2**7
    return (l0 << 24) & M, ((l1 << 24) | (l0 >> 8)) & M, ((t << 24) + (l1 >> 8)) & M


def lz_m48(a):
    l0, l1, t = a
    big1 = (l0 << 16) & M
    hl, hh = ((l1 << 16) | (l0 >> 16)) & M, l1 >> 16
    e0, e1, e2 = (t << 16) & M, sar(t, 16), sar(t, 31)
    c = Carry()
    w0 = c.sub_cc(0, e0)
    w1 = c.subc_cc(big1, e1)
    tp = c.subc(0, e2)
    c = Carry()
    w0 = c.sub_cc(w0, hl)
    w1 = c.subc_cc(w1, 0)
    tp = c.subc(tp, 0)
    c = Carry()
    w0 = c.sub_cc(w0, hh)
    w1 = c.subc_cc(w1, 0)
    tp = c.subc(tp, 0)
    c = Carry()
    w1 = c.add_cc(w1, hl)
    tp = c.addc(tp, 0)
    return fix_top(w0, w1, tp)


def lz_m72(a):
    l0, l1, t = a
    assert -2**23 < s32(t) < 2**23
    hl, hh, k = (l0 << 8) & M, ((l1 << 8) | (l0 >> 24)) & M, l1 >> 24
    e1, e2 = (t << 8) & M, sar(t, 31)
    c = Carry()
    w0 = c.sub_cc(0, hl)
    w1 = c.subc_cc(0, k)
    tp = c.subc(0, 0)
    c = Carry()
    w0 = c.sub_cc(w0, hh)
    w1 = c.subc_cc(w1, 0)
    tp = c.subc(tp, 0)
    c = Carry()
    w1 = c.add_cc(w1, hl)
    tp = c.addc(tp, 0)
    c = Carry()
    w1 = c.sub_cc(w1, e1)
    tp = c.subc(tp, e2)
    return fix_top(w0, w1, tp)


EDGE = [0, 1, 2, P - 1, P, P + 1, 2**64 - 1, 2**64 - 2, 2**63, 2**32 - 1, 2**32, 0xFFFFFFFF00000000,
        0xFFFF, 0xFFFF0000FFFF0000]


def words(rng, n):
    return [rng.choice(EDGE) if rng.random() < 0.4 else rng.getrandbits(64) for _ in range(n)]


def test_roots_are_the_shift_twiddles():
    # w_k = 7^((p - 1) / 2^k): w_2 = 2^48, w_3 = -2^24, w_3^2 = 2^48, w_3^3 = -2^72
    w2, w3 = pow(7, (P - 1) >> 2, P), pow(7, (P - 1) >> 3, P)
    assert w2 == pow(2, 48, P)
    assert w3 == (-pow(2, 24, P)) % P
    assert w3 * w3 % P == pow(2, 48, P)
    assert pow(w3, 3, P) == (-pow(2, 72, P)) % P


def test_lazy_sums_and_shift_products():
    rng = random.Random(20260512)
    for _ in range(20000):
        a, b, c, d = words(rng, 4)
        s = lz_add(lz(a), lz(b))
        assert value(s) == a + b
        e = lz_sub(lz(c), lz(d))
        assert value(e) == c - d
        mixed = [s, e, lz_add(s, e), lz_sub(s, e), lz_sub(lz_sub(s, e), lz_add(s, s))]
        for x in mixed:
            v = value(x)
            assert lz_reduce(x) % P == v % P
            assert lz_m48(x) % P == v * 2**48 % P
            assert lz_m72(x) % P == v * 2**72 % P
            y = lz_m24(x)
            assert value(y) % P == v * 2**24 % P
            # values with the large top word a 2^24 shift leaves, summed again
            z = lz_add(y, lz_add(y, s))
            assert lz_reduce(z) % P == value(z) % P
            assert lz_m48(z) % P == value(z) * 2**48 % P
