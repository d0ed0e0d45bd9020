"""CPU pins of the tensor-core forms: the digit tables and the unrolled partial rounds.

The tensor-core kernels compute each dense contraction (the full rounds'
M y, Alg. 1; the partial rounds' dot products U = (V' P) y3 and deferred
updates W s, their unrolled form) for 128 states at a time as an fp32
contraction of byte limbs (the digit tables of pg_tc_tables_export).  These
tests take the exported tables and redo, with Python integers, exactly what
the tensor cores and the combination step compute -- bytes of the operand
words times the decoded fp16 digits, plus the bias block, as fp32 bit
patterns, then sum_b 2^(8b) bits mod p -- and require the plain
matrix-vector products mod p, for both parameter sets, on random and extreme
inputs.  They check every bound the exactness argument needs (digits in
[-128, 127]; every fp32 sum an integer in [2^23, 2^24) for any input bytes,
including the final updates that accumulate two tables) and that the bias
offsets cancel mod p.  And they evaluate the whole permutation in the
unrolled form (pg_params_export_chain) against the oracle's plain Alg. 1.
"""
import numpy as np
import pytest

import oracle
import pg_synth

pg = pytest.importorskip("paper_2506_09505_gb300")

P = 0xFFFFFFFF00000001
T = 12
RP = 22
SPLIT = 11  # the chain's first half: s_0 .. s_10
TABLES = [("m", 12, 12), ("pre", 12, 12), ("b_bias", None, None), ("a_bias", None, None), ("a_zcap", None, None),
          ("vpa", 10, 12), ("vpb", 12, 12), ("bs", 12, 12), ("w1", 12, 12), ("w2", 12, 12)]


def half_to_float(h: int) -> float:
    return float(np.array([h], dtype=np.uint16).view(np.float16)[0])


def tables(params=None):
    pg.load(build_if_missing=True)
    pg.params_select(params)
    h = np.frombuffer(pg.tc_tables_export(), dtype=np.uint16)
    out, off = {}, 0
    for name, n, k in TABLES:
        # a table: 8n rows x 8k columns; the bias blocks two core matrices, zcap four
        size = (8 * n) * (8 * k) if n else (256 if name == "a_zcap" else 128)
        out[name] = h[off:off + size]
        off += size
    assert off == h.size
    return out


def decode(tab, n, k):
    """digits[i][b][j][a] of an n x k table (K-major core matrices, k chunks per row group)."""
    dig = np.zeros((n, 8, k, 8), dtype=np.int64)
    for row in range(8 * n):
        i, b = divmod(row, 8)
        for j in range(k):
            base = (row // 8 * k + j) * 64 + (row % 8) * 8
            for a in range(8):
                v = half_to_float(int(tab[base + a]))
                assert v == int(v)
                dig[i, b, j, a] = int(v)
    return dig


def bias_magic(t):
    """magic_b (integers, scaled by 2^24) from the bias blocks."""
    a = half_to_float(int(t["a_bias"][0]))
    assert a == 2.0 ** -13
    for r in range(8):
        for k in range(16):
            assert int(t["a_bias"][(k // 8) * 64 + r * 8 + k % 8]) == (0x0800 if k == 0 else 0)
    mags = []
    for b in range(8):
        for k in range(16):
            if k:
                assert int(t["b_bias"][(k // 8) * 64 + b * 8 + k % 8]) == 0
        mags.append(int(round(half_to_float(int(t["b_bias"][b * 8])) * a * 2 ** 24)))
    return mags


def contract(digs, magic, words_list):
    """What the kernels compute: sum over the tables (one accumulator) of bytes x digits, plus the bias."""
    n = digs[0].shape[0]
    out = []
    for i in range(n):
        acc = 0
        for bb in range(8):
            z = 0
            for dig, words in zip(digs, words_list):
                xb = np.array([[(int(v) >> (8 * a)) & 0xFF for a in range(8)] for v in words], dtype=np.int64)
                z += int((dig[i, bb] * xb).sum())
            v = magic[bb] + z
            assert (1 << 23) <= v < (1 << 24), "fp32 sum outside [2^23, 2^24): not exact"
            acc += (0x3F000000 + (v - (1 << 23))) << (8 * bb)  # fp32 bits of v * 2^-24
        out.append(acc % P)
    return out


def plain(mat, words):
    return [sum(int(mat[i][j]) * (int(words[j]) % P) for j in range(len(words))) % P for i in range(len(mat))]


def worst_window(digs, magic):
    """Every column's extreme sums over all byte inputs stay in the exact window."""
    for i in range(digs[0].shape[0]):
        for bb in range(8):
            pos = sum(int(d[i, bb][d[i, bb] > 0].sum()) for d in digs)
            neg = sum(int(-d[i, bb][d[i, bb] < 0].sum()) for d in digs)
            assert magic[bb] - 255 * neg >= 1 << 23 and magic[bb] + 255 * pos < 1 << 24


def _inputs(k, seed):
    xs = [pg_synth.words(seed + t, k, bound=None) for t in range(4)]
    xs.append(np.full(k, (1 << 64) - 1, dtype=np.uint64))   # every byte 255
    xs.append(np.zeros(k, dtype=np.uint64))
    xs.append(np.full(k, P - 1, dtype=np.uint64))
    return xs


@pytest.mark.parametrize("params", [None, "pg12_small"])
def test_digit_tables_reproduce_every_contraction(params):
    t = tables(params)
    opt = pg.params_export_optimized()
    vp, beta, w = pg.params_export_chain()
    magic = bias_magic(t)
    cases = [("m", opt["mds"], 12), ("pre", opt["pre"], 12), ("vpa", vp[:SPLIT - 1], 12)]
    for name, mat, k in cases:
        dig = decode(t[name], len(mat), k)
        assert dig.min() >= -128 and dig.max() <= 127
        worst_window([dig], magic)
        for x in _inputs(k, 0x7C00):
            assert contract([dig], magic, [x]) == plain(mat, x), name
    # input word 11 of bs, w1 and w2 meets a stale A column: its digits are zero
    stale = pg_synth.words(0x7E00, 1, bound=None)
    # the second half's chain values: U_q (q = 10 .. 21) from y3 plus, in the
    # same accumulator, beta[q][r] s_r for the first half's r = 0 .. 10 (row 21: none)
    bmat = [[int(beta[q, r]) if (q < 21 and r < SPLIT) else 0 for r in range(12)] for q in range(SPLIT - 1, 22)]
    dv, db = decode(t["vpb"], 12, 12), decode(t["bs"], 12, 12)
    worst_window([dv, db], magic)
    for y3, s in zip(_inputs(12, 0x7D00), _inputs(12, 0x7D80)):
        s = np.concatenate([s[:SPLIT], stale])
        want = [(a + b) % P for a, b in zip(plain(vp[SPLIT - 1:], y3), plain(bmat, s[:SPLIT]))]
        assert contract([dv, db], magic, [y3, s]) == want
    # the final updates: s_0 .. s_10 and s_11 .. s_21 into one accumulator
    d1, d2 = decode(t["w1"], 12, 12), decode(t["w2"], 12, 12)
    worst_window([d1, d2], magic)
    for s in _inputs(22, 0x7D00):
        s1 = np.concatenate([s[:SPLIT], stale])
        s2 = np.concatenate([s[SPLIT:], stale])
        assert contract([d1, d2], magic, [s1, s2]) == plain(w, s)
    pg.params_select(None)


def test_bias_offsets_cancel_mod_p():
    magic = bias_magic(tables(None))
    assert sum((0x3E800000 + mg) << (8 * bb) for bb, mg in enumerate(magic)) % P == 0


def test_zero_capacity_pattern_is_the_constant_sbox_outputs():
    t = tables(None)
    opt = pg.params_export_optimized()
    for j in range(8, 12):
        c7 = pow(int(opt["full_rc"][0][j]) % P, 7, P)
        for r in range(8):
            got = sum(int(t["a_zcap"][(j - 8) * 64 + r * 8 + a]) << (8 * a) for a in range(8))
            assert got == c7


def _chain_permute(x, op, vp, beta, w, split=None):
    """Alg. 1 with the partial rounds in their unrolled form (Python integers).

    split: the chain in two halves as the kernels run it -- the first half's
    terms beta[q][r] s_r (r < split) of the later chain values are added to
    U_q in one step after s_(split-1), the rest as the chain goes."""
    x = [int(v) % P for v in x]
    fr, M, pre = op["full_rc"], op["mds"], op["pre"]

    def sbox_layer(x, r):
        return [pow((x[i] + int(fr[r, i])) % P, 7, P) for i in range(12)]

    def dense(mat, y):
        return [sum(int(mat[i, j]) * y[j] for j in range(12)) % P for i in range(12)]
    for r in range(3):
        x = dense(M, sbox_layer(x, r))
    y3 = sbox_layer(x, 3)
    x0 = dense(pre, y3)
    u = [sum(int(vp[q, j]) * y3[j] for j in range(12)) % P for q in range(RP)]
    c, s = x0[0], []
    for q in range(RP):
        s.append(pow((c + int(op["part_rc"][q])) % P, 7, P))
        if split is not None and q == split - 1:
            u = u[:split - 1] + [(u[p] + sum(int(beta[p, r]) * s[r] for r in range(split))) % P
                                 for p in range(split - 1, RP - 1)] + [u[RP - 1]]
        if q < RP - 1:
            lo = split if (split is not None and q >= split - 1) else 0
            c = (u[q] + sum(int(beta[q, r]) * s[r] for r in range(lo, q + 1))) % P
    ws = [sum(int(w[i, r]) * s[r] for r in range(RP)) % P for i in range(12)]
    x = [(u[RP - 1] + ws[0]) % P] + [(x0[i] + ws[i]) % P for i in range(1, 12)]
    for r in range(4, 8):
        x = dense(M, sbox_layer(x, r))
    return x


@pytest.mark.parametrize("params", [None, "pg12_small"])
def test_unrolled_partial_rounds_equal_the_plain_permutation(params):
    pg.load(build_if_missing=True)
    pg.params_select(params)
    try:
        op = pg.params_export_optimized()
        vp, beta, w = pg.params_export_chain()
        rc, mds = (oracle.params() if params is None else oracle.params_small())[:2]
        st = pg_synth.matrix(0xCA1 + (params is not None), 24, 12)
        st[0] = 0
        st[1] = np.uint64((1 << 64) - 1)
        want = oracle.permute(st, rc=rc, mds=mds)
        for k in range(st.shape[0]):
            assert _chain_permute(st[k], op, vp, beta, w) == [int(v) for v in want[k]]
            assert _chain_permute(st[k], op, vp, beta, w, split=SPLIT) == [int(v) for v in want[k]]
    finally:
        pg.params_select(None)
