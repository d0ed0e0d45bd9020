"""CPU pins of the tensor-core form of the full rounds' dense layers.

The library's tensor-core kernels compute y = M x (Alg. 1, MDS) for 128
states at a time as an fp32 contraction of byte limbs (the digit tables of
pg_tc_tables_export).  These tests take the exported tables and redo, with
Python integers, exactly what the tensor cores and the combination step
compute -- bytes of x times the decoded fp16 digits, plus the bias row, as
fp32 bit patterns, then sum_b 2^(8b) bits mod p -- and require the result to
equal the plain matrix-vector product mod p, for both parameter sets and
both matrices (M, and the transition matrix of round 3), on random and
extreme inputs.  They also check every bound the exactness argument needs:
digits in [-128, 127], every fp32 sum an integer in [2^23, 2^24) for any
input bytes, and the bias offsets cancelling mod p.
"""
import numpy as np
import pytest

import pg_synth

pg = pytest.importorskip("paper_2506_09505_gb300")

P = 0xFFFFFFFF00000001
T = 12
KC = 14


def half_to_float(h: int) -> float:
    return float(np.array([h], dtype=np.uint16).view(np.float16)[0])


def tables(params=None):
    pg.load(build_if_missing=True)
    pg.params_select(params)
    raw = pg.tc_tables_export()
    h = np.frombuffer(raw, dtype=np.uint16)
    nb = 96 * KC * 8
    b = h[:2 * nb].reshape(2, nb)
    a_bias = h[2 * nb:2 * nb + 128]
    a_zcap = h[2 * nb + 128:2 * nb + 128 + 256]
    return b, a_bias, a_zcap


def b_entry(bt, n, k):
    """B operand value at output column n, K column k (K-major core matrices)."""
    c, a = divmod(k, 8)
    return half_to_float(int(bt[(n // 8 * KC + c) * 64 + (n % 8) * 8 + a]))


def decode(bt):
    """digits[i][b][j][a] (integers) and bias value per output column."""
    dig = np.zeros((T, 8, T, 8), dtype=np.int64)
    bias = np.zeros(96)
    for n in range(96):
        i, bb = divmod(n, 8)
        for k in range(96):
            j, a = divmod(k, 8)
            v = b_entry(bt, n, k)
            assert v == int(v)
            dig[i, bb, j, a] = int(v)
        bias[n] = b_entry(bt, n, 96)
        for k in range(97, 112):
            assert b_entry(bt, n, k) == 0.0
    return dig, bias


def dense_via_tables(dig, bias_prod, x):
    """What the kernels compute for one state x (12 weak words)."""
    xb = np.array([[(int(v) >> (8 * a)) & 0xFF for a in range(8)] for v in x], dtype=np.int64)
    out = []
    for i in range(T):
        acc = 0
        for bb in range(8):
            z = int((dig[i, bb] * xb).sum())
            magic = int(round(bias_prod[8 * i + bb] * 2**24))
            v = magic + z
            assert (1 << 23) <= v < (1 << 24), "fp32 sum outside [2^23, 2^24): not exact"
            bits = 0x3F000000 + (v - (1 << 23))  # fp32 bits of v * 2^-24 in [0.5, 1)
            acc += bits << (8 * bb)
        out.append(acc % P)
    return out


def plain_dense(m, x):
    return [sum(int(m[i][j]) * (int(x[j]) % P) for j in range(T)) % P for i in range(T)]


@pytest.mark.parametrize("params", [None, "pg12_small"])
def test_digit_tables_reproduce_the_dense_layers(params):
    b, a_bias, a_zcap = tables(params)
    opt = pg.params_export_optimized()
    a_scale = half_to_float(int(a_bias[0]))
    assert a_scale == 2.0**-13
    # the bias A operand is 2^-13 at column 0 of every row of both core matrices, else 0
    for r in range(8):
        for k in range(16):
            want = 0x0800 if k == 0 else 0
            assert int(a_bias[(k // 8) * 64 + r * 8 + k % 8]) == want
    xs = [pg_synth.words(0x7C00 + k, T, bound=None) for k in range(6)]
    xs.append(np.full(T, (1 << 64) - 1, dtype=np.uint64))   # every byte 255
    xs.append(np.zeros(T, dtype=np.uint64))
    xs.append(np.full(T, P - 1, dtype=np.uint64))
    for m, mat in ((0, opt["mds"]), (1, opt["pre"])):
        dig, bias = decode(b[m])
        assert dig.min() >= -128 and dig.max() <= 127
        # worst-case |Z| over all byte inputs stays inside the exact window
        zmax = int(np.abs(dig).sum(axis=(2, 3)).max()) * 255
        magic = bias * a_scale * 2**24
        assert (magic - zmax >= 2**23).all() and (magic + zmax < 2**24).all()
        for x in xs:
            assert dense_via_tables(dig, bias * a_scale, x) == plain_dense(mat, x)
    pg.params_select(None)


def test_bias_offsets_cancel_mod_p():
    b, a_bias, _ = tables(None)
    _, bias = decode(b[0])
    magic = [int(round(v * 2.0**-13 * 2**24)) for v in bias[:8]]
    assert sum((0x3E800000 + mg) << (8 * bb) for bb, mg in enumerate(magic)) % P == 0
    for i in range(1, T):   # every output row uses the same eight biases
        assert list(bias[8 * i:8 * i + 8]) == list(bias[:8])


def test_zero_capacity_pattern_is_the_constant_sbox_outputs():
    _, _, a_zcap = tables(None)
    opt = pg.params_export_optimized()
    for j in range(8, 12):
        c7 = pow(int(opt["full_rc"][0][j]) % P, 7, P)
        for r in range(8):
            got = sum(int(a_zcap[(j - 8) * 64 + r * 8 + a]) << (8 * a) for a in range(8))
            assert got == c7
