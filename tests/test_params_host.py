"""Host-side parts of the CUDA library, checked on the CPU (no GPU needed).

The library builds parameter set pg12_v1 with its own Grain-LFSR code and
derives the sparse optimised form of Alg. 1 from it.  Here the plain set is
compared with the oracle's independent generator, and the optimised form is
evaluated with Python integers (round structure of Alg. 1: MDSPartial with
vec[0] = first row, vec[1] = first column) against the oracle's plain
permutation.
"""
import os

import numpy as np
import pytest

import oracle
import pg_synth

pg = pytest.importorskip("paper_2506_09505_gb300")

P = 0xFFFFFFFF00000001


@pytest.fixture(scope="module")
def lib():
    try:
        return pg.load(build_if_missing=True)
    except Exception as e:  # pragma: no cover - toolchain missing
        pytest.skip(f"library unavailable: {e}")


def test_plain_params_match_oracle(lib):
    rc, mds = pg.params_export()
    orc_rc, orc_mds = oracle.params()[:2]
    assert (rc == orc_rc).all()
    assert (mds == orc_mds).all()


def _opt_permute(x, op):
    x = [int(v) % P for v in x]
    fr, M, pre = op["full_rc"], op["mds"], op["pre"]
    def full(x, r, mat):
        y = [pow((x[i] + int(fr[r, i])) % P, 7, P) for i in range(12)]
        return [sum(int(mat[i, j]) * y[j] for j in range(12)) % P for i in range(12)]
    for r in range(3):
        x = full(x, r, M)
    x = full(x, 3, pre)
    for q in range(22):
        x0 = pow((x[0] + int(op["part_rc"][q])) % P, 7, P)
        v, w = op["part_v"][q], op["part_w"][q]
        new0 = (int(v[0]) * x0 + sum(int(v[j]) * x[j] for j in range(1, 12))) % P
        x = [new0] + [(x[i] + int(w[i - 1]) * x0) % P for i in range(1, 12)]
    for r in range(4, 8):
        x = full(x, r, M)
    return x


def test_optimised_form_equals_plain_permutation(lib):
    op = pg.params_export_optimized()
    st = pg_synth.matrix(0xAB, 40, 12)
    want = oracle.permute(st)
    for k in range(st.shape[0]):
        assert _opt_permute(st[k], op) == [int(v) for v in want[k]]


def _opt_compress(x8, op):
    """The library's shortcut for a state [x8, 0, 0, 0, 0] whose digest is all
    that is read: round 0 takes the capacity cells' share of each dense row as
    one constant (their S-box inputs are the round constants alone), and the
    last dense layer computes rows 0..3 only."""
    fr, M, pre = op["full_rc"], op["mds"], op["pre"]
    k = [sum(int(M[i, j]) * pow(int(fr[0, j]), 7, P) for j in range(8, 12)) % P for i in range(12)]
    y = [pow((int(x8[j]) + int(fr[0, j])) % P, 7, P) for j in range(8)]
    x = [(k[i] + sum(int(M[i, j]) * y[j] for j in range(8))) % P for i in range(12)]

    def full(x, r, mat, rows=12):
        y = [pow((x[i] + int(fr[r, i])) % P, 7, P) for i in range(12)]
        return [sum(int(mat[i, j]) * y[j] for j in range(12)) % P for i in range(rows)]
    for r in (1, 2):
        x = full(x, r, M)
    x = full(x, 3, pre)
    for q in range(22):
        x0 = pow((x[0] + int(op["part_rc"][q])) % P, 7, P)
        v, w = op["part_v"][q], op["part_w"][q]
        new0 = (int(v[0]) * x0 + sum(int(v[j]) * x[j] for j in range(1, 12))) % P
        x = [new0] + [(x[i] + int(w[i - 1]) * x0) % P for i in range(1, 12)]
    for r in (4, 5, 6):
        x = full(x, r, M)
    return full(x, 7, M, rows=4)


def test_zero_capacity_digest_shortcut_equals_plain_permutation(lib):
    # node compressions and single-chunk leaves: [8 words, 0^4] -> first 4 words
    op = pg.params_export_optimized()
    st = pg_synth.matrix(0xAC, 24, 12, bound=None)
    st[:, 8:] = 0
    want = oracle.permute(st)
    for k in range(st.shape[0]):
        assert _opt_compress(st[k, :8], op) == [int(v) for v in want[k, :4]]
    left, right = pg_synth.matrix(0xAD, 1, 4)[0], pg_synth.matrix(0xAE, 1, 4)[0]
    node = oracle.hash_pair(left, right)
    assert _opt_compress(np.concatenate([left, right]), op) == [int(v) for v in node]


def test_optimised_constants_canonical(lib):
    op = pg.params_export_optimized()
    for name, a in op.items():
        assert (a < np.uint64(P)).all(), name
    # the dense full-round matrix is the plain MDS matrix
    assert (op["mds"] == oracle.params()[1]).all()


def test_small_set_matches_oracle_and_optimised_form(lib):
    try:
        pg.params_select("pg12_small")
        assert pg.params_name() == "pg12_small"
        rc, mds = pg.params_export()
        orc_rc, orc_mds, row, _ = oracle.params_small()
        assert (rc == orc_rc).all() and (mds == orc_mds).all()
        # circulant with 8-bit entries
        for i in range(12):
            for j in range(12):
                assert int(mds[i, j]) == int(row[(j - i) % 12]) and 1 <= int(mds[i, j]) <= 255
        op = pg.params_export_optimized()
        st = pg_synth.matrix(0xAC, 16, 12)
        want = oracle.permute(st, orc_rc, orc_mds)
        for k in range(st.shape[0]):
            assert _opt_permute(st[k], op) == [int(v) for v in want[k]]
    finally:
        pg.params_select(None)
    assert pg.params_name() == "pg12_v1"


def test_unknown_set_rejected(lib):
    with pytest.raises(pg.PGError) as e:
        pg.params_select("nope")
    assert e.value.status == 6


def _golden_sha():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pg12_v1.sha256")
    with open(path) as f:
        return dict(line.split() for line in f if line.strip())["sha256"]


def test_library_sha256_matches_golden_and_hashlib():
    import hashlib
    lib = pytest.importorskip("paper_2506_09505_gb300")
    lib.load(build_if_missing=True)
    lib.params_select(None)
    assert lib.params_sha256() == _golden_sha()
    for name in ("pg12_small", None):
        lib.params_select(name)
        rc, mds = lib.params_export()
        h = hashlib.sha256(np.ascontiguousarray(rc, dtype="<u8").tobytes() +
                           np.ascontiguousarray(mds, dtype="<u8").tobytes()).hexdigest()
        assert lib.params_sha256() == h
    assert lib.params_sha256() == _golden_sha()


def test_workspace_bytes_counts_plans_and_counters():
    import ctypes
    lib = pytest.importorskip("paper_2506_09505_gb300")
    raw = lib.load(build_if_missing=True)
    total = raw.pg_workspace_bytes(None, 0)
    assert total == 32 << 20
    sizes = [(1, 8), (32, 8), (64, 3), (1 << 12, 16), (1 << 20, 8)]
    arr = (lib.Tree * len(sizes))()
    for k, (n, w) in enumerate(sizes):
        arr[k].rows, arr[k].n_leaves, arr[k].width, arr[k].nodes = 0x1000, n, w, 0x2000

    def counters(n):
        # one arrival counter per 32-node group of each level whose children span more than one group
        c, lvl = 0, 1
        while (n >> lvl) >= 1 and lvl <= n.bit_length() - 1:
            if (n >> (lvl - 1)) > 32:
                c += ((n >> lvl) + 31) // 32
            lvl += 1
        return c
    want = (4 << 20) + 4 * (1 + sum(counters(n) for n, _ in sizes))
    assert raw.pg_workspace_bytes(arr, len(sizes)) == want
    arr[2].n_leaves = 48
    assert raw.pg_workspace_bytes(arr, len(sizes)) == 0
