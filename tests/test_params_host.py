"""Host-side parts of the CUDA library, checked on the CPU (no GPU needed).

The library builds parameter set pg12_v1 with its own Grain-LFSR code and
derives the sparse optimised form of Alg. 1 from it.  Here the plain set is
compared with the oracle's independent generator, and the optimised form is
evaluated with Python integers (round structure of Alg. 1: MDSPartial with
vec[0] = first row, vec[1] = first column) against the oracle's plain
permutation.
"""
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
