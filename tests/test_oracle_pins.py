"""Pins of the CPU oracle to facts outside itself (no GPU).

Each check ties an oracle function to something the paper or mathematics
fixes independently of the oracle's own code: Python big-integer arithmetic,
closed forms (Cauchy determinants, Fermat), special parameter sets whose
permutation collapses to scalar recurrences written here from the round
structure of Alg. 1 / Sec. 2.4, brute force, and structural invariants of
the sponge and the Merkle tree (Sec. 2.4, Sec. 4.2).
"""
import random

import numpy as np
import pytest

import oracle
import pg_synth

P = (1 << 64) - (1 << 32) + 1  # Eq. 1
EPS = (1 << 32) - 1
EDGE = [0, 1, 2, EPS - 1, EPS, EPS + 1, 1 << 32, (1 << 32) + 1, 1 << 63, (1 << 63) + 1,
        P - 2, P - 1, P, P + 1, (1 << 64) - 2, (1 << 64) - 1, 0x1234567890ABCDEF]


# ------------------------------------------------------------------ field

def test_prime_value():
    assert P == 0xFFFFFFFF00000001
    assert oracle.P == P
    # p - 1 = 2^32 * 3 * 5 * 17 * 257 * 65537, so gcd(7, p - 1) = 1 (x^7 is a bijection)
    assert P - 1 == (1 << 32) * 3 * 5 * 17 * 257 * 65537


def test_field_ops_edge_values_vs_bigint():
    for a in EDGE:
        assert oracle.canon(a) == a % P
        for b in EDGE:
            assert oracle.add(a, b) == (a + b) % P
            assert oracle.sub(a, b) == (a - b) % P
            assert oracle.mul(a, b) == (a * b) % P


def test_field_ops_random_vs_bigint():
    rng = random.Random(1234)
    for _ in range(20000):
        a, b = rng.getrandbits(64), rng.getrandbits(64)
        assert oracle.mul(a, b) == (a * b) % P
        assert oracle.add(a, b) == (a + b) % P
        assert oracle.sub(a, b) == (a - b) % P


@pytest.mark.parametrize("op,fn", [
    ("add", lambda a, b: (a + b) % P),
    ("sub", lambda a, b: (a - b) % P),
    ("mul", lambda a, b: (a * b) % P),
    ("sqr", lambda a, b: (a * a) % P),
    ("sbox", lambda a, b: pow(a, 7, P)),
])
def test_field_many_vs_bigint(op, fn):
    # the element-wise entry point that the GPU field tests compare against
    e = np.array(EDGE, dtype=np.uint64)
    a = np.concatenate([np.repeat(e, len(e)), pg_synth.words(0xA11, 4000, bound=None)])
    b = np.concatenate([np.tile(e, len(e)), pg_synth.words(0xA12, 4000, bound=None)])
    got = oracle.field_many(op, a, b)
    assert [int(v) for v in got] == [fn(int(x), int(y)) for x, y in zip(a, b)]


def test_limb_identities():
    # the special-prime identities behind Alg. 2 / Eqs. 2-4
    assert oracle.pow_(2, 64) == EPS
    assert oracle.pow_(2, 96) == P - 1
    assert oracle.pow_(2, 128) == (P - (1 << 32)) % P
    assert oracle.pow_(2, 192) == 1


def test_inverse_and_fermat():
    rng = random.Random(7)
    for _ in range(200):
        a = rng.randrange(1, P)
        assert oracle.mul(a, oracle.inv(a)) == 1
        assert oracle.pow_(a, P - 1) == 1
        assert oracle.pow_(a, 5) == pow(a, 5, P)


def test_sbox_inverse_exponent():
    d = oracle.sbox_inverse_exponent()
    assert (7 * d) % (P - 1) == 1
    rng = random.Random(3)
    for _ in range(100):
        x = rng.randrange(P)
        assert oracle.pow_(oracle.pow_(x, 7), d) == x


def test_sbox_no_collisions_sample():
    xs = pg_synth.words(99, 1 << 14)
    ys = {pow(int(x), 7, P) for x in xs}
    assert len(ys) == len(set(int(x) for x in xs))


# ------------------------------------------------------------ parameters

def test_params_deterministic_and_canonical():
    rc, mds, xs, ys, redraws = oracle.params()
    assert rc.shape == (30, 12) and mds.shape == (12, 12)
    assert all(int(v) < P for v in rc.ravel())
    assert all(int(v) < P for v in mds.ravel())
    rc2 = np.zeros((30, 12), dtype=np.uint64)
    # a second, independent generation gives the same words
    lib = oracle._load()
    mds2 = np.zeros((12, 12), dtype=np.uint64)
    lib.orc_params_generate(oracle._ptr(rc2), oracle._ptr(mds2), None, None)
    assert (rc2 == rc).all() and (mds2 == mds).all()
    assert redraws >= 0


def test_cauchy_structure_against_points():
    _, mds, xs, ys, _ = oracle.params()
    pts = [int(v) for v in xs] + [int(v) for v in ys]
    assert len(set(pts)) == 24
    for i in range(12):
        for j in range(12):
            s = (int(xs[i]) + int(ys[j])) % P
            assert s != 0
            assert (int(mds[i, j]) * s) % P == 1


def test_cauchy_determinant_closed_form():
    # det of a Cauchy matrix 1/(x_i + y_j):
    #   prod_{i<j} (x_j - x_i)(y_j - y_i) / prod_{i,j} (x_i + y_j)
    _, mds, xs, ys, _ = oracle.params()
    x = [int(v) for v in xs]
    y = [int(v) for v in ys]
    for k in (2, 5, 12):
        num, den = 1, 1
        for i in range(k):
            for j in range(i + 1, k):
                num = num * (x[j] - x[i]) * (y[j] - y[i]) % P
        for i in range(k):
            for j in range(k):
                den = den * (x[i] + y[j]) % P
        want = num * pow(den, P - 2, P) % P
        assert oracle.mat_det(mds[:k, :k]) == want


def test_grain_lfsr_against_recurrence():
    # The raw 1-bit words of the generator follow the published shrinking
    # rule applied to b_{i+80} = b_{i+62}+b_{i+51}+b_{i+38}+b_{i+23}+b_{i+13}+b_i
    # (mod 2); rebuild the same stream here from the seed bits.
    bits = []
    for v, n in ((1, 2), (0, 4), (64, 12), (12, 12), (8, 10), (22, 10), ((1 << 30) - 1, 30)):
        bits += [(v >> k) & 1 for k in range(n - 1, -1, -1)]
    assert len(bits) == 80

    def clock():
        nb = bits[62] ^ bits[51] ^ bits[38] ^ bits[23] ^ bits[13] ^ bits[0]
        bits.pop(0)
        bits.append(nb)
        return nb

    for _ in range(160):
        clock()
    want = []
    while len(want) < 256:
        a, b = clock(), clock()
        if a:
            want.append(b)
    got = oracle.grain_words(1, 0, 64, 12, 8, 22, 1, 256)
    assert [int(v) for v in got] == want
    # 64-bit words are the same bits read big-endian
    w64 = oracle.grain_words(1, 0, 64, 12, 8, 22, 64, 4)
    for k in range(4):
        assert int(w64[k]) == int("".join(str(b) for b in want[64 * k:64 * k + 64]), 2)


def test_first_round_constants_are_first_grain_words():
    # with rejection of words >= p (probability ~2^-32 each) the first
    # constants are the first 64-bit words of the stream
    rc = oracle.params()[0]
    w = oracle.grain_words(1, 0, 64, 12, 8, 22, 64, 8)
    good = [int(v) for v in w if int(v) < P]
    assert [int(v) for v in rc.ravel()[:len(good[:6])]] == good[:6]


@pytest.mark.slow
def test_mds_property_all_minors():
    # MDS <=> every square submatrix is nonsingular: C(24,12) - 1 minors
    _, mds, _, _, _ = oracle.params()
    bad, checked = oracle.count_singular_minors(mds)
    assert checked == 2704155
    assert bad == 0


def test_minor_checker_detects_singular():
    m = np.arange(1, 145, dtype=np.uint64).reshape(12, 12)  # rank 2: many singular minors
    bad, checked = oracle.count_singular_minors(m)
    assert checked == 2704155 and bad > 0


def test_matrix_inverse():
    _, mds, _, _, _ = oracle.params()
    inv = oracle.mat_inverse(mds)
    for i in range(12):
        for j in range(12):
            s = sum(int(mds[i, k]) * int(inv[k, j]) for k in range(12)) % P
            assert s == (1 if i == j else 0)


# ------------------------------------------------- permutation structure

FULL = [r < 4 or r >= 26 for r in range(30)]  # 4 full, 22 partial, 4 full (Alg. 1)


def _states(seed, n):
    return pg_synth.matrix(seed, n, 12)


def test_identity_matrix_zero_constants_is_pure_powers():
    # M = I, C = 0: cell 0 is raised to 7 in all 30 rounds, the others only in
    # the 8 full rounds.
    rc = np.zeros((30, 12), dtype=np.uint64)
    eye = np.eye(12, dtype=np.uint64)
    st = _states(11, 6)
    out = oracle.permute(st, rc, eye)
    for k in range(6):
        for i in range(12):
            e = 7 ** 30 if i == 0 else 7 ** 8
            assert int(out[k, i]) == pow(int(st[k, i]), e, P)


def test_shift_matrix_pins_orientation_and_partial_cell():
    # M with M[i][(i+1) % 12] = 1: new_i = x_{i+1}.  Track which input cell
    # sits in each position and how many S-boxes it went through.
    rc = np.zeros((30, 12), dtype=np.uint64)
    m = np.zeros((12, 12), dtype=np.uint64)
    for i in range(12):
        m[i, (i + 1) % 12] = 1
    st = _states(12, 4)
    pos = list(range(12))  # pos[i] = input cell now at position i
    exps = [1] * 12        # exps[i] = exponent of that cell
    for r in range(30):
        if FULL[r]:
            exps = [e * 7 for e in exps]
        else:
            exps[0] *= 7
        pos = [pos[(i + 1) % 12] for i in range(12)]
        exps = [exps[(i + 1) % 12] for i in range(12)]
    out = oracle.permute(st, rc, m)
    for k in range(4):
        for i in range(12):
            assert int(out[k, i]) == pow(int(st[k, pos[i]]), exps[i], P)


def test_constants_added_before_sbox_identity_matrix():
    rc = pg_synth.matrix(13, 30, 12)
    eye = np.eye(12, dtype=np.uint64)
    st = _states(14, 3)
    out = oracle.permute(st, rc, eye)
    for k in range(3):
        x = [int(v) for v in st[k]]
        for r in range(30):
            x = [(x[i] + int(rc[r, i])) % P for i in range(12)]
            x = [pow(v, 7, P) if (FULL[r] or i == 0) else v for i, v in enumerate(x)]
        assert [int(v) for v in out[k]] == x


def test_single_offdiagonal_pins_summation_index():
    # M = I + a*E_{0,1}: new_0 = y_0 + a*y_1, other cells unchanged.
    a = 0x0123456789ABCDEF % P
    rc = pg_synth.matrix(15, 30, 12)
    m = np.eye(12, dtype=np.uint64)
    m[0, 1] = a
    st = _states(16, 3)
    out = oracle.permute(st, rc, m)
    for k in range(3):
        x = [int(v) for v in st[k]]
        for r in range(30):
            y = [(x[i] + int(rc[r, i])) % P for i in range(12)]
            y = [pow(v, 7, P) if (FULL[r] or i == 0) else v for i, v in enumerate(y)]
            y[0] = (y[0] + a * y[1]) % P
            x = y
        assert [int(v) for v in out[k]] == x


def test_dense_round_structure_one_state_bigint():
    # The actual parameter set, evaluated here round by round with Python
    # integers (independent of the oracle's C arithmetic).
    rc, mds, _, _, _ = oracle.params()
    st = _states(17, 2)
    out = oracle.permute(st, rc, mds)
    M = [[int(v) for v in row] for row in mds]
    for k in range(2):
        x = [int(v) for v in st[k]]
        for r in range(30):
            y = [(x[i] + int(rc[r, i])) % P for i in range(12)]
            y = [pow(v, 7, P) if (FULL[r] or i == 0) else v for i, v in enumerate(y)]
            x = [sum(M[i][j] * y[j] for j in range(12)) % P for i in range(12)]
        assert [int(v) for v in out[k]] == x


def test_inverse_round_trip():
    st = _states(18, 64)
    out = oracle.permute(st)
    back = oracle.permute_inverse(out)
    assert (back == st).all()
    assert not (out == st).all()


def test_noncanonical_inputs_are_reduced():
    st = _states(19, 4)
    shifted = st.copy()
    small = st < np.uint64((1 << 64) - P)
    shifted[small] = st[small] + np.uint64(P)  # same residue, non-canonical word
    assert (oracle.permute(shifted) == oracle.permute(st)).all()


def test_permutation_outputs_canonical_and_distinct():
    st = _states(20, 512)
    out = oracle.permute(st)
    assert (out < np.uint64(P)).all()
    assert len({tuple(int(v) for v in row) for row in out}) == 512


# ----------------------------------------------------------------- sponge

def test_sponge_width8_is_one_permutation():
    rows = pg_synth.matrix(21, 5, 8)
    d = oracle.hash_rows(rows)
    st = np.zeros((5, 12), dtype=np.uint64)
    st[:, :8] = rows
    assert (d == oracle.permute(st)[:, :4]).all()


def test_sponge_width16_overwrite_mode():
    rows = pg_synth.matrix(22, 3, 16)
    d = oracle.hash_rows(rows)
    for k in range(3):
        s = np.zeros(12, dtype=np.uint64)
        s[:8] = rows[k, :8]
        s = oracle.permute(s)
        s[:8] = rows[k, 8:]  # overwrite rate, keep capacity
        s = oracle.permute(s)
        assert (d[k] == s[:4]).all()


def test_sponge_ragged_width_zero_fills():
    rows = pg_synth.matrix(23, 3, 11)
    padded = np.zeros((3, 16), dtype=np.uint64)
    padded[:, :11] = rows
    assert (oracle.hash_rows(rows) == oracle.hash_rows(padded)).all()
    short = pg_synth.matrix(24, 2, 3)
    p8 = np.zeros((2, 8), dtype=np.uint64)
    p8[:, :3] = short
    assert (oracle.hash_rows(short) == oracle.hash_rows(p8)).all()


# ----------------------------------------------------------------- Merkle

def test_merkle_tiny_trees_hand_composed():
    rows = pg_synth.matrix(25, 4, 8)
    leaves = oracle.hash_rows(rows)
    n1 = oracle.merkle_build(rows[:1])
    assert n1.shape == (1, 4) and (n1[0] == leaves[0]).all()
    n2 = oracle.merkle_build(rows[:2])
    assert (n2[:2] == leaves[:2]).all()
    assert (n2[2] == oracle.hash_pair(leaves[0], leaves[1])).all()
    n4 = oracle.merkle_build(rows)
    a = oracle.hash_pair(leaves[0], leaves[1])
    b = oracle.hash_pair(leaves[2], leaves[3])
    assert (n4[:4] == leaves).all()
    assert (n4[4] == a).all() and (n4[5] == b).all()
    assert (n4[6] == oracle.hash_pair(a, b)).all()
    # the pair hash is perm([L, R, 0, 0, 0, 0]) truncated to four words
    s = np.zeros(12, dtype=np.uint64)
    s[:4], s[4:8] = leaves[0], leaves[1]
    assert (oracle.permute(s)[:4] == a).all()


def test_merkle_auth_paths_recompute_root():
    n = 64
    rows = pg_synth.matrix(26, n, 8)
    nodes = oracle.merkle_build(rows)
    root = nodes[-1]
    for idx in (0, 1, 17, 42, 63):
        path = oracle.auth_path(nodes, n, idx)
        assert path.shape == (6, 4)
        assert (oracle.root_from_path(nodes[idx], idx, path) == root).all()
        bad = path.copy()
        bad[3, 1] ^= np.uint64(1)
        assert not (oracle.root_from_path(nodes[idx], idx, bad) == root).all()


def test_merkle_flip_changes_exactly_the_ancestors():
    n = 32
    rows = pg_synth.matrix(27, n, 8)
    a = oracle.merkle_build(rows)
    rows2 = rows.copy()
    rows2[13, 5] = (rows2[13, 5] + np.uint64(1)) % np.uint64(P)
    b = oracle.merkle_build(rows2)
    offs = oracle.level_offsets(n)
    changed = set()
    idx = 13
    for lvl, off in enumerate(offs):
        changed.add(off + idx)
        idx //= 2
    for k in range(2 * n - 1):
        assert (not (a[k] == b[k]).all()) == (k in changed)


def test_merkle_threads_match_single_thread():
    rows = pg_synth.matrix(28, 128, 24)
    assert (oracle.merkle_build(rows, nthreads=1) == oracle.merkle_build(rows, nthreads=4)).all()


def test_permute_threads_match_single_thread():
    st = pg_synth.matrix(0x3A1, 301, 12)
    assert (oracle.permute(st, nthreads=7) == oracle.permute(st)).all()


def test_merkle_subtree_split_recombines():
    # sharding invariant: G subtrees built apart, top levels hashed from their
    # roots, equals the whole tree
    n, g = 64, 4
    rows = pg_synth.matrix(29, n, 8)
    full = oracle.merkle_build(rows)
    subs = [oracle.merkle_build(rows[k * n // g:(k + 1) * n // g])[-1] for k in range(g)]
    l1 = [oracle.hash_pair(subs[0], subs[1]), oracle.hash_pair(subs[2], subs[3])]
    root = oracle.hash_pair(l1[0], l1[1])
    assert (root == full[-1]).all()


def test_merkle_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.merkle_build(pg_synth.matrix(30, 3, 8))


# ------------------------------------------------ small-entry parameter set

def test_small_set_is_circulant_mds_with_v1_constants():
    rc, mds, row, cand = oracle.params_small()
    assert (rc == oracle.params()[0]).all()
    assert all(1 <= int(v) <= 255 for v in row)
    for i in range(12):
        for j in range(12):
            assert int(mds[i, j]) == int(row[(j - i) % 12])
    assert cand >= 0
    assert oracle.is_mds(mds)


def test_is_mds_rejects_a_singular_minor():
    # a circulant whose first row repeats with period 6 has equal rows i, i+6
    row = [3, 5, 7, 11, 13, 17] * 2
    m = np.array([[row[(j - i) % 12] for j in range(12)] for i in range(12)], dtype=np.uint64)
    assert not oracle.is_mds(m)
    # and a 2x2 minor that vanishes: [[2, 4], [1, 2]] inside an otherwise random matrix
    r = pg_synth.matrix(0x77, 12, 12)
    r[0, 0], r[0, 1], r[1, 0], r[1, 1] = 2, 4, 1, 2
    assert not oracle.is_mds(r)
