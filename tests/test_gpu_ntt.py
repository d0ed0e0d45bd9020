"""GPU parity of the NTT and the low-degree extension (pg_ntt / pg_lde).

Bit-exact against the oracle (textbook definitions of the transform behind
the Sec. 2.3 NTT hotspot).  Sizes cover one pass (up to 2^10 rows), several
passes with uneven splits, ragged column chunks (the kernel takes eight
columns per block), non-canonical input words, the degenerate one-row case
and the LDE shape the commitment benchmark uses, there on sampled rows.
"""
import numpy as np
import pytest

import oracle
import pg_synth

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu
P = oracle.P


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)
    yield


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("log_n,ncols", [(0, 1), (0, 5), (1, 1), (3, 8), (10, 3), (10, 8), (11, 1),
                                         (11, 11), (13, 16), (15, 2), (17, 9)])
def test_ntt_forward_and_inverse(log_n, ncols):
    n = 1 << log_n
    x = pg_synth.matrix(0x7710 + 31 * log_n + ncols, n, ncols)
    want = oracle.ntt_columns(x)
    t = dev(x)
    pg.ntt(t)
    got = host(t)
    assert (got == want).all()
    pg.ntt(t, inverse=True)
    assert (host(t) == x).all()
    back = oracle.ntt_columns(want, inverse=True)
    t2 = dev(want)
    pg.ntt(t2, inverse=True)
    assert (host(t2) == back).all()


def test_ntt_non_canonical_words():
    n, c = 256, 4
    rng = np.random.default_rng(11)
    edge = np.array([0, 1, P - 1, P, P + 1, (1 << 64) - 1, 1 << 63, 0xFFFFFFFF], dtype=np.uint64)
    x = edge[rng.integers(0, len(edge), size=(n, c))]
    t = dev(x)
    pg.ntt(t)
    assert (host(t) == oracle.ntt_columns(x)).all()


def test_ntt_2e20x8_against_the_oracle():
    # two passes of ten bits (radix-8, -8, -4, -4 steps each), forward and inverse, every word
    n, c = 1 << 20, 8
    x = pg_synth.matrix(0x7711, n, c)
    want = oracle.ntt_columns(x)
    t = dev(x)
    pg.ntt(t)
    assert (host(t) == want).all()
    back = dev(want)
    pg.ntt(back, inverse=True)
    assert (host(back) == x).all()


def test_ntt_round_trip_large():
    n, c = 1 << 20, 8
    x = pg_synth.matrix_torch(0x7720, n, c, device="cuda")
    y = x.clone()
    pg.ntt(y)
    pg.ntt(y, inverse=True)
    assert torch.equal(x, y)


@pytest.mark.parametrize("log_n,log_b,ncols", [(0, 0, 1), (0, 3, 2), (1, 1, 1), (2, 4, 3), (4, 2, 3), (10, 1, 8),
                                               (10, 0, 5), (11, 3, 5), (13, 2, 9), (12, 1, 16), (4, 6, 2), (9, 5, 8),
                                               (15, 1, 8), (18, 1, 3), (18, 2, 4)])
def test_lde_matches_oracle(log_n, log_b, ncols):
    n = 1 << log_n
    evals = pg_synth.matrix(0x7730 + 37 * log_n + 5 * log_b + ncols, n, ncols)
    want = oracle.lde_columns(evals, log_b)
    e = dev(evals)
    out = pg.lde(e, log_b)
    assert (host(out) == want).all()
    assert (host(e) == evals).all()  # evals untouched when scratch is separate


def test_lde_in_place_scratch():
    n, c, b = 1 << 9, 6, 2
    evals = pg_synth.matrix(0x7740, n, c)
    e = dev(evals)
    out = pg.lde(e, b, scratch=e)
    assert (host(out) == oracle.lde_columns(evals, b)).all()


def test_lde_rejects_bad_arguments():
    e = torch.zeros((6, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(RuntimeError):
        pg.lde(e, 1)
    e = torch.zeros((8, 2), dtype=torch.int64, device="cuda")
    big = torch.zeros((16, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(RuntimeError):
        pg.lde(e, 1, out=big, scratch=big[:8])  # scratch inside out


def test_lde_feeds_the_commitment():
    n, c, b = 1 << 8, 8, 2
    evals = pg_synth.matrix(0x7750, n, c)
    want_rows = oracle.lde_columns(evals, b)
    out = pg.lde(dev(evals), b)
    nodes = pg.merkle_build(out)
    assert (host(nodes) == oracle.merkle_build(want_rows, nthreads=8)).all()


def test_lde_benchmark_shape_sampled_rows():
    # the commitment workload: 2^21 rows x 8 columns, blowup 2 -> 2^22 x 8
    log_n, c, b = 21, 8, 1
    n = 1 << log_n
    evals_t = pg_synth.matrix_torch(0x5EED0006, n, c, device="cuda")
    out = host(pg.lde(evals_t, b))
    evals = host(evals_t)
    rows = [0, 1, 2, 3, (n << b) - 1, (n << b) - 2] + [int(v) for v in pg_synth.integers(0x7760, 6, 0, (n << b) - 1)]
    w = oracle.two_adic_root(log_n + b)
    for col in (0, 5):
        coeffs = oracle.fft(np.ascontiguousarray(evals[:, col]), inverse=True)
        for r in rows:
            x = oracle.LDE_SHIFT * pow(w, r, P) % P
            assert int(out[r, col]) == oracle.poly_eval(coeffs, x), (col, r)
    # rows 2i are the extension evaluated on 7 * <w_n>: check one column against the oracle's own LDE with b = 0
    small = oracle.lde_columns(np.ascontiguousarray(evals[:, 3:4]), 0)
    assert (out[:: 1 << b, 3] == small[:, 0]).all()
