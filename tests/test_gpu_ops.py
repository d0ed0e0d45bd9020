"""GPU field operations (Table 1 counterparts) against big-integer math and
the oracle, bit-exact; and the per-operation microbenchmark runs."""
import numpy as np
import pytest

import oracle
import pg_synth

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu

P = 0xFFFFFFFF00000001
EDGE = [0, 1, 2, 0xFFFFFFFE, 0xFFFFFFFF, 1 << 32, (1 << 32) + 1, 1 << 63, P - 2, P - 1, P, P + 1,
        (1 << 64) - 2, (1 << 64) - 1, 0x1234567890ABCDEF]


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)
    yield


def _pairs():
    e = np.array(EDGE, dtype=np.uint64)
    a = np.concatenate([np.repeat(e, len(e)), pg_synth.words(0xF00, 20000, bound=None)])
    b = np.concatenate([np.tile(e, len(e)), pg_synth.words(0xF01, 20000, bound=None)])
    return a, b


def _run(op, a, b):
    ta = torch.from_numpy(a.view(np.int64)).cuda()
    tb = torch.from_numpy(b.view(np.int64)).cuda()
    out = pg.field_eval(op, ta, tb)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("op,fn", [
    ("add", lambda a, b: (a + b) % P),
    ("sub", lambda a, b: (a - b) % P),
    ("mul", lambda a, b: (a * b) % P),
    ("sqr", lambda a, b: (a * a) % P),
    ("reduce", lambda a, b: ((b << 64) + a) % P),
    ("mul_small", lambda a, b: (a * (b & 0xFF)) % P),
    ("sbox", lambda a, b: pow(a, 7, P)),
])
def test_field_op_bigint(op, fn):
    a, b = _pairs()
    got = _run(op, a, b)
    want = [fn(int(x), int(y)) for x, y in zip(a, b)]
    assert [int(v) for v in got] == want


def test_field_mul_matches_oracle():
    a, b = _pairs()
    got = _run("mul", a, b)
    assert all(int(g) == oracle.mul(int(x), int(y)) for g, x, y in zip(got[:3000], a[:3000], b[:3000]))


@pytest.mark.parametrize("op", ["add", "mul", "sqr", "reduce", "sbox", "dot12"])
def test_field_bench_runs(op):
    rate, per_clk = pg.field_bench(op)
    assert rate > 0 and per_clk > 0


def test_latency_chains_are_ordered():
    # one dependent chain per op: an S-box is at least three products deep, a permutation
    # (8 full + 22 partial rounds, 30 S-boxes in sequence) far deeper than one S-box
    lat = {op: pg.field_bench(op)[1] for op in ("lat_mul", "lat_sbox", "lat_dot12", "lat_perm", "lat_perm_wide")}
    assert all(v > 0 for v in lat.values())
    assert lat["lat_sbox"] > 2.5 * lat["lat_mul"]
    assert lat["lat_perm_wide"] > 20 * lat["lat_sbox"]
    assert lat["lat_perm"] > lat["lat_perm_wide"]


@pytest.fixture(scope="module")
def big_pairs():
    # 10^8 full-range words per operand (weak, non-canonical inputs included)
    n = 10 ** 8
    return pg_synth.words(0xF10, n, bound=None), pg_synth.words(0xF11, n, bound=None)


@pytest.mark.parametrize("op", ["add", "sub", "mul", "sqr", "sbox"])
def test_field_op_1e8_random_pairs_vs_oracle(big_pairs, op):
    a, b = big_pairs
    got = _run(op, a, b)
    want = oracle.field_many(op, a, b)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (op, bad[:5], a[bad[:5]], b[bad[:5]])
