"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Every comparison is bit-exact: the path is integer arithmetic mod p and
every stored word is canonical, so any difference is a defect.
"""
import numpy as np
import pytest

import oracle
import pg_synth
from tree_check import check_tree_sampled

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu

P = 0xFFFFFFFF00000001
EDGE = [0, 1, 2, 0xFFFFFFFE, 0xFFFFFFFF, 1 << 32, 1 << 63, P - 2, P - 1, P, P + 1,
        (1 << 64) - 2, (1 << 64) - 1, 0x1234567890ABCDEF]


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)
    yield


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


# ------------------------------------------------------------ permutation

@pytest.mark.parametrize("n", [1, 2, 31, 127, 128, 129, 1000, 4097])
def test_permute_batch_ragged(n):
    st = pg_synth.matrix(0x100 + n, n, 12)
    t = dev(st)
    pg.permute_batch(t)
    assert (host(t) == oracle.permute(st)).all()


def test_permute_batch_edge_words():
    rng = np.random.default_rng(5)
    st = np.array(EDGE, dtype=np.uint64)[rng.integers(0, len(EDGE), size=(300, 12))]
    st[0] = 0
    st[1] = np.uint64((1 << 64) - 1)
    st[2] = np.uint64(P - 1)
    t = dev(st)
    pg.permute_batch(t)
    assert (host(t) == oracle.permute(st)).all()


def test_permute_batch_unaligned_pointer():
    st = pg_synth.matrix(0x222, 257, 12)
    buf = torch.zeros(257 * 12 + 1, dtype=torch.int64, device="cuda")
    view = buf[1:].view(257, 12)  # 8-byte but not 16-byte aligned
    view.copy_(dev(st))
    pg.permute_batch(view)
    assert (host(view) == oracle.permute(st)).all()


def test_permute_batch_empty_is_noop():
    t = torch.zeros((0, 12), dtype=torch.int64, device="cuda")
    pg.permute_batch(t)


def test_permute_batch_full_size_sampled():
    # 2^24 independent states (the raw-throughput workload), in place; every
    # output canonical, a seeded sample recomputed by the oracle
    n = 1 << 24
    st = pg_synth.matrix(pg_synth.config_seed(2), n, 12)
    t = dev(st)
    pg.permute_batch(t)
    out = host(t)
    assert (out < np.uint64(P)).all()
    idx = np.sort(pg_synth.integers(0xC0FFEE, 2048, 0, n - 1))
    idx = np.unique(np.concatenate([idx, [0, 1, n - 2, n - 1]]))
    assert (out[idx] == oracle.permute(st[idx])).all()


# ----------------------------------------------------------------- sponge

@pytest.mark.parametrize("w", [1, 3, 4, 7, 8, 9, 15, 16, 17, 24, 64, 100, 256])
def test_hash_rows_widths(w):
    n = 130
    rows = pg_synth.matrix(0x300 + w, n, w)
    d = pg.hash_rows(dev(rows))
    assert (host(d) == oracle.hash_rows(rows)).all()


def test_hash_rows_non_canonical_inputs():
    rows = pg_synth.matrix(0x333, 64, 16)
    rows[:, ::3] = np.uint64((1 << 64) - 1)
    rows[:, 1] = np.uint64(P)
    d = pg.hash_rows(dev(rows))
    assert (host(d) == oracle.hash_rows(rows)).all()


def test_hash_rows_unaligned_rows():
    w, n = 10, 77
    rows = pg_synth.matrix(0x344, n, w)
    buf = torch.zeros(n * w + 1, dtype=torch.int64, device="cuda")
    view = buf[1:].view(n, w)
    view.copy_(dev(rows))
    d = pg.hash_rows(view)
    assert (host(d) == oracle.hash_rows(rows)).all()


def test_hash_rows_width_zero_rejected():
    t = torch.zeros((4, 0), dtype=torch.int64, device="cuda")
    with pytest.raises(pg.PGError) as e:
        pg.hash_rows(t, digests=torch.zeros((4, 4), dtype=torch.int64, device="cuda"))
    assert e.value.status == 1


# ----------------------------------------------------------------- Merkle

def test_merkle_workload1_all_levels_and_golden_root():
    # 2^10 leaves of 8 elements: every level against the oracle, root
    # against the stored value
    rows = pg_synth.matrix(pg_synth.config_seed(1), 1 << 10, 8)
    nodes, root = pg.merkle_build(dev(rows), want_root=True)
    want = oracle.merkle_build(rows, nthreads=4)
    assert (host(nodes) == want).all()
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "cfg1_root.txt")) as f:
        golden = [int(v, 16) for v in f.read().split()]
    assert root == golden


@pytest.mark.parametrize("log_n", [0, 1, 2, 3, 5, 6, 7, 8, 9, 10, 12, 13, 14, 15, 16])
@pytest.mark.parametrize("w", [8, 5, 16])
def test_merkle_sizes_full_compare(log_n, w):
    n = 1 << log_n
    rows = pg_synth.matrix(0x400 + 37 * log_n + w, n, w)
    nodes = pg.merkle_build(dev(rows))
    assert (host(nodes) == oracle.merkle_build(rows, nthreads=8)).all()


@pytest.mark.parametrize("w", [1, 64, 100])
def test_merkle_wide_and_narrow_rows(w):
    n = 1 << 11
    rows = pg_synth.matrix(0x500 + w, n, w)
    nodes = pg.merkle_build(dev(rows))
    assert (host(nodes) == oracle.merkle_build(rows, nthreads=8)).all()


def _check_tree_sampled(rows, out, seed, per_level=64):
    check_tree_sampled(rows, out, seed, per_level=per_level)


@pytest.mark.parametrize("w", [8, 64])
def test_merkle_paper_scale_sampled(w):
    # 2^22 leaves (the paper's tree) at widths 8 and 64: sampled leaves and
    # nodes of every level recomputed by the oracle from the GPU's children
    n = 1 << 22
    rows = pg_synth.matrix(pg_synth.config_seed(3) + w, n, w)
    t = dev(rows)
    nodes, root = pg.merkle_build(t, want_root=True)
    out = host(nodes)
    assert [int(v) for v in out[-1]] == root
    _check_tree_sampled(rows, out, seed=0x700 + w)
    # a rebuild is bit-identical
    again = host(pg.merkle_build(t))
    assert (again == out).all()


def test_merkle_rejects_non_power_of_two():
    t = torch.zeros((3, 8), dtype=torch.int64, device="cuda")
    with pytest.raises(pg.PGError) as e:
        pg.merkle_build(t, nodes=torch.zeros((5, 4), dtype=torch.int64, device="cuda"))
    assert e.value.status == 2


@pytest.mark.parametrize("log_n", [7, 12, 17])
def test_merkle_back_to_back_builds(log_n):
    # consecutive builds queued on one stream with no synchronisation between
    # them (each level launch may start while the one before finishes): every
    # tree must still equal its oracle build
    n = 1 << log_n
    sets = [pg_synth.matrix(0x900 + 11 * log_n + k, n, 8) for k in range(6)]
    devs = [dev(r) for r in sets]
    outs = [torch.empty((2 * n - 1, 4), dtype=torch.int64, device="cuda") for _ in sets]
    torch.cuda.synchronize()
    for t, o in zip(devs, outs):
        pg.merkle_build(t, o)
    # the same buffers again, in reverse order, over the first results
    for t, o in zip(reversed(devs), outs):
        pg.merkle_build(t, o)
    for r, o in zip(reversed(sets), outs):
        assert (host(o) == oracle.merkle_build(r, nthreads=8)).all()


def test_merkle_on_side_stream():
    rows = pg_synth.matrix(0x777, 1 << 9, 8)
    s = torch.cuda.Stream()
    t = dev(rows)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        nodes = pg.merkle_build(t, stream=s)
    s.synchronize()
    assert (host(nodes) == oracle.merkle_build(rows, nthreads=4)).all()


@pytest.mark.parametrize("engine", [pg.ENGINE_TENSOR, pg.ENGINE_INT])
def test_merkle_builds_on_two_streams_at_once(engine):
    # two different trees built concurrently on two streams with no
    # synchronisation between them: the build keeps no shared device state
    n = 1 << 16
    a_np = pg_synth.matrix(0xA51, n, 8)
    b_np = pg_synth.matrix(0xB52, n, 24)
    a, b = dev(a_np), dev(b_np)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    pg.set_engine(engine)
    try:
        outs = []
        for _ in range(3):
            with torch.cuda.stream(sa):
                na = pg.merkle_build(a, stream=sa)
            with torch.cuda.stream(sb):
                nb = pg.merkle_build(b, stream=sb)
            outs.append((na, nb))
        sa.synchronize()
        sb.synchronize()
    finally:
        pg.set_engine(pg.ENGINE_TENSOR)
    want_a = oracle.merkle_build(a_np, nthreads=8)
    want_b = oracle.merkle_build(b_np, nthreads=8)
    for na, nb in outs:
        assert (host(na) == want_a).all()
        assert (host(nb) == want_b).all()


def test_merkle_rejects_overlapping_rows_and_nodes():
    # checked on the host before anything is launched
    buf = torch.zeros(1 << 16, dtype=torch.int64, device="cuda")
    rows = buf[: 1024 * 8].view(1024, 8)
    nodes = buf[4096: 4096 + 2047 * 4].view(2047, 4)
    with pytest.raises(pg.PGError) as e:
        pg.merkle_build(rows, nodes)
    assert e.value.status == 1 and "overlap" in pg.last_error()
    # two trees of a batch whose node buffers share words
    ra = torch.zeros((1024, 8), dtype=torch.int64, device="cuda")
    rb = torch.zeros((1024, 8), dtype=torch.int64, device="cuda")
    nbuf = torch.zeros(3 * 2047 * 4, dtype=torch.int64, device="cuda")
    na, nb = nbuf[: 2047 * 4].view(2047, 4), nbuf[4000: 4000 + 2047 * 4].view(2047, 4)
    with pytest.raises(pg.PGError) as e:
        pg.merkle_build_batch([ra, rb], nodes_list=[na, nb])
    assert e.value.status == 1 and "overlap" in pg.last_error()
