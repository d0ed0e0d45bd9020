"""Launch timing (pg_profile_enable / pg_profile_read) on the GPU.

The permutations the library attributes to its launches must add up to the
work the method defines (Sec. 2.4: ceil(w/8) sponge permutations per leaf
plus one per inner node), whichever kernels a build is split across.
"""
import numpy as np
import pytest

import pg_synth

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)
    yield
    pg.profile_enable(False)


def _rows(log_n, w, seed):
    return pg_synth.matrix_torch(seed, 1 << log_n, w, device="cuda")


def _tree_perms(n, w):
    return n * ((w + 7) // 8) + n - 1


@pytest.mark.parametrize("engine", [pg.ENGINE_TENSOR, pg.ENGINE_INT])
@pytest.mark.parametrize("log_n,w", [(4, 8), (12, 3), (16, 8), (17, 20), (20, 8)])
def test_build_launches_account_for_every_permutation(log_n, w, engine):
    rows = _rows(log_n, w, 0x7000 + log_n)
    nodes = torch.empty((2 * (1 << log_n) - 1, 4), dtype=torch.int64, device="cuda")
    pg.set_engine(engine)
    try:
        pg.profile_enable(True)
        pg.merkle_build(rows, nodes)
        pg.merkle_build(rows, nodes)
        got = pg.profile_read()
        pg.profile_enable(False)
    finally:
        pg.set_engine(pg.ENGINE_TENSOR)
    assert got.pop("_dropped") == 0
    assert sum(v["perms"] for v in got.values()) == 2 * _tree_perms(1 << log_n, w)
    assert all(v["total_ms"] > 0 for v in got.values())
    n = 1 << log_n
    tc = engine == pg.ENGINE_TENSOR
    leaf_kernel = "k_tc_sponge:leaves" if tc else "k_merkle"
    # the leaves in one launch (the persistent or tensor-core kernel above 8,192 leaves,
    # else the 16-lane kernel), then one launch per level: the tensor-core kernel for
    # levels of at least 2^13 nodes (tensor engine), one thread per node (k_merkle_level)
    # above 8,192 nodes (integer engine), else the 16-lane kernel (k_merkle_top)
    if n > 8192:
        assert got[leaf_kernel]["launches"] == 2 and got[leaf_kernel]["perms"] == 2 * n * ((w + 7) // 8)
    else:
        assert leaf_kernel not in got and got["k_merkle_top_leaf"]["launches"] == 2
    levels = [n >> l for l in range(1, log_n + 1)]
    is_tc = [tc and n > 8192 and c >= 1 << 13 for c in levels]
    tc_levels = sum(is_tc)
    assert got.get("k_tc_sponge:level", {"launches": 0})["launches"] == 2 * tc_levels
    per_node = sum(1 for c, t in zip(levels, is_tc) if c > 8192 and not t)
    assert got.get("k_merkle_level", {"launches": 0})["launches"] == 2 * per_node
    # levels of 65..8,192 nodes not on the tensor cores: one k_merkle_top launch each; from
    # the first level of at most 64 nodes up to the root: one k_merkle_top_tail launch (or a
    # lone root: k_merkle_top)
    mid = sum(1 for c, t in zip(levels, is_tc) if 64 < c <= 8192 and not t)
    tail_first = next((l for l in range(1, log_n + 1) if n >> l <= 64), None)
    if tail_first is not None and tail_first < log_n:
        assert got.get("k_merkle_top_tail", {"launches": 0})["launches"] == 2
        assert got.get("k_merkle_top", {"launches": 0})["launches"] == 2 * mid
    else:
        assert "k_merkle_top_tail" not in got
        assert got.get("k_merkle_top", {"launches": 0})["launches"] == 2 * (log_n - per_node - tc_levels)


def test_other_entry_points_are_recorded():
    st = pg_synth.matrix_torch(0x7100, 1000, 12, device="cuda")
    rows = _rows(10, 8, 0x7101)
    pg.profile_enable(True)
    pg.permute_batch(st)
    pg.hash_rows(rows)
    trees = [_rows(9, 8, 0x7102), _rows(11, 16, 0x7103)]
    nodes = pg.alloc_nodes(trees)
    pg.merkle_build_batch(trees, nodes)
    g = pg.BatchGraph(trees, nodes)
    g.launch()
    got = pg.profile_read()
    g.close()
    pg.profile_enable(False)
    assert got["k_tc_permute"] == {"launches": 1, "perms": 1000, "total_ms": got["k_tc_permute"]["total_ms"]}
    assert got["k_tc_sponge:rows"]["perms"] == 1024
    batch = _tree_perms(1 << 9, 8) + _tree_perms(1 << 11, 16)
    # the batch launch and the graph launch (captured launches are not recorded)
    assert got["k_tc_batch"]["launches"] == 1 and got["k_tc_batch"]["perms"] == batch
    assert got["batch_graph"]["launches"] == 1 and got["batch_graph"]["perms"] == batch


def test_disabled_records_nothing():
    pg.profile_enable(False)
    rows = _rows(8, 8, 0x7200)
    pg.hash_rows(rows)
    torch.cuda.synchronize()
    assert pg.profile_read() == {"_dropped": 0}
