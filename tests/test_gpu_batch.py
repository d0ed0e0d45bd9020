"""GPU parity of the batched Merkle path (pg_merkle_build_batch, captured
graphs, the autotuner): every tree of a batch must equal the same tree built
alone and the CPU oracle, bit for bit, whatever the schedule.
"""
import numpy as np
import pytest

import oracle
import pg_synth

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu

MIX = [(0, 8), (1, 8), (5, 3), (6, 16), (10, 8), (12, 24), (3, 64), (11, 1), (9, 100), (7, 8)]


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)
    yield


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def _mix(seed=0x900):
    host_rows = [pg_synth.matrix(seed + k, 1 << lg, w) for k, (lg, w) in enumerate(MIX)]
    return host_rows, [_dev(r) for r in host_rows]


INT, TC = pg.BATCH_ENGINE_INT, pg.BATCH_ENGINE_TENSOR
SCHEDULES = [None,
             {"engine": INT, "block": 128}, {"engine": INT, "block": 256, "order": 1},
             {"engine": INT, "block": 128, "blocks_per_sm": 1, "order": 1},
             {"engine": INT, "top_lanes": 16},
             {"engine": TC}, {"engine": TC, "order": 1}, {"engine": TC, "fuse_levels": 1},
             {"engine": TC, "fuse_levels": 2, "top_lanes": 16}, {"engine": TC, "fuse_levels": 3, "order": 1},
             {"engine": TC, "top_lanes": 16}]


@pytest.mark.parametrize("sched", SCHEDULES)
def test_batch_equals_oracle(sched):
    host_rows, rows = _mix()
    nodes = pg.merkle_build_batch(rows, schedule=sched)
    for hr, nd in zip(host_rows, nodes):
        assert (_host(nd) == oracle.merkle_build(hr, nthreads=8)).all()


@pytest.mark.parametrize("sched", [{"order": 1}, {"engine": TC, "fuse_levels": 2, "order": 1},
                                   {"engine": TC, "fuse_levels": 1, "top_lanes": 16}])
def test_batch_equals_single_builds_larger_trees(sched):
    sizes = [(14, 8), (16, 8), (13, 64), (15, 16), (12, 128), (16, 32)]
    rows = [_dev(pg_synth.matrix(0xA00 + k, 1 << lg, w)) for k, (lg, w) in enumerate(sizes)]
    batch = pg.merkle_build_batch(rows, schedule=sched)
    for r, nd in zip(rows, batch):
        assert torch.equal(nd, pg.merkle_build(r))


def test_batch_rejects_bad_schedules():
    _, rows = _mix(0xE00)
    for bad in ({"engine": 3}, {"fuse_levels": 4}, {"top_lanes": 8}, {"block": 64}, {"order": 2}):
        with pytest.raises(pg.PGError) as e:
            pg.merkle_build_batch(rows, schedule=bad)
        assert e.value.status == 1, bad


def test_batch_graph_replays_identically():
    host_rows, rows = _mix(0xB00)
    g = pg.BatchGraph(rows, schedule={"order": 1})
    try:
        first = [t.clone() for t in g.launch()]
        torch.cuda.synchronize()
        for t in g.nodes:
            t.zero_()
        second = g.launch()
        torch.cuda.synchronize()
        for a, b in zip(first, second):
            assert torch.equal(a, b)
        for hr, nd in zip(host_rows, second):
            assert (_host(nd) == oracle.merkle_build(hr, nthreads=8)).all()
    finally:
        g.close()


def test_batch_graph_on_side_stream():
    _, rows = _mix(0xB80)
    g = pg.BatchGraph(rows)
    try:
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        out = g.launch(stream=s)
        s.synchronize()
        for r, nd in zip(rows, out):
            assert torch.equal(nd, pg.merkle_build(r))
    finally:
        g.close()


def test_autotune_returns_a_valid_schedule():
    _, rows = _mix(0xC00)
    best, ms = pg.batch_autotune(rows)
    assert best["engine"] in (INT, TC) and best["order"] in (0, 1) and best["top_lanes"] in (1, 16)
    if best["engine"] == INT:
        assert best["block"] in (128, 256)
    else:
        assert best["fuse_levels"] in (0, 1, 2)
    assert ms > 0
    nodes = pg.merkle_build_batch(rows, schedule=best)
    for r, nd in zip(rows, nodes):
        assert torch.equal(nd, pg.merkle_build(r))


def test_batch_rejects_bad_trees():
    ok = _dev(pg_synth.matrix(0xD00, 8, 8))
    bad = torch.zeros((3, 8), dtype=torch.int64, device="cuda")
    with pytest.raises(pg.PGError) as e:
        pg.merkle_build_batch([ok, bad], nodes_list=[torch.empty((15, 4), dtype=torch.int64, device="cuda"),
                                                   torch.empty((5, 4), dtype=torch.int64, device="cuda")])
    assert e.value.status == 2
    with pytest.raises(pg.PGError) as e:
        pg.merkle_build_batch([])
    assert e.value.status == 1
