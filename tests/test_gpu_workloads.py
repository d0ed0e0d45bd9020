"""GPU parity at the size distributions of the batched and served workloads.

The 64-tree batch is the one the benchmark times (leaf counts 2^k, k in
[12, 20], widths in {8, 16, 32, 64, 128}), built through the autotuned
captured graph; the served stream draws k in [10, 18] and widths in
{8, 32, 128, 256} (the workload's distribution with the largest trees left
out to bound memory).  Batch trees of at most 2^16 leaves are compared with
the oracle in full, larger ones on sampled leaves and sampled nodes of every
level; every served tree equals its solo build and each served shape is
checked the sampled way.
"""
import os

import numpy as np
import pytest

import oracle
import pg_synth
from tree_check import check_tree_sampled

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)
    yield


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def test_batch_workload_distribution():
    sizes = pg_synth.batch_sizes(64, 20)
    rows = [pg_synth.matrix_torch(pg_synth.batch_tree_seed(k), 1 << lg, w, device="cuda")
            for k, (lg, w) in enumerate(sizes)]
    nodes = pg.alloc_nodes(rows)
    best, _ = pg.batch_autotune(rows, nodes)
    g = pg.BatchGraph(rows, nodes, schedule=best)
    try:
        g.launch()
        torch.cuda.synchronize()
        for k, (r, nd) in enumerate(zip(rows, nodes)):
            out = _host(nd)
            if r.shape[0] <= 1 << 16:
                assert (out == oracle.merkle_build(_host(r), nthreads=os.cpu_count() or 1)).all(), k
            else:
                check_tree_sampled(r, out, seed=0xB000 + k, n_leaves=64, per_level=16)
    finally:
        g.close()


def test_served_stream_distribution():
    seed = pg_synth.config_seed(5) + 1
    nreq = 48
    ks = pg_synth.integers(seed, nreq, 10, 18)
    ws = [(8, 32, 128, 256)[int(v)] for v in pg_synth.integers(seed + 1, nreq, 0, 3)]
    cache = {}
    reqs = []
    for i in range(nreq):
        key = (int(ks[i]), ws[i])
        if key not in cache:
            cache[key] = pg_synth.matrix_torch(pg_synth.tree_seed(seed, len(cache)), 1 << key[0], key[1], device="cuda")
        reqs.append(cache[key])
    torch.cuda.synchronize()
    srv = pg.Server(pool_bytes=4 << 30, max_batch=32, max_inflight=2)
    try:
        ids = [srv.submit(r) for r in reqs]
        srv.drain(300.0)
        checked = set()
        for i, (rid, r) in enumerate(zip(ids, reqs)):
            assert srv.query(rid)["state"] == pg.REQ_DONE
            got = srv.nodes(rid, r.shape[0])
            assert torch.equal(got, pg.merkle_build(r)), i
            key = (int(ks[i]), ws[i])
            if key not in checked:
                checked.add(key)
                check_tree_sampled(r, _host(got), seed=0xC000 + i, n_leaves=32, per_level=8)
            srv.release(rid)
    finally:
        srv.close()
