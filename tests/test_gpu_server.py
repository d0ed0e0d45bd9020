"""GPU tests of the serving runtime: requests that arrive while others run
are batched together, admission waits for pool memory, and every result is
bit-identical to the same tree built alone (tolerance zero)."""
import time

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def test_server_results_equal_solo_builds():
    sizes = [(10, 8), (14, 32), (12, 8), (16, 8), (11, 128), (13, 256), (15, 8), (10, 1)]
    rows = [_dev(pg_synth.matrix(0xE00 + k, 1 << lg, w)) for k, (lg, w) in enumerate(sizes)]
    torch.cuda.synchronize()
    srv = pg.Server(pool_bytes=1 << 28, max_inflight=2)
    try:
        ids = []
        for r in rows:
            ids.append(srv.submit(r))
            time.sleep(0.0005)  # staggered arrivals: later ones join later launches
        srv.drain(60.0)
        batches = set()
        for rid, r in zip(ids, rows):
            info = srv.query(rid)
            assert info["state"] == pg.REQ_DONE
            assert info["submit_s"] <= info["launch_s"] <= info["done_s"]
            batches.add(info["batch_size"])
            got = srv.nodes(rid, r.shape[0])
            assert torch.equal(got, pg.merkle_build(r))
            srv.release(rid)
    finally:
        srv.close()


def test_server_admission_waits_for_pool_memory():
    # pool holds one 2^14-leaf node buffer (1 MiB) at a time: the second
    # request is admitted only after the first is released
    n = 1 << 14
    rows = [_dev(pg_synth.matrix(0xE80 + k, n, 8)) for k in range(2)]
    srv = pg.Server(pool_bytes=(2 * n - 1) * 32 + 4096, max_inflight=2)
    try:
        a = srv.submit(rows[0])
        b = srv.submit(rows[1])
        t0 = time.time()
        while srv.query(a)["state"] != pg.REQ_DONE and time.time() - t0 < 30:
            time.sleep(0.001)
        assert srv.query(a)["state"] == pg.REQ_DONE
        time.sleep(0.05)
        assert srv.query(b)["state"] == pg.REQ_QUEUED
        first = srv.nodes(a, n).clone()
        srv.release(a)
        srv.drain(30.0)
        assert srv.query(b)["state"] == pg.REQ_DONE
        assert torch.equal(first, pg.merkle_build(rows[0]))
        assert torch.equal(srv.nodes(b, n), pg.merkle_build(rows[1]))
        srv.release(b)
    finally:
        srv.close()


def test_server_drain_times_out_and_rejects_oversize():
    n = 1 << 12
    rows = _dev(pg_synth.matrix(0xEC0, n, 8))
    srv = pg.Server(pool_bytes=(2 * n - 1) * 32 + 256)
    try:
        big = _dev(pg_synth.matrix(0xEC1, 4 * n, 8))
        with pytest.raises(pg.PGError) as e:
            srv.submit(big)
        assert e.value.status == 3
        a = srv.submit(rows)
        srv.drain(30.0)
        b = srv.submit(rows)  # cannot be admitted until a is released
        with pytest.raises(pg.PGError) as e:
            srv.drain(0.2)
        assert e.value.status == 5
        srv.release(a)
        srv.drain(30.0)
        assert srv.query(b)["state"] == pg.REQ_DONE
        srv.release(b)
    finally:
        srv.close()
