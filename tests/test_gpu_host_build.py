"""pg_merkle_build_host: rows in host memory, copied in chunks overlapped with
leaf hashing.  The nodes must equal pg_merkle_build's on the same rows bit for
bit (tolerance zero), for single-chunk and many-chunk trees, odd widths (no
16-byte loads), pageable and page-locked host memory, and repeated calls that
reuse the staging buffer."""
import numpy as np
import pytest

import oracle
import pg_synth

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)
    yield


@pytest.mark.parametrize("log_n,w,pinned", [(0, 8, False), (6, 3, True), (13, 8, True), (14, 8, False),
                                            (18, 8, True), (19, 5, True), (21, 8, True), (20, 16, False)])
def test_host_build_equals_device_build(log_n, w, pinned):
    n = 1 << log_n
    rows = pg_synth.matrix_torch(0x8800 + 3 * log_n + w, n, w).contiguous()
    host = rows.pin_memory() if pinned else rows
    want = pg.merkle_build(rows.cuda())
    nodes, root = pg.merkle_build_host(host, want_root=True)
    assert torch.equal(nodes, want)
    assert root == [int(v) for v in want[-1].cpu().numpy().view(np.uint64)]


def test_host_build_small_tree_matches_oracle():
    rows = pg_synth.matrix(0x8900, 1 << 10, 8)
    nodes = pg.merkle_build_host(torch.from_numpy(rows.view(np.int64)))
    torch.cuda.synchronize()
    assert (nodes.cpu().numpy().view(np.uint64) == oracle.merkle_build(rows, nthreads=8)).all()


def test_host_build_reuses_staging_buffer_back_to_back():
    n, w = 1 << 20, 8
    a = pg_synth.matrix_torch(0x8A00, n, w).pin_memory()
    b = pg_synth.matrix_torch(0x8A01, n, w).pin_memory()
    stage = torch.empty((n, w), dtype=torch.int64, device="cuda")
    na = torch.empty((2 * n - 1, 4), dtype=torch.int64, device="cuda")
    nb = torch.empty_like(na)
    # queued without synchronising: b's copies must wait for a's leaf hashing
    pg.merkle_build_host(a, stage, na)
    pg.merkle_build_host(b, stage, nb)
    torch.cuda.synchronize()
    assert torch.equal(na, pg.merkle_build(a.cuda()))
    assert torch.equal(nb, pg.merkle_build(b.cuda()))
    assert torch.equal(stage, b.cuda())


def test_host_build_streams_its_leaves_in_one_launch():
    # tensor engine, rows of at least 64 MiB: one leaf launch consumes the copied chunks as they land
    n, w = 1 << 21, 8
    rows = pg_synth.matrix_torch(0x8B00, n, w).pin_memory()
    torch.cuda.synchronize()
    pg.profile_enable(True)
    nodes = pg.merkle_build_host(rows)
    torch.cuda.synchronize()
    kern = pg.profile_read()
    pg.profile_enable(False)
    assert kern["k_tc_sponge:leaves"]["launches"] == 1
    assert torch.equal(nodes, pg.merkle_build(rows.cuda()))


def test_host_build_arrival_counter_restarts():
    # every streamed build takes 16 values of the chunk arrival counter, which
    # restarts after 4096 builds; alternating two row sets makes a launch that
    # read a chunk before it arrived hash the other set's rows
    n, w = 1 << 20, 8
    sets = [pg_synth.matrix_torch(0x8C00 + k, n, w).pin_memory() for k in range(2)]
    want = [pg.merkle_build(r.cuda()) for r in sets]
    stage = torch.empty((n, w), dtype=torch.int64, device="cuda")
    nodes = torch.empty((2 * n - 1, 4), dtype=torch.int64, device="cuda")
    faults = pg.device_faults()
    for i in range(4100):
        pg.merkle_build_host(sets[i % 2], stage, nodes)
        if i % 512 == 0 or 4090 <= i:
            torch.cuda.synchronize()
            assert torch.equal(nodes, want[i % 2]), i
    assert pg.device_faults() == 0 and faults == 0


_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import torch, paper_2506_09505_gb300 as pg, pg_synth
pg.load()
pg.init(0)
n, w = 1 << 21, 8
rows = pg_synth.matrix_torch(0x8D00, n, w).pin_memory()
torch.cuda.synchronize()
pg.profile_enable(True)
nodes = pg.merkle_build_host(rows)
torch.cuda.synchronize()
kern = pg.profile_read()
launches = sum(kern[k]["launches"] for k in ("k_tc_sponge:leaves", "k_tc_sponge:rows") if k in kern)
pg.profile_enable(False)
ok = torch.equal(nodes, pg.merkle_build(rows.cuda()))
print("child", launches, ok, pg.device_faults())
"""


@pytest.mark.parametrize("env,streamed", [({"CUDA_LAUNCH_BLOCKING": "1"}, True), ({"PG12_HOST_STREAM": "0"}, False)])
def test_host_build_in_a_fresh_process(env, streamed):
    # blocking launches: the chunk copies are queued before the streamed leaf
    # launch, so it still finds them arriving; PG12_HOST_STREAM=0: one leaf
    # launch per chunk (the form to use under tools that hold copies back)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _CHILD.format(root=root)], capture_output=True, text=True,
                         timeout=600, cwd=root, env={**os.environ, **env})
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("child ")][-1].split()
    launches, ok, faults = int(line[1]), line[2] == "True", int(line[3])
    assert ok and faults == 0
    assert (launches == 1) == streamed
