"""Allocation-free Merkle build (pg_merkle_build_noalloc) against pg_merkle_build.

The allocation-free entry point exists for callers that cannot call
cudaMalloc -- for example code running under an allocator that forbids it,
or a process that may only use the device buffers it was given.  It keeps
its scratch in a fixed array inside the library.  This file runs last in a
pytest session (its name sorts last) and also passes on its own in a fresh
process.  The path is exact integer arithmetic, so the tolerance is zero:
outputs must match word for word.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import pg_synth

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)  # for the reference entry point only; the no-alloc call needs no init
    yield


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _noalloc_raw(rows, nodes):
    # straight through the C ABI
    n, w = rows.shape
    stream = torch.cuda.current_stream().cuda_stream
    return pg.load().pg_merkle_build_noalloc(ctypes.c_void_p(rows.data_ptr()), n, w,
                                              ctypes.c_void_p(nodes.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_matches_merkle_build_two_calls_in_a_row():
    cases = [(1 << 14, 8, 0x11), (1 << 12, 24, 0x22)]
    outs = []
    for n, w, seed in cases:
        rows = _dev(pg_synth.matrix(seed, n, w))
        nodes = torch.full((2 * n - 1, 4), -1, dtype=torch.int64, device="cuda")
        assert _noalloc_raw(rows, nodes) == 0, pg.last_error()
        outs.append((rows, nodes))
    for rows, nodes in outs:
        want = pg.merkle_build(rows)
        torch.cuda.synchronize()
        assert torch.equal(nodes, want)


def test_noalloc_repeated_same_input_is_stable_at_the_limit():
    n, w = 1 << 22, 8  # the largest tree the fixed scratch array serves
    rows = _dev(pg_synth.matrix(0x33, n, w))
    a = torch.empty((2 * n - 1, 4), dtype=torch.int64, device="cuda")
    b = torch.empty_like(a)
    assert _noalloc_raw(rows, a) == 0
    assert _noalloc_raw(rows, b) == 0
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.equal(a, pg.merkle_build(rows))


def test_noalloc_rejects_more_than_the_limit():
    # checked on the host before anything is launched
    n = (1 << 22) * 2
    rows = torch.empty((1, 8), dtype=torch.int64, device="cuda")
    nodes = torch.empty((1, 4), dtype=torch.int64, device="cuda")
    status = pg.load().pg_merkle_build_noalloc(ctypes.c_void_p(rows.data_ptr()), n, 8,
                                                ctypes.c_void_p(nodes.data_ptr()), None)
    assert status == 1
    assert "limit" in pg.last_error()


_FRESH = r"""
import ctypes, sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
import oracle, pg_synth
import paper_2506_09505_gb300 as pg
lib = pg.load()
rows_np = pg_synth.matrix(0x44, 1 << 10, 8)
rows = torch.from_numpy(rows_np.view(np.int64)).cuda()
nodes = torch.full((2047, 4), -1, dtype=torch.int64, device="cuda")
# first call of the process: no pg_init() before it
st = lib.pg_merkle_build_noalloc(ctypes.c_void_p(rows.data_ptr()), 1 << 10, 8,
                                 ctypes.c_void_p(nodes.data_ptr()), ctypes.c_void_p(0))
assert st == 0, pg.last_error()
torch.cuda.synchronize()
got = nodes.cpu().numpy().view(np.uint64)
assert (got == oracle.merkle_build(rows_np, nthreads=4)).all()
# a second call, then the allocating entry point after pg_init, agree
again = torch.empty_like(nodes)
assert lib.pg_merkle_build_noalloc(ctypes.c_void_p(rows.data_ptr()), 1 << 10, 8,
                                   ctypes.c_void_p(again.data_ptr()), ctypes.c_void_p(0)) == 0
pg.init(0)
assert torch.equal(again, nodes) and torch.equal(pg.merkle_build(rows), nodes)
print("fresh-process no-alloc ok")
"""


def test_noalloc_in_a_fresh_process_without_pg_init():
    # the promise that the entry point needs no pg_init(): its own set-up
    # (constant tables, scratch address) runs on the first call
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _FRESH.format(root=root)], capture_output=True, text=True,
                         timeout=600, cwd=root)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]
    assert "fresh-process no-alloc ok" in out.stdout
