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
