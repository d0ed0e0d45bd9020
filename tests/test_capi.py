"""The C-ABI shared library loads and exports every symbol of include/pg12.h.

No compute call is made here (no GPU); calls that need a device must fail
with a status, not crash, when the library is not initialised.
"""
import ctypes
import os
import re

import pytest

pg = pytest.importorskip("paper_2506_09505_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "pg12.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"\b(pg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    try:
        return pg.load(build_if_missing=True)
    except Exception as e:  # pragma: no cover
        pytest.skip(f"library unavailable: {e}")


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pg_merkle_build" in names and "pg_permute_batch" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in pg.SIGNATURES, f"binding lacks {name}"


def test_version_and_errors(lib):
    assert pg.version().startswith("pg12")
    assert isinstance(pg.last_error(), str)


def test_device_calls_refuse_before_init(lib):
    # never touches the GPU: the library reports PG_ERR_NOT_INIT on the host
    raw = pg.load()
    assert raw.pg_permute_batch(ctypes.c_void_p(0x1000), 1, None) == 7
    assert raw.pg_hash_rows(ctypes.c_void_p(0x1000), 1, 8, ctypes.c_void_p(0x2000), None) == 7
    assert raw.pg_merkle_build(ctypes.c_void_p(0x1000), 4, 8, ctypes.c_void_p(0x2000), None, None) == 7
    assert "pg_init" in pg.last_error()


def test_init_rejects_external_params(lib):
    assert pg.load().pg_init(0, b"/nonexistent") == 6


def test_profile_store_empty_on_host(lib):
    # with nothing recorded, enabling and reading the launch-timing store
    # makes no CUDA call
    pg.profile_enable(True)
    got = pg.profile_read()
    pg.profile_enable(False)
    assert got == {"_dropped": 0}


def test_undersized_node_buffers_are_refused_before_any_launch():
    # the kernels write (2N-1) x 4 words and cannot check the buffer, so the
    # binding refuses a short one (or one on another device) before calling
    # the library
    torch = pytest.importorskip("torch")
    rows = torch.zeros((1 << 10, 8), dtype=torch.int64)
    short = torch.zeros((2 * (1 << 10) - 2, 4), dtype=torch.int64)
    with pytest.raises(ValueError, match="needs"):
        pg.merkle_build_noalloc(rows, short)
    with pytest.raises(ValueError, match="needs"):
        pg.merkle_build(rows, short)
    meta = torch.zeros((2 * (1 << 10) - 1, 4), dtype=torch.int64, device="meta")
    with pytest.raises(ValueError, match="meta"):
        pg.merkle_build_noalloc(rows, meta)


def test_engine_switch_is_validated(lib):
    assert pg.get_engine() in (pg.ENGINE_INT, pg.ENGINE_TENSOR)
    before = pg.get_engine()
    pg.set_engine(pg.ENGINE_INT)
    assert pg.get_engine() == pg.ENGINE_INT
    pg.set_engine(before)
    with pytest.raises(pg.PGError) as e:
        pg.set_engine(7)
    assert e.value.status == 1
    assert pg.get_engine() == before
