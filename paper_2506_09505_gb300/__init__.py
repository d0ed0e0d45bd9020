"""GB300 Poseidon-12 / Goldilocks Merkle library -- Python binding.

Thin ctypes marshalling over the C ABI of ``include/pg12.h`` (the in-tree
``libpg12.so``).  Every step of the hash path runs in the library's CUDA
kernels; PyTorch only supplies device memory and streams.  There is no CPU
fallback: if the shared object is missing or cannot be loaded, every call
raises.

Tensors are 64-bit words on the GPU (``torch.int64`` or ``torch.uint64``,
C-contiguous); the bits are the Goldilocks words of the ABI.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

P = 0xFFFFFFFF00000001
T = 12
DIGEST = 4

PG_OK = 0
_STATUS = {
    0: "PG_OK", 1: "PG_ERR_INVALID_ARG", 2: "PG_ERR_NOT_POW2", 3: "PG_ERR_OOM",
    4: "PG_ERR_CUDA", 5: "PG_ERR_TIMEOUT", 6: "PG_ERR_PARAMS", 7: "PG_ERR_NOT_INIT",
}


class PGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_u64p = ctypes.POINTER(ctypes.c_uint64)


class Tree(ctypes.Structure):
    """pg_tree of include/pg12.h."""
    _fields_ = [("rows", ctypes.c_void_p), ("n_leaves", ctypes.c_uint64), ("width", ctypes.c_uint64),
                ("nodes", ctypes.c_void_p)]


class Schedule(ctypes.Structure):
    """pg_schedule of include/pg12.h."""
    _fields_ = [("block", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32), ("order", ctypes.c_uint32),
                ("engine", ctypes.c_uint32), ("fuse_levels", ctypes.c_uint32), ("top_lanes", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 2)]

    KEYS = ("block", "blocks_per_sm", "order", "engine", "fuse_levels", "top_lanes")

    def as_dict(self):
        return {k: int(getattr(self, k)) for k in self.KEYS}

    @classmethod
    def of(cls, d):
        sc = cls()
        for k, v in (d or {}).items():
            if k not in cls.KEYS:
                raise ValueError(f"unknown schedule field {k!r}")
            setattr(sc, k, int(v))
        return sc


BATCH_ENGINE_DEFAULT, BATCH_ENGINE_INT, BATCH_ENGINE_TENSOR = 0, 1, 2

class ServerConfig(ctypes.Structure):
    """pg_server_config of include/pg12.h."""
    _fields_ = [("pool_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("sched", Schedule)]


class RequestInfo(ctypes.Structure):
    """pg_request_info of include/pg12.h."""
    _fields_ = [("state", ctypes.c_int32), ("batch_size", ctypes.c_int32), ("submit_s", ctypes.c_double),
                ("launch_s", ctypes.c_double), ("done_s", ctypes.c_double), ("nodes", ctypes.c_void_p)]


class KernelTime(ctypes.Structure):
    """pg_kernel_time of include/pg12.h."""
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("perms", ctypes.c_uint64),
                ("total_ms", ctypes.c_double)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3

# name -> (restype, argtypes) for every symbol declared in include/pg12.h
SIGNATURES = {
    "pg_version": (ctypes.c_char_p, []),
    "pg_last_error": (ctypes.c_char_p, []),
    "pg_init": (ctypes.c_int, [ctypes.c_int, ctypes.c_char_p]),
    "pg_params_select": (ctypes.c_int, [ctypes.c_char_p]),
    "pg_params_name": (ctypes.c_char_p, []),
    "pg_set_engine": (ctypes.c_int, [ctypes.c_int]),
    "pg_tc_tables_export": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_size_t]),
    "pg_params_export_chain": (ctypes.c_int, [_u64p, _u64p, _u64p]),
    "pg_get_engine": (ctypes.c_int, []),
    "pg_device_faults": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
    "pg_shutdown": (ctypes.c_int, []),
    "pg_params_export": (ctypes.c_int, [_u64p, _u64p]),
    "pg_params_export_optimized": (ctypes.c_int, [_u64p] * 6),
    "pg_permute_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "pg_hash_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "pg_merkle_build": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                       ctypes.c_void_p, _u64p, ctypes.c_void_p]),
    "pg_merkle_build_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "pg_merkle_build_batch": (ctypes.c_int, [ctypes.POINTER(Tree), ctypes.c_size_t,
                                             ctypes.POINTER(Schedule), ctypes.c_void_p]),
    "pg_batch_graph_create": (ctypes.c_int, [ctypes.POINTER(Tree), ctypes.c_size_t,
                                             ctypes.POINTER(Schedule), ctypes.POINTER(ctypes.c_void_p)]),
    "pg_batch_graph_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pg_batch_graph_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pg_batch_autotune": (ctypes.c_int, [ctypes.POINTER(Tree), ctypes.c_size_t, ctypes.c_void_p,
                                         ctypes.POINTER(Schedule), ctypes.POINTER(ctypes.c_float)]),
    "pg_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]),
    "pg_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "pg_server_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(RequestInfo)]),
    "pg_server_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "pg_server_drain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "pg_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pg_merkle_open": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "pg_merkle_verify": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pg_field_eval": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.c_void_p]),
    "pg_field_bench": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]),
    "pg_merkle_build_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_void_p,
                                            ctypes.c_void_p, _u64p, ctypes.c_void_p]),
    "pg_params_sha256": (ctypes.c_char_p, []),
    "pg_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Tree), ctypes.c_size_t]),
    "pg_ntt": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]),
    "pg_lde": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_uint32,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pg_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "pg_profile_read": (ctypes.c_int, [ctypes.POINTER(KernelTime), ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_uint64)]),
}

OPS = {"add": 1, "sub": 2, "mul": 3, "sqr": 4, "reduce": 5, "mul_small": 6, "sbox": 7, "dot12": 8,
       "pipe_imad": 9, "pipe_imad_wide": 10, "pipe_iadd": 11,
       "lat_mul": 12, "lat_sbox": 13, "lat_dot12": 14, "lat_perm": 15, "lat_perm_wide": 16}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libpg12.so (optionally compiling it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"{_build.LIB} is missing: run paper_2506_09505_gb300._build.build() "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().pg_last_error().decode()


def _check(status: int) -> None:
    if status != PG_OK:
        raise PGError(status, last_error())


def version() -> str:
    return load().pg_version().decode()


# ------------------------------------------------------------ host-only calls

def params_export():
    """Plain parameter set (rc[30,12], mds[12,12]) as generated by the library."""
    rc = np.zeros((30, T), dtype=np.uint64)
    mds = np.zeros((T, T), dtype=np.uint64)
    _check(load().pg_params_export(rc.ctypes.data_as(_u64p), mds.ctypes.data_as(_u64p)))
    return rc, mds


def params_export_optimized():
    """Optimised-form constants the kernels use (see include/pg12.h)."""
    full_rc = np.zeros((8, T), dtype=np.uint64)
    mds = np.zeros((T, T), dtype=np.uint64)
    pre = np.zeros((T, T), dtype=np.uint64)
    part_rc = np.zeros(22, dtype=np.uint64)
    part_v = np.zeros((22, T), dtype=np.uint64)
    part_w = np.zeros((22, T - 1), dtype=np.uint64)
    arrs = (full_rc, mds, pre, part_rc, part_v, part_w)
    _check(load().pg_params_export_optimized(*[a.ctypes.data_as(_u64p) for a in arrs]))
    return dict(full_rc=full_rc, mds=mds, pre=pre, part_rc=part_rc, part_v=part_v, part_w=part_w)


# ------------------------------------------------------------ device calls

def init(device: int = 0, params: str | None = None) -> None:
    """pg_init on `device` with a built-in parameter set (None = pg12_v1)."""
    _check(load().pg_init(int(device), params.encode() if params else None))


def params_select(name: str | None) -> None:
    _check(load().pg_params_select(name.encode() if name else None))


def params_name() -> str:
    return load().pg_params_name().decode()


def shutdown() -> None:
    _check(load().pg_shutdown())


ENGINE_INT, ENGINE_TENSOR = 0, 1


def set_engine(engine: int) -> None:
    """Permutation engine of later launches: ENGINE_TENSOR (default, the
    linear layers as exact tensor-core contractions) or ENGINE_INT (integer
    pipes only)."""
    _check(load().pg_set_engine(int(engine)))


def get_engine() -> int:
    return int(load().pg_get_engine())


def params_export_chain():
    """Unrolled partial rounds: (vp[22,12], beta[22,22], w[12,22]) (see include/pg12.h)."""
    vp = np.zeros((22, T), dtype=np.uint64)
    beta = np.zeros((22, 22), dtype=np.uint64)
    w = np.zeros((T, 22), dtype=np.uint64)
    _check(load().pg_params_export_chain(vp.ctypes.data_as(_u64p), beta.ctypes.data_as(_u64p),
                                         w.ctypes.data_as(_u64p)))
    return vp, beta, w


def tc_tables_export() -> bytes:
    """The tensor-core digit tables of the active parameter set (see include/pg12.h)."""
    n = int(load().pg_tc_tables_export(None, 0))
    buf = ctypes.create_string_buffer(n)
    if int(load().pg_tc_tables_export(buf, n)) != n:
        raise PGError(6, "tensor-core tables unavailable: " + last_error())
    return buf.raw


def device_faults() -> int:
    """1 if a tensor-core wait ran out since the last call (then cleared), else 0."""
    v = ctypes.c_uint32(0)
    _check(load().pg_device_faults(ctypes.byref(v)))
    return int(v.value)


def _dev_ptr(t, name: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in (torch.int64, torch.uint64):
        raise TypeError(f"{name} must hold 64-bit words (int64/uint64), got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def permute_batch(states, stream=None):
    """Alg. 1 on every row of a (n, 12) CUDA tensor, in place; returns it."""
    if states.dim() != 2 or states.shape[1] != T:
        raise ValueError("states must have shape (n, 12)")
    _check(load().pg_permute_batch(_dev_ptr(states, "states"), states.shape[0], _stream(stream)))
    return states


def hash_rows(rows, digests=None, stream=None):
    """Sponge digest of every row of a (n, w) CUDA tensor -> (n, 4)."""
    import torch
    if rows.dim() != 2:
        raise ValueError("rows must have shape (n, w)")
    n, w = rows.shape
    if digests is None:
        digests = torch.empty((n, DIGEST), dtype=rows.dtype, device=rows.device)
    _check(load().pg_hash_rows(_dev_ptr(rows, "rows"), n, w, _dev_ptr(digests, "digests"),
                               _stream(stream)))
    return digests


def _check_nodes(nodes, n: int, rows) -> None:
    """A caller-supplied node buffer must hold the whole tree on the rows' GPU:
    the kernels write (2N-1) x 4 words into it and cannot check its size."""
    need = 4 * (2 * n - 1) if n > 0 else 0
    if nodes.numel() < need:
        raise ValueError(f"nodes holds {nodes.numel()} words; a tree of {n} leaves needs {need}")
    if nodes.device != rows.device:
        raise ValueError(f"nodes is on {nodes.device}, rows on {rows.device}")
    _dev_ptr(nodes, "nodes")


def merkle_build(rows, nodes=None, want_root: bool = False, stream=None):
    """Whole tree over a (N, w) CUDA tensor -> nodes (2N-1, 4), level-major.

    With ``want_root`` the call synchronises the stream and also returns the
    root as four Python ints.
    """
    import torch
    if rows.dim() != 2:
        raise ValueError("rows must have shape (N, w)")
    n, w = rows.shape
    if nodes is None:
        nodes = torch.empty((max(2 * n - 1, 1), DIGEST), dtype=rows.dtype, device=rows.device)
    else:
        _check_nodes(nodes, n, rows)
    root = (ctypes.c_uint64 * 4)() if want_root else None
    _check(load().pg_merkle_build(_dev_ptr(rows, "rows"), n, w, _dev_ptr(nodes, "nodes"),
                                  ctypes.cast(root, _u64p) if want_root else None,
                                  _stream(stream)))
    if want_root:
        return nodes, [int(v) for v in root]
    return nodes


def merkle_build_host(rows_host, rows_dev=None, nodes=None, want_root: bool = False, stream=None):
    """Tree over the (N, w) int64 rows of a host tensor (page-locked for overlap): the rows are
    copied into ``rows_dev`` (a CUDA staging tensor of the same shape, allocated when not given)
    in chunks while earlier chunks are hashed.  Returns nodes, or (nodes, root) with want_root."""
    import torch
    if rows_host.dim() != 2 or rows_host.is_cuda:
        raise ValueError("rows_host must be a (N, w) host tensor")
    if rows_host.dtype not in (torch.int64, torch.uint64) or not rows_host.is_contiguous():
        raise TypeError("rows_host must be a contiguous 64-bit tensor")
    n, w = rows_host.shape
    if rows_dev is None:
        rows_dev = torch.empty((n, w), dtype=rows_host.dtype, device="cuda")
    if tuple(rows_dev.shape) != (n, w):
        raise ValueError("rows_dev must have the shape of rows_host")
    if nodes is None:
        nodes = torch.empty((2 * n - 1, DIGEST), dtype=torch.int64, device=rows_dev.device)
    root = (ctypes.c_uint64 * 4)() if want_root else None
    _check(load().pg_merkle_build_host(rows_host.data_ptr(), n, w, _dev_ptr(rows_dev, "rows_dev"),
                                       _dev_ptr(nodes, "nodes"),
                                       ctypes.cast(root, _u64p) if want_root else None, _stream(stream)))
    if want_root:
        return nodes, [int(v) for v in root]
    return nodes


def merkle_build_noalloc(rows, nodes, stream=None):
    """Allocation-free variant of merkle_build (at most 2^22 leaves).

    For callers that cannot allocate device memory: the caller passes both
    buffers and the library uses only a fixed scratch array it owns.
    """
    if rows.dim() != 2:
        raise ValueError("rows must have shape (N, w)")
    n, w = rows.shape
    _check_nodes(nodes, n, rows)
    _check(load().pg_merkle_build_noalloc(_dev_ptr(rows, "rows"), n, w, _dev_ptr(nodes, "nodes"),
                                          _stream(stream)))
    return nodes


def _trees(rows_list, nodes_list):
    arr = (Tree * len(rows_list))()
    for k, (r, nd) in enumerate(zip(rows_list, nodes_list)):
        if r.dim() != 2:
            raise ValueError("rows must have shape (N, w)")
        arr[k].rows = _dev_ptr(r, "rows")
        arr[k].n_leaves = r.shape[0]
        arr[k].width = r.shape[1]
        arr[k].nodes = _dev_ptr(nd, "nodes")
    return arr


def _sched(schedule):
    if schedule is None:
        return None
    if isinstance(schedule, Schedule):
        return ctypes.byref(schedule)
    return ctypes.byref(Schedule.of(schedule))


def alloc_nodes(rows_list):
    import torch
    return [torch.empty((2 * r.shape[0] - 1, DIGEST), dtype=r.dtype, device=r.device) for r in rows_list]


def merkle_build_batch(rows_list, nodes_list=None, schedule=None, stream=None):
    """Many trees (list of (N_k, w_k) CUDA tensors) in one persistent launch."""
    if nodes_list is None:
        nodes_list = alloc_nodes(rows_list)
    arr = _trees(rows_list, nodes_list)
    _check(load().pg_merkle_build_batch(arr, len(rows_list), _sched(schedule), _stream(stream)))
    return nodes_list


class BatchGraph:
    """A batch captured once into a CUDA graph and replayed with launch()."""

    def __init__(self, rows_list, nodes_list=None, schedule=None):
        self.rows = list(rows_list)
        self.nodes = nodes_list if nodes_list is not None else alloc_nodes(self.rows)
        self._arr = _trees(self.rows, self.nodes)
        self._h = ctypes.c_void_p()
        _check(load().pg_batch_graph_create(self._arr, len(self.rows), _sched(schedule),
                                            ctypes.byref(self._h)))

    def launch(self, stream=None):
        _check(load().pg_batch_graph_launch(self._h, _stream(stream)))
        return self.nodes

    def close(self):
        if self._h:
            _check(load().pg_batch_graph_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_autotune(rows_list, nodes_list=None, stream=None):
    """Fastest schedule for this batch: (schedule dict, milliseconds)."""
    if nodes_list is None:
        nodes_list = alloc_nodes(rows_list)
    arr = _trees(rows_list, nodes_list)
    best = Schedule()
    ms = ctypes.c_float()
    _check(load().pg_batch_autotune(arr, len(rows_list), _stream(stream), ctypes.byref(best),
                                    ctypes.byref(ms)))
    return best.as_dict(), float(ms.value)


def merkle_open(nodes, n_leaves: int, indices, stream=None):
    """Authentication paths (k, log2 N, 4) of the leaves in `indices` (int64 CUDA tensor)."""
    import torch
    depth = int(n_leaves).bit_length() - 1
    k = indices.numel()
    paths = torch.empty((k, depth, DIGEST), dtype=torch.int64, device=nodes.device)
    _check(load().pg_merkle_open(_dev_ptr(nodes, "nodes"), n_leaves, _dev_ptr(indices, "indices"), k,
                                 paths.data_ptr() if paths.numel() else None, _stream(stream)))
    return paths


def merkle_verify(root, n_leaves: int, leaves, indices, paths, stream=None):
    """Bool tensor: does each (leaf digest, index, path) reproduce `root`?"""
    import torch
    k = indices.numel()
    ok = torch.zeros(k, dtype=torch.uint8, device=indices.device)
    _check(load().pg_merkle_verify(_dev_ptr(root, "root"), n_leaves, _dev_ptr(leaves, "leaves"),
                                   _dev_ptr(indices, "indices"), k,
                                   paths.data_ptr() if paths.numel() else None, ok.data_ptr(), _stream(stream)))
    return ok.bool()


def field_eval(op: str, a, b=None, stream=None):
    """Element-wise field operation on CUDA tensors (canonical result)."""
    import torch
    out = torch.empty_like(a)
    _check(load().pg_field_eval(OPS[op], _dev_ptr(a, "a"), _dev_ptr(b, "b") if b is not None else None,
                                _dev_ptr(out, "out"), a.numel(), _stream(stream)))
    return out


def field_bench(op: str):
    """(results per second, results per SM clock) of one field operation; for the
    ``lat_*`` ops, (operations per second of one dependent chain, cycles per operation)."""
    rate, per_clk = ctypes.c_double(), ctypes.c_double()
    _check(load().pg_field_bench(OPS[op], ctypes.byref(rate), ctypes.byref(per_clk)))
    return rate.value, per_clk.value


def ntt(data, inverse: bool = False, stream=None):
    """In-place NTT (or inverse) of every column of a (n, ncols) CUDA tensor."""
    if data.dim() != 2:
        raise ValueError("data must have shape (n, ncols)")
    _check(load().pg_ntt(_dev_ptr(data, "data"), data.shape[0], data.shape[1], 1 if inverse else 0,
                         _stream(stream)))
    return data


def lde(evals, log_blowup: int, out=None, scratch=None, stream=None):
    """Low-degree extension of the (n, ncols) CUDA tensor ``evals`` onto the
    coset 7 * <w_N>, N = n * 2^log_blowup -> (N, ncols).  ``scratch`` (n, ncols)
    is allocated when not given; pass ``evals`` to work in place."""
    import torch
    if evals.dim() != 2:
        raise ValueError("evals must have shape (n, ncols)")
    n, c = evals.shape
    if out is None:
        out = torch.empty((n << log_blowup, c), dtype=evals.dtype, device=evals.device)
    if scratch is None:
        scratch = torch.empty_like(evals)
    _check(load().pg_lde(_dev_ptr(evals, "evals"), n, c, log_blowup, _dev_ptr(out, "out"),
                         _dev_ptr(scratch, "scratch"), _stream(stream)))
    return out


def params_sha256() -> str:
    """SHA-256 (hex) of the active plain parameter set: rc[30][12] then mds[12][12], little-endian words."""
    h = load().pg_params_sha256()
    if not h:
        raise RuntimeError(last_error())
    return h.decode()


def workspace_bytes(rows_list=None, nodes_list=None) -> int:
    """Workspace bytes a batch of trees needs (None: the size pg_init allocates)."""
    if rows_list is None:
        return int(load().pg_workspace_bytes(None, 0))
    arr = _trees(rows_list, nodes_list if nodes_list is not None else alloc_nodes(rows_list))
    return int(load().pg_workspace_bytes(arr, len(rows_list)))


def profile_enable(on: bool = True) -> None:
    """Start (or stop) event timing of every launch; discards earlier records."""
    _check(load().pg_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """Per-kernel launches, permutations and summed event time since the last
    enable/read: {name: {"launches", "perms", "total_ms"}} plus "_dropped"."""
    n, dropped = ctypes.c_size_t(), ctypes.c_uint64()
    cap = 16
    arr = (KernelTime * cap)()
    _check(load().pg_profile_read(arr, cap, ctypes.byref(n), ctypes.byref(dropped)))
    out = {arr[k].name.decode(): {"launches": int(arr[k].launches), "perms": int(arr[k].perms),
                                  "total_ms": float(arr[k].total_ms)} for k in range(n.value)}
    out["_dropped"] = int(dropped.value)
    return out


class Server:
    """Continuous-batching tree-build server (pg_server_* of include/pg12.h)."""

    def __init__(self, pool_bytes=0, max_batch=0, max_inflight=0, schedule=None):
        cfg = ServerConfig(pool_bytes, max_batch, max_inflight, Schedule.of(schedule))
        self._h = ctypes.c_void_p()
        _check(load().pg_server_create(ctypes.byref(cfg), ctypes.byref(self._h)))

    def submit(self, rows) -> int:
        """Queue a build of the (N, w) CUDA tensor ``rows`` (kept alive by the caller)."""
        rid = ctypes.c_uint64()
        _check(load().pg_server_submit(self._h, _dev_ptr(rows, "rows"), rows.shape[0], rows.shape[1],
                                       ctypes.byref(rid)))
        return int(rid.value)

    def query(self, rid: int) -> dict:
        info = RequestInfo()
        _check(load().pg_server_query(self._h, rid, ctypes.byref(info)))
        return {"state": info.state, "batch_size": info.batch_size, "submit_s": info.submit_s,
                "launch_s": info.launch_s, "done_s": info.done_s, "nodes": info.nodes}

    def nodes(self, rid: int, n_leaves: int):
        """The finished request's node buffer as a (2N-1, 4) int64 CUDA tensor.

        A view of the server's pool (no copy): valid until release(rid).
        """
        import torch
        info = self.query(rid)
        if info["state"] != REQ_DONE:
            raise RuntimeError(f"request {rid} is not done (state {info['state']})")
        view = _DeviceView(info["nodes"], (2 * n_leaves - 1, DIGEST))
        return torch.as_tensor(view, device="cuda")

    def release(self, rid: int) -> None:
        _check(load().pg_server_release(self._h, rid))

    def drain(self, timeout_s: float = 60.0) -> None:
        _check(load().pg_server_drain(self._h, timeout_s))

    def close(self) -> None:
        if self._h:
            _check(load().pg_server_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DeviceView:
    """Exposes a raw device pointer to torch through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<i8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def level_offsets(n_leaves: int):
    """Start row of every level inside the level-major node array."""
    offs, base, cnt = [], 0, n_leaves
    while True:
        offs.append(base)
        if cnt == 1:
            return offs
        base += cnt
        cnt //= 2
