"""CPU oracle for the Poseidon-12 / Goldilocks Merkle path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it.  The arithmetic lives in ``pg_oracle.c`` and
``ntt_oracle.c`` (plain ``unsigned __int128`` products followed by ``% p``);
this module only loads that shared object with ctypes and marshals numpy
arrays.

Functions follow arXiv 2506.09505: Eq. 1 (the field), Alg. 1 and Sec. 2.4
(the permutation and the sponge), Sec. 2.4 / Sec. 4.2 (the Merkle tree), and
the textbook NTT / low-degree extension behind the Sec. 2.3 NTT hotspot.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

P = 0xFFFFFFFF00000001  # Eq. 1
T = 12
ROUNDS = 30

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "pg_oracle.c"), os.path.join(_HERE, "ntt_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into liboracle.so (plain gcc, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               *_SRCS, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u64, sz, i = ctypes.c_uint64, ctypes.c_size_t, ctypes.c_int
    sig = {
        "orc_canon": (u64, [u64]),
        "orc_add": (u64, [u64, u64]),
        "orc_sub": (u64, [u64, u64]),
        "orc_mul": (u64, [u64, u64]),
        "orc_pow": (u64, [u64, u64]),
        "orc_inv": (u64, [u64]),
        "orc_field_many": (i, [i, _u64p, _u64p, _u64p, sz]),
        "orc_sbox_inverse_exponent": (u64, []),
        "orc_mat_inverse": (i, [_u64p, _u64p, i]),
        "orc_mat_det": (u64, [_u64p, i]),
        "orc_grain_words": (None, [i, i, i, i, i, i, i, _u64p, sz]),
        "orc_params_generate": (i, [_u64p, _u64p, _u64p, _u64p]),
        "orc_permute": (None, [_u64p, _u64p, _u64p]),
        "orc_permute_inverse": (None, [_u64p, _u64p, _u64p]),
        "orc_permute_many": (None, [_u64p, _u64p, _u64p, sz]),
        "orc_permute_many_mt": (None, [_u64p, _u64p, _u64p, sz, i]),
        "orc_hash_row": (None, [_u64p, _u64p, _u64p, sz, _u64p]),
        "orc_hash_pair": (None, [_u64p, _u64p, _u64p, _u64p, _u64p]),
        "orc_merkle_build": (i, [_u64p, _u64p, _u64p, sz, sz, _u64p, i]),
        "orc_auth_path": (i, [_u64p, sz, sz, _u64p]),
        "orc_root_from_path": (None, [_u64p, _u64p, _u64p, sz, _u64p, sz, _u64p]),
        "orc_count_singular_minors": (ctypes.c_long, [_u64p, ctypes.POINTER(ctypes.c_long)]),
        "orc_is_mds": (i, [_u64p]),
        "orc_params_generate_small": (i, [_u64p, _u64p, _u64p]),
        "orc_two_adic_root": (u64, [i, i]),
        "orc_dft_naive": (i, [_u64p, _u64p, sz, i]),
        "orc_fft": (i, [_u64p, sz, i]),
        "orc_ntt_columns": (i, [_u64p, sz, sz, i]),
        "orc_poly_eval": (u64, [_u64p, sz, u64]),
        "orc_interpolate_columns": (i, [_u64p, sz, sz, _u64p]),
        "orc_lde_columns": (i, [_u64p, sz, sz, i, u64, _u64p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags.c_contiguous
    return a.ctypes.data_as(_u64p)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


# ----------------------------------------------------------------- field (Eq. 1)

def add(a: int, b: int) -> int:
    return int(_load().orc_add(a, b))


def sub(a: int, b: int) -> int:
    return int(_load().orc_sub(a, b))


def mul(a: int, b: int) -> int:
    return int(_load().orc_mul(a, b))


FIELD_MANY_OPS = {"add": 1, "sub": 2, "mul": 3, "sqr": 4, "sbox": 5}


def field_many(op: str, a, b=None) -> np.ndarray:
    """Element-wise add / sub / mul / sqr / sbox (x^7) over arrays of words, canonical (Eq. 1)."""
    a = _u64(a)
    b = _u64(b) if b is not None else a
    assert a.shape == b.shape
    out = np.empty_like(a)
    if _load().orc_field_many(FIELD_MANY_OPS[op], _ptr(a), _ptr(b), _ptr(out), a.size) != 0:
        raise ValueError(op)
    return out


def pow_(a: int, e: int) -> int:
    return int(_load().orc_pow(a, e))


def inv(a: int) -> int:
    return int(_load().orc_inv(a))


def canon(a: int) -> int:
    return int(_load().orc_canon(a))


def sbox_inverse_exponent() -> int:
    return int(_load().orc_sbox_inverse_exponent())


def mat_inverse(m) -> np.ndarray:
    m = _u64(m)
    n = m.shape[0]
    out = np.zeros((n, n), dtype=np.uint64)
    rc = _load().orc_mat_inverse(_ptr(m), _ptr(out), n)
    if rc != 0:
        raise ValueError("singular matrix")
    return out


def count_singular_minors(m):
    """(singular, checked) over every square submatrix of a 12x12 matrix."""
    m = _u64(m)
    checked = ctypes.c_long(0)
    bad = _load().orc_count_singular_minors(_ptr(m), ctypes.byref(checked))
    return int(bad), int(checked.value)


def mat_det(m) -> int:
    m = _u64(m)
    return int(_load().orc_mat_det(_ptr(m), m.shape[0]))


# ------------------------------------------------------------------ parameters

def grain_words(field: int, sbox: int, n: int, t: int, rf: int, rp: int, nbits: int,
                count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint64)
    _load().orc_grain_words(field, sbox, n, t, rf, rp, nbits, _ptr(out), count)
    return out


_PARAMS = None


def params():
    """Parameter set pg12_v1: (rc[30,12], mds[12,12], xs[12], ys[12], redraws)."""
    global _PARAMS
    if _PARAMS is None:
        rc = np.zeros((ROUNDS, T), dtype=np.uint64)
        mds = np.zeros((T, T), dtype=np.uint64)
        xs = np.zeros(T, dtype=np.uint64)
        ys = np.zeros(T, dtype=np.uint64)
        redraws = _load().orc_params_generate(_ptr(rc), _ptr(mds), _ptr(xs), _ptr(ys))
        for a in (rc, mds, xs, ys):
            a.setflags(write=False)
        _PARAMS = (rc, mds, xs, ys, int(redraws))
    return _PARAMS


_PARAMS_SMALL = None


def params_small():
    """Parameter set pg12_small: (rc[30,12], mds[12,12], first circulant row[12], candidate index)."""
    global _PARAMS_SMALL
    if _PARAMS_SMALL is None:
        rc = np.zeros((ROUNDS, T), dtype=np.uint64)
        mds = np.zeros((T, T), dtype=np.uint64)
        row = np.zeros(T, dtype=np.uint64)
        cand = _load().orc_params_generate_small(_ptr(rc), _ptr(mds), _ptr(row))
        for a in (rc, mds, row):
            a.setflags(write=False)
        _PARAMS_SMALL = (rc, mds, row, int(cand))
    return _PARAMS_SMALL


def is_mds(m) -> bool:
    return bool(_load().orc_is_mds(_ptr(_u64(m))))


def _rc_mds(rc, mds):
    if rc is None or mds is None:
        prc, pmds = params()[:2]
        rc = prc if rc is None else rc
        mds = pmds if mds is None else mds
    return _u64(rc), _u64(mds)


# ---------------------------------------------------------------- permutation

def permute(states, rc=None, mds=None, nthreads: int = 1) -> np.ndarray:
    """Plain-form Poseidon-12 on an array of states shaped (..., 12)."""
    rc, mds = _rc_mds(rc, mds)
    st = _u64(states).copy()
    flat = st.reshape(-1, T)
    if nthreads > 1:
        _load().orc_permute_many_mt(_ptr(rc), _ptr(mds), _ptr(flat), flat.shape[0], nthreads)
    else:
        _load().orc_permute_many(_ptr(rc), _ptr(mds), _ptr(flat), flat.shape[0])
    return flat.reshape(st.shape)


def permute_inverse(states, rc=None, mds=None) -> np.ndarray:
    rc, mds = _rc_mds(rc, mds)
    minv = mat_inverse(mds)
    st = _u64(states).copy()
    flat = st.reshape(-1, T)
    lib = _load()
    for k in range(flat.shape[0]):
        row = np.ascontiguousarray(flat[k])
        lib.orc_permute_inverse(_ptr(rc), _ptr(minv), _ptr(row))
        flat[k] = row
    return flat.reshape(st.shape)


# --------------------------------------------------------------- sponge / tree

def hash_rows(rows, rc=None, mds=None) -> np.ndarray:
    """Sponge digest of every row of a (n, w) array -> (n, 4)."""
    rc, mds = _rc_mds(rc, mds)
    rows = _u64(rows)
    n, w = rows.shape
    out = np.zeros((n, 4), dtype=np.uint64)
    lib = _load()
    for k in range(n):
        r = rows[k]
        lib.orc_hash_row(_ptr(rc), _ptr(mds), _ptr(r), w, _ptr(out[k]))
    return out


def hash_pair(left, right, rc=None, mds=None) -> np.ndarray:
    rc, mds = _rc_mds(rc, mds)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_hash_pair(_ptr(rc), _ptr(mds), _ptr(_u64(left)), _ptr(_u64(right)), _ptr(out))
    return out


def merkle_build(rows, nthreads: int = 1, rc=None, mds=None) -> np.ndarray:
    """All (2N-1) nodes, level-major, root last, shape (2N-1, 4)."""
    rc, mds = _rc_mds(rc, mds)
    rows = _u64(rows)
    n, w = rows.shape
    nodes = np.zeros((2 * n - 1, 4), dtype=np.uint64)
    rcode = _load().orc_merkle_build(_ptr(rc), _ptr(mds), _ptr(rows), n, w, _ptr(nodes), nthreads)
    if rcode != 0:
        raise ValueError("number of leaves must be a power of two")
    return nodes


def auth_path(nodes, n_leaves: int, index: int) -> np.ndarray:
    nodes = _u64(nodes)
    depth = int(n_leaves).bit_length() - 1
    path = np.zeros((max(depth, 1), 4), dtype=np.uint64)
    if _load().orc_auth_path(_ptr(nodes), n_leaves, index, _ptr(path)) != 0:
        raise ValueError("bad leaf index or leaf count")
    return path[:depth]


def root_from_path(leaf_digest, index: int, path, rc=None, mds=None) -> np.ndarray:
    rc, mds = _rc_mds(rc, mds)
    path = _u64(path).reshape(-1, 4)
    root = np.zeros(4, dtype=np.uint64)
    pp = path if path.size else np.zeros((1, 4), dtype=np.uint64)
    _load().orc_root_from_path(_ptr(rc), _ptr(mds), _ptr(_u64(leaf_digest)), index, _ptr(pp),
                               path.shape[0], _ptr(root))
    return root


def level_offsets(n_leaves: int):
    """Start row of every level in the level-major node array."""
    offs, base, cnt = [], 0, n_leaves
    while True:
        offs.append(base)
        if cnt == 1:
            break
        base += cnt
        cnt //= 2
    return offs


# ------------------------------------------------------ NTT / LDE (Sec. 2.3)
GENERATOR = 7      # generates the multiplicative group of Eq. 1's field
LDE_SHIFT = 7      # coset shift of the low-degree extension


def two_adic_root(log_n: int, inverse: bool = False) -> int:
    """Primitive 2^log_n-th root of unity 7^((p-1)/2^log_n) (or its inverse)."""
    return int(_load().orc_two_adic_root(log_n, 1 if inverse else 0))


def dft_naive(x, inverse: bool = False) -> np.ndarray:
    """The definition: y_i = sum_j x_j w^(ij) (inverse: w^-1, times n^-1)."""
    x = _u64(x)
    y = np.zeros_like(x)
    if _load().orc_dft_naive(_ptr(x), _ptr(y), x.size, 1 if inverse else 0) != 0:
        raise ValueError("length must be a power of two")
    return y


def fft(x, inverse: bool = False) -> np.ndarray:
    """Recursive radix-2 evaluation of the same transform."""
    y = _u64(x).copy()
    if _load().orc_fft(_ptr(y), y.size, 1 if inverse else 0) != 0:
        raise ValueError("length must be a power of two")
    return y


def ntt_columns(data, inverse: bool = False) -> np.ndarray:
    """Transform every column of a row-major (n, ncols) array."""
    d = _u64(data).copy()
    n, c = d.shape
    if _load().orc_ntt_columns(_ptr(d), n, c, 1 if inverse else 0) != 0:
        raise ValueError("row count must be a power of two")
    return d


def poly_eval(coeffs, x: int) -> int:
    """Horner: sum_j c_j x^j."""
    c = _u64(coeffs)
    return int(_load().orc_poly_eval(_ptr(c), c.size, x))


def interpolate_columns(evals) -> np.ndarray:
    """Coefficients (rows = powers) of every column's interpolant on the subgroup."""
    e = _u64(evals)
    out = np.zeros_like(e)
    if _load().orc_interpolate_columns(_ptr(e), e.shape[0], e.shape[1], _ptr(out)) != 0:
        raise ValueError("row count must be a power of two")
    return out


def lde_columns(evals, log_blowup: int, shift: int = LDE_SHIFT) -> np.ndarray:
    """(n 2^b, ncols): column c at row i is P_c(shift * w^i), w of order n 2^b."""
    e = _u64(evals)
    n, c = e.shape
    out = np.zeros((n << log_blowup, c), dtype=np.uint64)
    if _load().orc_lde_columns(_ptr(e), n, c, log_blowup, shift, _ptr(out)) != 0:
        raise ValueError("bad LDE arguments")
    return out
