"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the hashing method: it only draws
64-bit words.  Element k of stream ``seed`` is the SplitMix64 finaliser
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) applied to ``key(seed) + (k + 1) * 0x9E3779B97F4A7C15``; a word
that is not below ``bound`` is re-mixed until it is (an ``O(2^-32)`` event for
the Goldilocks bound), so every element depends only on (seed, k) and any
slice can be generated independently.

Seeds: workload ``cfg`` uses ``0x5EED0000 + cfg``; tree ``i`` of a batch uses
``tree_seed(seed, i)``.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
FIELD_BOUND = 0xFFFFFFFF00000001  # inputs are drawn uniform in [0, bound)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= M1
    z ^= z >> np.uint64(27)
    z *= M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int) -> np.uint64:
    return _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]


def words(seed: int, count: int, start: int = 0, bound: int | None = FIELD_BOUND,
          chunk: int = 1 << 22) -> np.ndarray:
    """``count`` words of stream ``seed`` starting at element ``start``."""
    out = np.empty(count, dtype=np.uint64)
    key = _key(seed)
    with np.errstate(over="ignore"):
        for lo in range(0, count, chunk):
            hi = min(count, lo + chunk)
            idx = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            z = _mix(key + idx * GOLDEN)
            if bound is not None:
                b = np.uint64(bound)
                bad = z >= b
                while bad.any():
                    z[bad] = _mix(z[bad])
                    bad = z >= b
            out[lo:hi] = z
    return out


def matrix(seed: int, rows: int, cols: int, bound: int | None = FIELD_BOUND) -> np.ndarray:
    """A (rows, cols) uint64 matrix, row-major, element (r, c) = word r*cols+c."""
    return words(seed, rows * cols, bound=bound).reshape(rows, cols)


def tree_seed(seed: int, tree: int) -> int:
    """Per-tree sub-seed of a batch."""
    return int(_mix(np.array([(seed * 0x100000001B3 + tree + 1) & 0xFFFFFFFFFFFFFFFF],
                             dtype=np.uint64))[0])


def config_seed(cfg: int) -> int:
    return 0x5EED0000 + cfg


def integers(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """``count`` integers uniform in [lo, hi] (inclusive), from stream ``seed``."""
    span = hi - lo + 1
    w = words(seed, count, bound=None)
    return (lo + (w % np.uint64(span)).astype(np.int64)).astype(np.int64)


def uniform01(seed: int, count: int) -> np.ndarray:
    """``count`` doubles uniform in [0, 1) from the top 53 bits of the words."""
    w = words(seed, count, bound=None)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# ------------------------------------------------------------- torch version
# The same streams computed with torch int64 arithmetic (wrapping multiply,
# logical shifts emulated by masking), so large inputs can be generated where
# they are used (for example directly in GPU memory).  Bit-identical to
# words() / matrix() above.

def _signed(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def _mix_t(z):
    import torch  # noqa: F401
    z = z ^ ((z >> 30) & ((1 << 34) - 1))
    z = z * _signed(int(M1))
    z = z ^ ((z >> 27) & ((1 << 37) - 1))
    z = z * _signed(int(M2))
    z = z ^ ((z >> 31) & ((1 << 33) - 1))
    return z


def words_torch(seed: int, count: int, start: int = 0, device="cpu", bound: int | None = FIELD_BOUND):
    """torch.int64 tensor holding the bits of words(seed, count, start, bound)."""
    import torch
    key = int(_key(seed))
    idx = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = _mix_t(idx * _signed(int(GOLDEN)) + _signed(key))
    if bound is not None:
        b = _signed(bound)

        def bad_of(t):
            # unsigned t >= bound, on the int64 view of the words
            if bound >= (1 << 63):
                return (t < 0) & (t >= b)
            return (t < 0) | (t >= b)
        bad = bad_of(z)
        while bool(bad.any()):
            z = torch.where(bad, _mix_t(z), z)
            bad = bad_of(z)
    return z


def matrix_torch(seed: int, rows: int, cols: int, device="cpu", bound: int | None = FIELD_BOUND):
    return words_torch(seed, rows * cols, device=device, bound=bound).view(rows, cols)


# ------------------------------------------------------------ workload recipes
# Shapes and seeds of the benchmark workloads (no arithmetic of the method):
# the bench, the tests and the script that stores the oracle's full-size
# results all draw their inputs from here, so the stored values describe
# exactly the inputs the GPU path is run on.

def tree_rows_seed(log_n: int, width: int) -> int:
    """Seed of the single-tree workloads (2^22 leaves x width 8 or 64)."""
    return config_seed(3) if width == 8 else config_seed(3) + width


def batch_sizes(trees: int = 64, max_log_n: int = 20, seed: int | None = None):
    """(log2 leaves, width) of each tree of the batched workload: k log-uniform
    in [12, min(20, max_log_n)], width uniform in {8, 16, 32, 64, 128}."""
    seed = config_seed(4) if seed is None else seed
    u = uniform01(seed, trees)
    top = min(max_log_n, 20)
    ks = [12 + int(v * (top - 12 + 1)) for v in u]
    widths = [(8, 16, 32, 64, 128)[int(v)] for v in integers(seed + 1, trees, 0, 4)]
    return [(min(k, top), w) for k, w in zip(ks, widths)]


def batch_tree_seed(tree: int) -> int:
    return tree_seed(config_seed(4), tree)


SERVE_WIDTHS = (8, 32, 128, 256)


def served_stream(requests: int = 2000, rate: float = 200.0, min_log_n: int = 10, max_log_n: int = 22,
                  seed: int | None = None):
    """Arrival times (s, Poisson at `rate`), log2 leaf counts (uniform in
    [min_log_n, max_log_n]) and widths (uniform in SERVE_WIDTHS) of a served stream."""
    seed = config_seed(5) if seed is None else seed
    gaps = -np.log(1.0 - uniform01(seed, requests)) / rate
    arrivals = np.cumsum(gaps)
    ks = [int(k) for k in integers(seed + 1, requests, min_log_n, max_log_n)]
    ws = [SERVE_WIDTHS[int(v)] for v in integers(seed + 2, requests, 0, len(SERVE_WIDTHS) - 1)]
    return arrivals, ks, ws


def served_rows_seed(log_n: int, width: int) -> int:
    """Rows of every served request of shape (2^log_n leaves, width) come from this seed."""
    return tree_seed(config_seed(5), (log_n << 16) | width)
