"""Sampled check of a Merkle node array against the oracle (test helper).

Leaves: the oracle hashes sampled rows (Sec. 2.4 sponge).  Every level: for
sampled nodes (always the first and last) the oracle compresses the GPU's own
two children and must get the GPU's parent.  Together with a full-size root
this pins every level without rebuilding the whole tree on the CPU.
"""
import numpy as np

import oracle
import pg_synth

P = oracle.P


def level_offsets(n):
    offs, base, cnt = [], 0, n
    while True:
        offs.append(base)
        if cnt == 1:
            return offs
        base += cnt
        cnt //= 2


def check_tree_sampled(rows, out, seed, n_leaves=256, per_level=64):
    """rows: numpy (n, w) or a CUDA tensor of int64 words; out: numpy (2n-1, 4) uint64."""
    n = rows.shape[0]
    offs = level_offsets(n)
    assert (out < np.uint64(P)).all()
    leaves = np.unique(np.concatenate([pg_synth.integers(seed, n_leaves, 0, n - 1), [0, n - 1]]))
    if isinstance(rows, np.ndarray):
        sample = rows[leaves]
    else:
        import torch
        idx = torch.from_numpy(leaves).to(rows.device)
        sample = rows.index_select(0, idx).cpu().numpy().view(np.uint64)
    assert (out[leaves] == oracle.hash_rows(sample)).all()
    cnt = n // 2
    for lvl in range(1, len(offs)):
        ks = np.unique(np.concatenate([pg_synth.integers(seed + lvl, per_level, 0, cnt - 1), [0, cnt - 1]]))
        for k in ks:
            left = out[offs[lvl - 1] + 2 * k]
            right = out[offs[lvl - 1] + 2 * k + 1]
            assert (out[offs[lvl] + k] == oracle.hash_pair(left, right)).all(), (lvl, k)
        cnt //= 2
