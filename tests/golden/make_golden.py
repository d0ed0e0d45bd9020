"""Writes the stored expected values under tests/golden/ (calls only oracle/).

  pg12_v1.sha256      SHA-256 of the plain parameter set (rc[30][12] then
                      mds[12][12], little-endian uint64) and its first words
  cfg1_root.txt       root of the 2^10-leaf, width-8 tree of workload 1
                      (seed 0x5EED0001), four canonical words in hex
  full_size.json      the oracle's complete outputs at the benchmark sizes,
                      as SHA-256 digests of their little-endian bytes (plus
                      the root of every tree): the 2^24 permuted states of
                      workload 2, the 2^22 x 8 and 2^22 x 64 trees of
                      workload 3, every tree of the 64-tree batch of
                      workload 4 and the 2^22-leaf served shapes of
                      workload 5 at widths 8 and 32, and the low-degree
                      extension of the 2^21 x 8 trace (blowup 2) with the
                      root of its 2^22 x 8 commitment.  Inputs come from
                      pg_synth's workload recipes.

Run from the repository root:
  python tests/golden/make_golden.py            # the two small files
  python tests/golden/make_golden.py --full     # also full_size.json
                                                # (about 2e8 oracle
                                                # permutations; entries
                                                # already stored are kept)
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import pg_synth  # noqa: E402

FULL = os.path.join(HERE, "full_size.json")


def params_digest():
    rc, mds = oracle.params()[:2]
    h = hashlib.sha256()
    h.update(rc.astype("<u8").tobytes())
    h.update(mds.astype("<u8").tobytes())
    return h.hexdigest(), rc, mds


def sha256_words(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).astype("<u8").tobytes()).hexdigest()


def tree_entry(seed: int, log_n: int, width: int, threads: int) -> dict:
    rows = pg_synth.matrix(seed, 1 << log_n, width)
    nodes = oracle.merkle_build(rows, nthreads=threads)
    return {"seed": hex(seed), "log_n": log_n, "width": width,
            "root": [f"{int(v):016x}" for v in nodes[-1]], "nodes_sha256": sha256_words(nodes)}


def full_entries():
    """(key, thunk) of every stored full-size result."""
    threads = os.cpu_count() or 1
    out = []

    def permute():
        seed = pg_synth.config_seed(2)
        st = pg_synth.matrix(seed, 1 << 24, 12)
        res = oracle.permute(st, nthreads=threads)
        return {"seed": hex(seed), "states": 1 << 24, "states_sha256": sha256_words(res),
                "first": [f"{int(v):016x}" for v in res[0]], "last": [f"{int(v):016x}" for v in res[-1]]}
    out.append(("permute_2e24", permute))
    for w in (8, 64):
        out.append((f"merkle_2e22_w{w}",
                    lambda w=w: tree_entry(pg_synth.tree_rows_seed(22, w), 22, w, threads)))
    for k, (lg, w) in enumerate(pg_synth.batch_sizes()):
        out.append((f"batch_{k:02d}", lambda k=k, lg=lg, w=w: tree_entry(pg_synth.batch_tree_seed(k), lg, w, threads)))
    for w in (8, 32):
        out.append((f"serve_2e22_w{w}",
                    lambda w=w: tree_entry(pg_synth.served_rows_seed(22, w), 22, w, threads)))

    def lde():
        seed, log_n, cols, log_b = pg_synth.config_seed(6), 21, 8, 1
        ext = oracle.lde_columns(pg_synth.matrix(seed, 1 << log_n, cols), log_b)
        nodes = oracle.merkle_build(ext, nthreads=threads)
        return {"seed": hex(seed), "log_n": log_n, "cols": cols, "log_blowup": log_b,
                "out_sha256": sha256_words(ext), "root": [f"{int(v):016x}" for v in nodes[-1]],
                "nodes_sha256": sha256_words(nodes)}
    out.append(("lde_2e21x8_b1", lde))
    return out


def write_full():
    data = {}
    if os.path.exists(FULL):
        with open(FULL) as f:
            data = json.load(f)
    for key, fn in full_entries():
        if key in data:
            continue
        t0 = time.time()
        data[key] = fn()
        print(f"{key}: {time.time() - t0:.1f} s", flush=True)
        tmp = FULL + ".tmp"
        with open(tmp, "w") as f:
            json.dump(dict(sorted(data.items())), f, indent=1)
            f.write("\n")
        os.replace(tmp, FULL)


def main():
    digest, rc, mds = params_digest()
    with open(os.path.join(HERE, "pg12_v1.sha256"), "w") as f:
        f.write(f"sha256 {digest}\n")
        f.write(f"rc[0][0] {int(rc[0, 0]):016x}\n")
        f.write(f"rc[29][11] {int(rc[29, 11]):016x}\n")
        f.write(f"mds[0][0] {int(mds[0, 0]):016x}\n")
    rows = pg_synth.matrix(pg_synth.config_seed(1), 1 << 10, 8)
    root = oracle.merkle_build(rows, nthreads=4)[-1]
    with open(os.path.join(HERE, "cfg1_root.txt"), "w") as f:
        f.write(" ".join(f"{int(v):016x}" for v in root) + "\n")
    if "--full" in sys.argv[1:]:
        write_full()


if __name__ == "__main__":
    main()
