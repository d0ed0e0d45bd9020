"""Writes the stored expected values under tests/golden/ (calls only oracle/).

  pg12_v1.sha256      SHA-256 of the plain parameter set (rc[30][12] then
                      mds[12][12], little-endian uint64) and its first words
  cfg1_root.txt       root of the 2^10-leaf, width-8 tree of workload 1
                      (seed 0x5EED0001), four canonical words in hex

Run from the repository root:  python tests/golden/make_golden.py
"""
import hashlib
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import pg_synth  # noqa: E402


def params_digest():
    rc, mds = oracle.params()[:2]
    h = hashlib.sha256()
    h.update(rc.astype("<u8").tobytes())
    h.update(mds.astype("<u8").tobytes())
    return h.hexdigest(), rc, mds


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


if __name__ == "__main__":
    main()
