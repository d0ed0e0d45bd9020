"""Reader of tests/golden/full_size.json (test helper).

The file holds the CPU oracle's complete outputs at the benchmark sizes as
SHA-256 digests of their little-endian words plus every tree's root; it is
written by tests/golden/make_golden.py, which calls only oracle/ and draws
its inputs from pg_synth's workload recipes.
"""
import hashlib
import json
import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size.json")


def load() -> dict:
    with open(PATH) as f:
        return json.load(f)


def sha256_words(a) -> str:
    """SHA-256 of an array of 64-bit words (numpy, or a torch tensor anywhere)."""
    if not isinstance(a, np.ndarray):
        a = a.detach().cpu().numpy()
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint64).astype("<u8").tobytes()).hexdigest()


def root_words(entry) -> list:
    return [int(v, 16) for v in entry["root"]]
