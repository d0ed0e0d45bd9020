"""The seeded input generator: numpy and torch versions agree bit for bit,
values respect the bound, and slices are independent of how they are cut."""
import numpy as np
import torch

import pg_synth

P = 0xFFFFFFFF00000001


def test_numpy_torch_identical():
    for seed in (0, 1, 0x5EED0003, 2**63 + 5):
        a = pg_synth.words(seed, 5000, start=17)
        b = pg_synth.words_torch(seed, 5000, start=17).numpy().view(np.uint64)
        assert (a == b).all()
        a = pg_synth.words(seed, 3000, bound=None)
        b = pg_synth.words_torch(seed, 3000, bound=None).numpy().view(np.uint64)
        assert (a == b).all()


def test_bound_and_rejection_path():
    a = pg_synth.words(7, 100000)
    assert (a < np.uint64(P)).all()
    # a tiny bound forces the re-mix loop on almost every element
    small = pg_synth.words(9, 2000, bound=1 << 62)
    t = pg_synth.words_torch(9, 2000, bound=1 << 62).numpy().view(np.uint64)
    assert (small < np.uint64(1 << 62)).all() and (small == t).all()


def test_slices_are_counter_based():
    whole = pg_synth.words(11, 1000)
    parts = np.concatenate([pg_synth.words(11, 300, start=0), pg_synth.words(11, 700, start=300)])
    assert (whole == parts).all()
    m = pg_synth.matrix(12, 10, 7)
    assert (m.ravel() == pg_synth.words(12, 70)).all()


def test_uniformity_rough():
    a = pg_synth.words(13, 1 << 16) >> np.uint64(60)
    counts = np.bincount(a.astype(np.int64), minlength=16)
    assert counts.min() > 0.8 * (1 << 12) and counts.max() < 1.2 * (1 << 12)
