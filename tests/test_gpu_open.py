"""Authentication paths on the GPU (pg_merkle_open / pg_merkle_verify)
against the oracle's paths and root recomputation."""
import numpy as np
import pytest

import oracle
import pg_synth

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)
    yield


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


@pytest.mark.parametrize("log_n", [1, 5, 12])
def test_open_matches_oracle_and_verifies(log_n):
    n = 1 << log_n
    rows = pg_synth.matrix(0x1100 + log_n, n, 8)
    nodes_h = oracle.merkle_build(rows, nthreads=8)
    nodes = _dev(nodes_h)
    idx_h = np.unique(np.concatenate([pg_synth.integers(0x1200 + log_n, 50, 0, n - 1), [0, n - 1]]))
    idx = torch.from_numpy(idx_h.astype(np.int64)).cuda()
    paths = pg.merkle_open(nodes, n, idx)
    torch.cuda.synchronize()
    got = paths.cpu().numpy().view(np.uint64)
    for q, i in enumerate(idx_h):
        assert (got[q] == oracle.auth_path(nodes_h, n, int(i))).all()
    leaves = nodes[idx]
    root = nodes[-1].contiguous()
    ok = pg.merkle_verify(root, n, leaves.contiguous(), idx, paths)
    assert bool(ok.all())
    bad = paths.clone()
    bad[0, log_n - 1, 2] ^= 1
    ok2 = pg.merkle_verify(root, n, leaves.contiguous(), idx, bad)
    assert not bool(ok2[0]) and bool(ok2[1:].all())
    # a path checked against the wrong leaf index fails
    ok3 = pg.merkle_verify(root, n, leaves.contiguous(), (idx ^ 1), paths)
    assert not bool(ok3.all())
