"""GPU parity with the small-entry parameter set pg12_small (circulant MDS
with 8-bit entries, Table 1's mult_72 / mmult_4x12_8 shape), on both engines:
the integer engine's dense layers take the specialised 8-bit path, the
tensor engine's digit tables are built from the small matrix like from any
other; every output must equal the oracle."""
import numpy as np
import pytest

import oracle
import pg_synth

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def small_set():
    pg.load(build_if_missing=True)
    pg.init(0, "pg12_small")
    yield
    torch.cuda.synchronize()
    pg.params_select(None)
    pg.set_engine(pg.ENGINE_TENSOR)


@pytest.fixture(params=["tensor", "int"], autouse=True)
def engine(request):
    pg.set_engine(pg.ENGINE_TENSOR if request.param == "tensor" else pg.ENGINE_INT)
    yield request.param
    torch.cuda.synchronize()
    pg.set_engine(pg.ENGINE_TENSOR)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint64)


def _orc():
    rc, mds, _, _ = oracle.params_small()
    return rc, mds


def test_permute_small_set():
    rc, mds = _orc()
    st = pg_synth.matrix(0x1300, 3000, 12)
    st[0] = np.uint64((1 << 64) - 1)
    t = _dev(st)
    pg.permute_batch(t)
    assert (_host(t) == oracle.permute(st, rc, mds)).all()


@pytest.mark.parametrize("log_n,w", [(0, 8), (5, 8), (10, 24), (14, 8), (16, 8)])
def test_merkle_small_set(log_n, w):
    rc, mds = _orc()
    n = 1 << log_n
    rows = pg_synth.matrix(0x1400 + log_n, n, w)
    nodes = pg.merkle_build(_dev(rows))
    assert (_host(nodes) == oracle.merkle_build(rows, nthreads=8, rc=rc, mds=mds)).all()


def test_batch_small_set():
    rc, mds = _orc()
    host_rows = [pg_synth.matrix(0x1500 + k, 1 << lg, w) for k, (lg, w) in enumerate([(6, 8), (9, 16), (12, 8)])]
    rows = [_dev(r) for r in host_rows]
    nodes = pg.merkle_build_batch(rows)
    for hr, nd in zip(host_rows, nodes):
        assert (_host(nd) == oracle.merkle_build(hr, nthreads=8, rc=rc, mds=mds)).all()
