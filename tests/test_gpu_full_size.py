"""Full-size parity: every output of every benchmark workload, word for word.

The CPU oracle's complete outputs at the benchmark sizes are stored as
SHA-256 digests (plus roots) in tests/golden/full_size.json, written by
tests/golden/make_golden.py from oracle/ alone.  Here the GPU path, through
the C ABI, builds the same outputs from the same seeded inputs and every
word must match:

  workload 2  2^24 independent states permuted in place (both engines)
  workload 3  the 2^22-leaf trees of width 8 (both engines, and through the
              host-rows call) and width 64
  workload 4  all 64 trees of the mixed batch, in one captured launch with
              the autotuned schedule
  workload 5  2^22-leaf served requests of widths 8 and 32, admitted into
              the serving runtime together with smaller requests
  LDE         the 2^21 x 8 trace extended with blowup 2 (every output word)
              and its 2^22 x 8 commitment

The path is exact integer arithmetic, so the tolerance is zero.
"""
import pytest

import golden_values
import pg_synth

torch = pytest.importorskip("torch")
pg = pytest.importorskip("paper_2506_09505_gb300")

pytestmark = pytest.mark.gpu

GOLD = golden_values.load()


@pytest.fixture(scope="module", autouse=True)
def ready():
    pg.load(build_if_missing=True)
    pg.init(0)
    yield
    pg.set_engine(pg.ENGINE_TENSOR)


def _tree_rows(entry):
    return pg_synth.matrix_torch(int(entry["seed"], 16), 1 << entry["log_n"], entry["width"], device="cuda")


def _check_tree(nodes, root, entry):
    assert root == golden_values.root_words(entry)
    assert golden_values.sha256_words(nodes) == entry["nodes_sha256"]


@pytest.mark.parametrize("engine", [pg.ENGINE_TENSOR, pg.ENGINE_INT])
def test_permute_2e24_states(engine):
    e = GOLD["permute_2e24"]
    st = pg_synth.matrix_torch(int(e["seed"], 16), e["states"], 12, device="cuda")
    pg.set_engine(engine)
    pg.permute_batch(st)
    torch.cuda.synchronize()
    pg.set_engine(pg.ENGINE_TENSOR)
    assert pg.device_faults() == 0
    assert golden_values.sha256_words(st) == e["states_sha256"]
    del st
    torch.cuda.empty_cache()


@pytest.mark.parametrize("engine", [pg.ENGINE_TENSOR, pg.ENGINE_INT])
def test_merkle_2e22_width8(engine):
    e = GOLD["merkle_2e22_w8"]
    rows = _tree_rows(e)
    pg.set_engine(engine)
    nodes, root = pg.merkle_build(rows, want_root=True)
    pg.set_engine(pg.ENGINE_TENSOR)
    _check_tree(nodes, root, e)


def test_merkle_2e22_width64():
    e = GOLD["merkle_2e22_w64"]
    rows = _tree_rows(e)
    nodes, root = pg.merkle_build(rows, want_root=True)
    _check_tree(nodes, root, e)
    assert pg.device_faults() == 0


def test_merkle_2e22_width8_from_host_rows():
    e = GOLD["merkle_2e22_w8"]
    host = _tree_rows(e).cpu().pin_memory()
    nodes, root = pg.merkle_build_host(host, want_root=True)
    _check_tree(nodes, root, e)


def test_batch_of_64_trees_in_one_captured_launch():
    sizes = pg_synth.batch_sizes()
    entries = [GOLD[f"batch_{k:02d}"] for k in range(len(sizes))]
    for (lg, w), e in zip(sizes, entries):
        assert (e["log_n"], e["width"]) == (lg, w)
    rows = [_tree_rows(e) for e in entries]
    nodes = pg.alloc_nodes(rows)
    best, _ = pg.batch_autotune(rows, nodes)
    for t in nodes:
        t.fill_(-1)
    g = pg.BatchGraph(rows, nodes, schedule=best)
    try:
        g.launch()
        torch.cuda.synchronize()
        for k, (nd, e) in enumerate(zip(nodes, entries)):
            assert [int(v) for v in nd[-1].cpu().numpy().view("uint64")] == golden_values.root_words(e), k
            assert golden_values.sha256_words(nd) == e["nodes_sha256"], k
    finally:
        g.close()


def test_served_2e22_requests_in_a_mix():
    big = [GOLD["serve_2e22_w8"], GOLD["serve_2e22_w32"]]
    small = [(10, 8), (14, 256), (12, 32), (16, 128), (11, 8), (13, 32)]
    reqs = [_tree_rows(e) for e in big]
    reqs += [pg_synth.matrix_torch(pg_synth.served_rows_seed(k, w), 1 << k, w, device="cuda") for k, w in small]
    torch.cuda.synchronize()
    srv = pg.Server(pool_bytes=2 << 30, max_batch=16, max_inflight=2)
    try:
        order = [2, 0, 3, 4, 1, 5, 6, 7]   # the big requests arrive among the small ones
        ids = {i: srv.submit(reqs[i]) for i in order}
        srv.drain(300.0)
        for i, rid in ids.items():
            assert srv.query(rid)["state"] == pg.REQ_DONE
            got = srv.nodes(rid, reqs[i].shape[0])
            if i < 2:
                root = [int(v) for v in got[-1].cpu().numpy().view("uint64")]
                _check_tree(got, root, big[i])
            else:
                assert torch.equal(got, pg.merkle_build(reqs[i])), i
            srv.release(rid)
    finally:
        srv.close()


def test_lde_2e21x8_and_its_commitment():
    e = GOLD["lde_2e21x8_b1"]
    evals = pg_synth.matrix_torch(int(e["seed"], 16), 1 << e["log_n"], e["cols"], device="cuda")
    before = golden_values.sha256_words(evals)
    out = pg.lde(evals, e["log_blowup"])
    assert golden_values.sha256_words(out) == e["out_sha256"]
    assert golden_values.sha256_words(evals) == before
    nodes, root = pg.merkle_build(out, want_root=True)
    _check_tree(nodes, root, e)
    # in place: the input buffer doubles as the scratch buffer
    work = evals.clone()
    assert torch.equal(pg.lde(work, e["log_blowup"], scratch=work), out)
