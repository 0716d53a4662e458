"""GPU parity of batched connected components (many independent graphs in
one persistent launch) against the oracle applied graph by graph."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2008_11839_gb300 as g
from gpu_util import dev, host_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g.build()


def _batch(G, seed, nmin=16, nmax=80_000):
    vo, eo, e = graphgen.batched(G, seed, nmin=nmin, nmax=nmax)
    return vo, eo, e, oracle.batched_cc(vo, eo, e)


def _run(vo, eo, e, tune=None):
    import torch
    lab = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    g.gconn_cc_batched(len(vo) - 1, vo, eo, dev(e), lab, tune)
    g.gconn_sync()
    return host_u32(lab)


def test_batched_matches_oracle_all_classes():
    vo, eo, e, _ = _batch(96, 3)              # sizes 16 .. 80,000: every class
    big_n = 70_001                            # plus one graph above the shared-memory classes
    big = graphgen.er(big_n, 120_000, 4)
    vo = np.append(vo, vo[-1] + big_n).astype(np.uint64)
    eo = np.append(eo, eo[-1] + len(big)).astype(np.uint64)
    e = np.concatenate([e, big])
    ref = oracle.batched_cc(vo, eo, e)
    assert np.diff(vo).max() > 65536
    assert (_run(vo, eo, e) == ref).all()


@pytest.mark.parametrize("rule", [("async", "naive"), ("async", "halve"), ("remcas", "naive")])
@pytest.mark.parametrize("block", [64, 256, 1024])
def test_every_rule_and_block(rule, block):
    vo, eo, e, ref = _batch(40, 5, nmax=65536)
    t = g.gconn_batch_tune_default()
    for c in range(g.GCONN_BATCH_CLASSES):
        t.block[c] = block
        t.link[c] = g.LINKS[rule[0]]
        t.find[c] = g.FINDS[rule[1]]
    assert (_run(vo, eo, e, t) == ref).all()


def test_plan_graph_replay_and_refill():
    import torch
    vo, eo, e, ref = _batch(64, 7, nmax=30_000)
    de = dev(e)
    lab = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    h = g.gconn_batch_create(len(vo) - 1, dev(vo), dev(eo), de, lab)
    for _ in range(2):
        lab.fill_(-1)
        g.gconn_batch_run(h)
        g.gconn_sync()
        assert (host_u32(lab) == ref).all()
    # same sizes, new edges in the same buffer: the captured graph sees them
    e2 = e.copy()
    rng = np.random.default_rng(1)
    for gi in range(len(vo) - 1):
        n = int(vo[gi + 1] - vo[gi])
        a, b = int(eo[gi]), int(eo[gi + 1])
        e2[a:b] = rng.integers(0, n, size=(b - a, 2))
    de.copy_(dev(e2))
    g.gconn_batch_run(h)
    g.gconn_sync()
    assert (host_u32(lab) == oracle.batched_cc(vo, eo, e2)).all()
    g.gconn_batch_destroy(h)


def test_autotune_then_exact():
    import torch
    vo, eo, e, ref = _batch(48, 9, nmax=65536)
    lab = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    t = g.gconn_batch_autotune(len(vo) - 1, vo, eo, dev(e), lab)
    d = t.as_dict()
    assert all(b in (128, 256, 512, 1024) for b in d["block"])
    assert (_run(vo, eo, e, t) == ref).all()


def test_empty_graphs_and_range_error():
    import torch
    vo = np.array([0, 0, 3, 3, 10], np.uint64)         # graphs with n = 0, 3, 0, 7
    eo = np.array([0, 0, 2, 2, 2], np.uint64)
    e = np.array([[0, 2], [1, 1]], np.uint32)
    lab = torch.empty(10, dtype=torch.int32, device="cuda")
    g.gconn_cc_batched(4, vo, eo, dev(e), lab)
    g.gconn_sync()
    assert host_u32(lab).tolist() == [0, 1, 0, 0, 1, 2, 3, 4, 5, 6]
    bad = np.array([[0, 3], [1, 1]], np.uint32)          # 3 is not a vertex of a 3-vertex graph
    g.gconn_cc_batched(4, vo, eo, dev(bad), lab)
    with pytest.raises(g.GconnError) as ex:
        g.gconn_sync()
    assert ex.value.status == g.GCONN_E_RANGE
    with pytest.raises(g.GconnError):                    # edges must be device memory
        g.gconn_cc_batched(4, vo, eo, e, lab)
