"""GPU parity of incremental connectivity (Section 3.5, Algorithm 3): a
replay of the same insert/query stream by the sequential oracle gives the
same answers bit for bit, and the final labels equal static components of
everything inserted."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2008_11839_gb300 as g
from conftest import read_inc_golden
from gpu_util import LT_ROOT, UF_COMBOS, combo_id, dev, host_u32

pytestmark = pytest.mark.gpu

INC_VARIANTS = [dict(link=l, find=f, splice=s) for (l, f, s) in UF_COMBOS] + \
    [dict(link="sv")] + [dict(link="lt", lt=r) for r in LT_ROOT]


def _vid(kw):
    return "-".join(str(x) for x in kw.values())


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g.build()


def _stream(n, seed, nbatches=8):
    rng = np.random.default_rng(seed)
    scale = int(np.ceil(np.log2(n)))
    perm = graphgen.permutation(1 << scale, seed, 6)
    start, qstart = 0, 0
    ops = []
    for _ in range(nbatches):
        b = int(rng.integers(0, 3000))
        e = graphgen.rmat_range(scale, start, b, seed, perm=perm)
        e = e % np.uint32(n)
        start += b
        q = int(rng.integers(1, 4000))
        p = graphgen.pairs_range(n, qstart, q, seed)
        qstart += q
        ops.append((e, p))
    return ops


@pytest.mark.parametrize("kw", INC_VARIANTS, ids=_vid)
def test_replay_matches_oracle(kw):
    n = 6000
    inc = g.Incremental(n, g.make_variant(**kw))
    ref = oracle.Incremental(n)
    allins = []
    for e, p in _stream(n, 11):
        inc.insert(dev(e))
        ref.insert(e)
        allins.append(e)
        got = inc.query(dev(p)).cpu().numpy()
        g.gconn_sync()
        assert (got == ref.query(p)).all()
    lab = host_u32(inc.labels())
    g.gconn_sync()
    assert (lab == oracle.cc_uf(n, np.concatenate(allins))).all()
    inc.close()


def test_golden_stream():
    n, ops, labels = read_inc_golden("inc_stream.txt")
    for kw in (dict(link="async"), dict(link="remcas", splice="splice"), dict(link="jtb")):
        inc = g.Incremental(n, g.make_variant(**kw))
        for op in ops:
            if op[0] == "insert":
                inc.insert(dev(np.array([[op[1], op[2]]], np.uint32)))
            else:
                got = int(inc.query(dev(np.array([[op[1], op[2]]], np.uint32))).cpu()[0])
                assert got == op[3], (kw, op)
        assert host_u32(inc.labels()).tolist() == labels
        inc.close()


def test_host_buffers_and_empty_batches():
    n = 1000
    h = g.gconn_inc_create(n, g.make_variant(link="async"))
    e = graphgen.er(n, 700, 3)
    g.gconn_inc_insert_batch(h, 0, None)
    g.gconn_inc_insert_batch(h, len(e), e)
    p = graphgen.pairs_range(n, 0, 500, 3)
    out = np.empty(500, np.uint8)
    g.gconn_inc_query(h, 500, p, out)
    ref = oracle.cc_uf(n, e)
    assert (out == (ref[p[:, 0]] == ref[p[:, 1]])).all()
    lab = np.empty(n, np.uint32)
    g.gconn_inc_labels(h, lab)
    assert (lab == ref).all()
    with pytest.raises(g.GconnError) as ex:
        g.gconn_inc_query(h, 1, np.array([[0, n]], np.uint32), np.empty(1, np.uint8))
    assert ex.value.status == g.GCONN_E_RANGE
    g.gconn_inc_destroy(h)


@pytest.mark.parametrize("kw", [dict(link="sv"), dict(link="lt", lt="PRS"), dict(link="early"),
                                dict(link="remcas", splice="split_one")], ids=_vid)
def test_edges_inspected_per_batch(kw):
    """Section 4.4's edges-inspected count: a union-find finish reads each
    inserted edge once; SV and Liu-Tarjan re-read the whole batch every round,
    and a path inserted from its far end needs several rounds."""
    n = 4096
    path = np.stack([np.arange(n - 1, 0, -1), np.arange(n - 2, -1, -1)], 1).astype(np.uint32)
    h = g.Incremental(n, g.make_variant(**kw))
    try:
        assert h.edges_inspected() == (0, 0)
        h.insert(dev(path))
        g.gconn_sync()
        last, total = h.edges_inspected()
        b = len(path)
        if kw["link"] in ("sv", "lt"):
            assert last % b == 0 and last >= 2 * b, last
        else:
            assert last == b
        assert total == last
        h.insert(dev(path[:10]))
        g.gconn_sync()
        last2, total2 = h.edges_inspected()
        assert total2 == total + last2 and last2 % 10 == 0 and last2 >= 10
        lab = host_u32(h.labels())
        assert (lab == 0).all()
    finally:
        h.close()


def test_incremental_rejects_non_root_based():
    with pytest.raises(g.GconnError) as ex:
        g.gconn_inc_create(10, g.make_variant(link="lt", lt="PUS"))
    assert ex.value.status == g.GCONN_E_UNSUPPORTED
    with pytest.raises(g.GconnError):
        g.gconn_inc_create(10, g.make_variant(sample="kout"))


MIXED_VARIANTS = [dict(link=l, find=f, splice=s) for (l, f, s) in UF_COMBOS]


@pytest.mark.parametrize("kw", MIXED_VARIANTS, ids=_vid)
def test_mixed_batches_linearizable(kw):
    """Algorithm 3's mixed batches: every answer lies between the state before
    and after its batch, and the final labels equal static components."""
    n = 5000
    inc = g.gconn_inc_create(n, g.make_variant(**kw))
    ref = oracle.Incremental(n)
    rng = np.random.default_rng(5)
    allins = []
    for bi in range(6):
        b = int(rng.integers(1, 5000))
        pairs = graphgen.er(n, b, 300 + bi)
        isq = (rng.random(b) < 0.5).astype(np.uint8)
        before = ref.query(pairs)
        ins = pairs[isq == 0]
        ref.insert(ins)
        allins.append(ins)
        after = ref.query(pairs)
        bits = np.zeros((b + 31) // 32, np.uint32)
        g.gconn_inc_process_batch(inc, b, pairs, isq, bits)
        got = ((bits[np.arange(b) // 32] >> (np.arange(b) % 32).astype(np.uint32)) & 1).astype(bool)
        q = isq == 1
        assert not got[~q].any()                        # inserts have no bit
        assert (got[q] >= before[q].astype(bool)).all()  # connected before => 1
        assert (got[q] <= after[q].astype(bool)).all()   # not connected after => 0
    lab = np.empty(n, np.uint32)
    g.gconn_inc_labels(inc, lab)
    assert (lab == oracle.cc_uf(n, np.concatenate(allins))).all()
    g.gconn_inc_destroy(inc)
