"""CSR with uint32 offsets (gconn_cc_csr32, gconn_spanning_forest_csr32 and
their plans) against the oracle, bit-exact on canonical labels, on the
vectorised gathering path (16-byte aligned buffers) and the scalar one
(unaligned labels), other finish block sizes, and a graph whose finish moves
the L_max root (finalisation must then walk every vertex)."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2008_11839_gb300 as g
from gpu_util import UF_COMBOS, UF_FOREST, combo_id, dev, host_u32, small_graphs

pytestmark = pytest.mark.gpu

GRAPHS = small_graphs()
REF = {name: oracle.cc_uf(n, e) for name, n, e in GRAPHS}
CSR = {name: graphgen.csr(n, e) for name, n, e in GRAPHS}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g.build()
    g.lib()


def _u32(off):
    assert int(off[-1]) < 2 ** 32
    return off.astype(np.uint32)


@pytest.mark.parametrize("sample", ["none", "kout", "hb", "bfs"])
@pytest.mark.parametrize("combo", UF_COMBOS, ids=combo_id)
def test_csr32_sampling_union_find(sample, combo):
    link, f, sp = combo
    v = g.make_variant(sample=sample, link=link, find=f, splice=sp)
    for name, n, e in GRAPHS:
        off, cols = CSR[name]
        lab = g.cc_csr(n, dev(_u32(off)), dev(cols), v)       # int32 offsets select gconn_cc_csr32
        g.gconn_sync()
        assert (host_u32(lab) == REF[name]).all(), name


@pytest.mark.parametrize("sample", ["none", "kout", "hb", "bfs"])
@pytest.mark.parametrize("combo", UF_FOREST[::3], ids=combo_id)
def test_csr32_spanning_forest(sample, combo):
    link, f, sp = combo
    v = g.make_variant(sample=sample, link=link, find=f, splice=sp)
    for name, n, e in GRAPHS:
        off, cols = CSR[name]
        ids, lab = g.spanning_forest_csr(n, dev(_u32(off)), dev(cols), v, labels=True)
        g.gconn_sync()
        assert oracle.sf_check_arcs(n, off, cols, ids.cpu().numpy().astype(np.uint64), REF[name]) == 0, name
        assert (host_u32(lab) == REF[name]).all(), name


@pytest.mark.parametrize("link", ["sv", "lt", "lp"])
def test_csr32_round_finishes(link):
    v = g.make_variant(sample="kout", link=link, lt="PRF")
    for name, n, e in GRAPHS:
        off, cols = CSR[name]
        lab = g.cc_csr(n, dev(_u32(off)), dev(cols), v)
        g.gconn_sync()
        assert (host_u32(lab) == REF[name]).all(), (name, link)


def test_csr32_host_buffers_and_plans():
    import torch
    n = 30011
    e = graphgen.rmat(15, 150_000, 31)[:, :] % n
    e = e.astype(np.uint32)
    ref = oracle.cc_uf(n, e)
    off, cols = graphgen.csr(n, e)
    off32 = _u32(off)
    out = np.empty(n, np.uint32)
    g.gconn_cc_csr32(n, off32, cols, out, g.make_variant(sample="kout", link="remcas", splice="split_one"))
    assert (out == ref).all()
    d_off, d_cols = dev(off32), dev(cols)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    for spec in [dict(sample="kout", link="remcas", splice="split_one"), dict(sample="hb", link="early"),
                 dict(sample="none", link="async", find="halve")]:
        p = g.gconn_plan_create_cc_csr32(n, d_off, d_cols, lab, g.make_variant(**spec))
        for _ in range(3):
            lab.fill_(-1)
            g.gconn_plan_run(p)
            g.gconn_sync()
            assert (host_u32(lab) == ref).all(), spec
        g.gconn_plan_destroy(p)
    forest = torch.empty(n, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    p = g.gconn_plan_create_forest_csr32(n, d_off, d_cols, forest, cnt, lab,
                                         g.make_variant(sample="kout", link="remcas", splice="split_one"))
    for _ in range(3):
        g.gconn_plan_run(p)
        g.gconn_sync()
        c = int(cnt.item())
        assert oracle.sf_check_arcs(n, off, cols, forest[:c].cpu().numpy().astype(np.uint64), ref) == 0
        assert (host_u32(lab) == ref).all()
    g.gconn_plan_destroy(p)


def _moved_lmax_graph():
    """A graph whose sampled giant component (min id 3) is joined in the
    finish to a cluster {0, 1, 100} through the unsampled edge 100-200: the
    finish links the L_max root under 0, so finalisation must walk every
    vertex, not only the gathered ones.  Vertex 2 is isolated."""
    n = 5000
    rng = np.random.default_rng(7)
    giant = np.array([x for x in range(3, n) if x != 100], np.uint32)
    a = rng.choice(giant, 40_000)
    b = rng.choice(giant, 40_000)
    path = np.stack([giant[:-1], giant[1:]], 1)                 # keeps the giant connected
    extra = np.array([[0, 1], [0, 100], [1, 100], [100, 200], [200, 3], [200, 4]], np.uint32)
    e = np.concatenate([np.stack([a, b], 1), path, extra]).astype(np.uint32)
    # 200's two smallest neighbours must be 3 and 4 (so sampling never takes 200-100)
    return n, e


@pytest.mark.parametrize("sample", ["kout", "hb", "bfs"])
@pytest.mark.parametrize("aligned", [True, False])
def test_lmax_root_moved_in_finish(sample, aligned):
    """k-out / HB: the finish moves the L_max root (full finalisation);
    BFS labels the whole component, so its finish has nothing to link."""
    import torch
    n, e = _moved_lmax_graph()
    ref = oracle.cc_uf(n, e)
    assert ref[3] == 0 and ref[2] == 2
    off, cols = graphgen.csr(n, e)
    row200 = cols[off[200]:off[201]]
    assert sorted(row200)[:2] == [3, 4]
    v = g.make_variant(sample=sample, link="remcas", splice="split_one")
    buf = torch.empty(n + 4, dtype=torch.int32, device="cuda")
    lab = buf[:n] if aligned else buf[1:n + 1]                 # 4-byte offset: the scalar gathering kernel
    for offs in (dev(off), dev(_u32(off))):
        fn = g.gconn_cc_csr32 if offs.dtype == torch.int32 else g.gconn_cc_csr
        fn(n, offs, dev(cols), lab, v)
        g.gconn_sync()
        assert (host_u32(lab) == ref).all()
        st = g.gconn_cc_csr_stats(n, dev(off), dev(cols), buf[:n], v)
        if sample == "bfs":    # BFS reaches the source's whole component: nothing is left to link
            assert st.lmax == 0 and st.active_vertices == 0
        else:                  # the giant is sampled whole under vertex 3
            assert st.lmax == 3 and st.active_vertices == 3


@pytest.mark.parametrize("block", [128, 192])
def test_other_finish_block_sizes(block):
    """Finish kernels with another block size give the same labels."""
    v = g.make_variant(sample="kout", link="remcas", splice="split_one", block=block)
    for name, n, e in GRAPHS:
        off, cols = CSR[name]
        for o in (off, _u32(off)):
            lab = g.cc_csr(n, dev(o), dev(cols), v)
            g.gconn_sync()
            assert (host_u32(lab) == REF[name]).all(), (name, block)
