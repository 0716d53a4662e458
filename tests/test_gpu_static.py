"""GPU parity of static connectivity and spanning forests (Algorithms 1, 2)
against the CPU oracle, bit-exact on canonical labels, through the C ABI."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2008_11839_gb300 as g
from gpu_util import LT_ALL, LT_ROOT, UF_COMBOS, UF_FOREST, combo_id, dev, host_u32, small_graphs

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


def _cc_coo(n, e, v):
    lab = g.cc(n, dev(e), v)
    g.gconn_sync()
    return host_u32(lab)


def _cc_csr(n, off, cols, v):
    lab = g.cc_csr(n, dev(off), dev(cols), v)
    g.gconn_sync()
    return host_u32(lab)


@pytest.mark.parametrize("combo", UF_COMBOS, ids=combo_id)
def test_coo_union_find(combo):
    link, f, sp = combo
    v = g.make_variant(link=link, find=f, splice=sp)
    for name, n, e in GRAPHS:
        assert (_cc_coo(n, e, v) == REF[name]).all(), name


@pytest.mark.parametrize("combo", UF_FOREST, ids=combo_id)
def test_coo_spanning_forest(combo):
    link, f, sp = combo
    v = g.make_variant(link=link, find=f, splice=sp)
    for name, n, e in GRAPHS:
        ids, lab = g.spanning_forest(n, dev(e), v, labels=True)
        g.gconn_sync()
        ids = ids.cpu().numpy().astype(np.uint64)
        assert oracle.sf_check(n, e, ids, REF[name]) == 0, name
        assert (host_u32(lab) == REF[name]).all(), name


@pytest.mark.parametrize("sample", ["none", "kout", "hb", "bfs"])
@pytest.mark.parametrize("combo", UF_COMBOS, ids=combo_id)
def test_csr_sampling_union_find(sample, combo):
    link, f, sp = combo
    v = g.make_variant(sample=sample, link=link, find=f, splice=sp)
    for name, n, e in GRAPHS:
        off, cols = CSR[name]
        assert (_cc_csr(n, off, cols, v) == REF[name]).all(), name


@pytest.mark.parametrize("sample", ["none", "kout", "hb", "bfs"])
@pytest.mark.parametrize("combo", UF_FOREST, ids=combo_id)
def test_csr_spanning_forest(sample, combo):
    link, f, sp = combo
    v = g.make_variant(sample=sample, link=link, find=f, splice=sp)
    for name, n, e in GRAPHS:
        off, cols = CSR[name]
        ids, lab = g.spanning_forest_csr(n, dev(off), dev(cols), v, labels=True)
        g.gconn_sync()
        assert oracle.sf_check_arcs(n, off, cols, ids.cpu().numpy().astype(np.uint64), REF[name]) == 0, name
        assert (host_u32(lab) == REF[name]).all(), name


def _hub_bipartite(seed=11):
    """K(64, 4096) with every 7th edge listed twice, vertex ids permuted.  The
    BFS source is one of the 64 vertices of degree ~4,700 (all 1,024 seeded
    samples missing them has probability ~1e-7), and its top-down first level
    claims 4,096 vertices in one warp: more than a block stages in shared
    memory, in chunks of fewer than 32 claims where a duplicate falls, so the
    staging list overflows part way through a warp's reservation."""
    a, b = 64, 4096
    rng = np.random.default_rng(seed)
    perm = rng.permutation(a + b).astype(np.uint32)
    ai, bi = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    e = np.stack([ai.ravel(), bi.ravel()], 1)
    e = np.concatenate([e, e[::7]])
    rng.shuffle(e)
    return a + b, perm[e].astype(np.uint32)


@pytest.mark.parametrize("combo", UF_FOREST, ids=combo_id)
def test_bfs_staged_claims_overflow(combo):
    link, f, sp = combo
    n, e = _hub_bipartite()
    # plus an isolated edge and isolated vertices: the BFS reaches one component
    e = np.concatenate([e, np.array([[n, n + 1]], np.uint32)])
    n += 5
    ref = oracle.cc_uf(n, e)
    off, cols = graphgen.csr(n, e)
    v = g.make_variant(sample="bfs", link=link, find=f, splice=sp)
    assert (_cc_csr(n, off, cols, v) == ref).all()
    ids, lab = g.spanning_forest_csr(n, dev(off), dev(cols), v, labels=True)
    g.gconn_sync()
    assert oracle.sf_check_arcs(n, off, cols, ids.cpu().numpy().astype(np.uint64), ref) == 0
    assert (host_u32(lab) == ref).all()


def _two_hubs():
    """Hub A with 20,000 leaves, hub B with 10,000, A-B joined, plus a path of
    300 vertices hanging off one of A's leaves, ids permuted.  Wherever the
    BFS starts, B enters a frontier together with A's leaves: a level of low
    mean degree that holds one vertex of degree 10,001."""
    rng = np.random.default_rng(5)
    A, B = 0, 1
    la = np.arange(2, 20002)
    lb = np.arange(20002, 30002)
    path = np.arange(30002, 30302)
    e = np.concatenate([np.stack([np.full(len(la), A), la], 1), np.stack([np.full(len(lb), B), lb], 1),
                        np.array([[A, B], [la[7], path[0]]]), np.stack([path[:-1], path[1:]], 1)])
    n = 30302 + 11                              # and eleven isolated vertices
    perm = rng.permutation(n).astype(np.uint32)
    e = perm[e].astype(np.uint32)
    rng.shuffle(e)
    return n, e


@pytest.mark.parametrize("combo", UF_FOREST, ids=combo_id)
def test_bfs_hub_in_low_degree_frontier(combo):
    link, f, sp = combo
    n, e = _two_hubs()
    ref = oracle.cc_uf(n, e)
    off, cols = graphgen.csr(n, e)
    v = g.make_variant(sample="bfs", link=link, find=f, splice=sp)
    assert (_cc_csr(n, off, cols, v) == ref).all()
    ids, lab = g.spanning_forest_csr(n, dev(off), dev(cols), v, labels=True)
    g.gconn_sync()
    assert oracle.sf_check_arcs(n, off, cols, ids.cpu().numpy().astype(np.uint64), ref) == 0
    assert (host_u32(lab) == ref).all()


def _dense_graph():
    """Two cliques of 1,200 vertices (~1.44 M edges) plus a path, ids permuted:
    without sampling every vertex is active with 1,199 arcs (5 tasks of 256
    arcs), ~12,000 tasks against a task array of n + 1,024 slots, so the
    reservations run past the cap part way through some vertex's tasks."""
    rng = np.random.default_rng(21)
    k = 1200
    iu, ju = np.triu_indices(k, 1)
    e = np.concatenate([np.stack([iu, ju], 1), np.stack([iu + k, ju + k], 1),
                        np.stack([np.arange(2 * k, 2 * k + 99), np.arange(2 * k + 1, 2 * k + 100)], 1)])
    n = 2 * k + 100 + 7                         # and seven isolated vertices
    perm = rng.permutation(n).astype(np.uint32)
    e = perm[e].astype(np.uint32)
    rng.shuffle(e)
    return n, e


@pytest.mark.parametrize("spec", ["none/remcas/naive/split_one", "none/async/halve/none", "none/sv/naive/none",
                                  "none/lt/PRS/none", "hb/remcas/naive/split_one"])
def test_task_array_overflow(spec):
    n, e = _dense_graph()
    ref = oracle.cc_uf(n, e)
    off, cols = graphgen.csr(n, e)
    p = spec.split("/")
    kw = dict(sample=p[0], link=p[1])
    if p[1] == "lt":
        kw["lt"] = p[2]
    else:
        kw["find"], kw["splice"] = p[2], p[3]
    v = g.make_variant(**kw)
    for _ in range(2):                          # the second run reuses the first run's scratch
        assert (_cc_csr(n, off, cols, v) == ref).all(), spec
    if p[1] in ("remcas", "sv"):
        ids, lab = g.spanning_forest_csr(n, dev(off), dev(cols), v, labels=True)
        g.gconn_sync()
        assert oracle.sf_check_arcs(n, off, cols, ids.cpu().numpy().astype(np.uint64), ref) == 0
        assert (host_u32(lab) == ref).all()


@pytest.mark.parametrize("sample", ["none", "kout"])
def test_shiloach_vishkin(sample):
    v = g.make_variant(sample=sample, link="sv")
    for name, n, e in GRAPHS:
        if sample == "none":
            assert (_cc_coo(n, e, v) == REF[name]).all(), name
            ids, _ = g.spanning_forest(n, dev(e), v)
            g.gconn_sync()
            assert oracle.sf_check(n, e, ids.cpu().numpy().astype(np.uint64), REF[name]) == 0, name
        off, cols = CSR[name]
        assert (_cc_csr(n, off, cols, v) == REF[name]).all(), name


@pytest.mark.parametrize("rules", LT_ALL)
def test_liu_tarjan(rules):
    for sample in ["none", "hb"]:
        v = g.make_variant(sample=sample, link="lt", lt=rules)
        for name, n, e in GRAPHS:
            if sample == "none":
                assert (_cc_coo(n, e, v) == REF[name]).all(), (name, rules)
            off, cols = CSR[name]
            assert (_cc_csr(n, off, cols, v) == REF[name]).all(), (name, rules, sample)


@pytest.mark.parametrize("link", ["lp", "stergiou"])
def test_label_propagation_and_stergiou(link):
    for sample in ["none", "kout"]:
        v = g.make_variant(sample=sample, link=link)
        for name, n, e in GRAPHS:
            if sample == "none":
                assert (_cc_coo(n, e, v) == REF[name]).all(), (name, link)
            off, cols = CSR[name]
            assert (_cc_csr(n, off, cols, v) == REF[name]).all(), (name, link, sample)
    import torch
    f = torch.empty(4, dtype=torch.int64, device="cuda")
    c = torch.empty(1, dtype=torch.int64, device="cuda")
    with pytest.raises(g.GconnError) as ex:          # not root-based: no forest
        g.gconn_spanning_forest(3, 1, dev(np.array([[0, 1]], np.uint32)), f, c, None, g.make_variant(link=link))
    assert ex.value.status == g.GCONN_E_UNSUPPORTED


@pytest.mark.parametrize("rules", LT_ROOT)
def test_liu_tarjan_forest(rules):
    v = g.make_variant(link="lt", lt=rules)
    for name, n, e in GRAPHS:
        ids, _ = g.spanning_forest(n, dev(e), v)
        g.gconn_sync()
        assert oracle.sf_check(n, e, ids.cpu().numpy().astype(np.uint64), REF[name]) == 0, (name, rules)
        off, cols = CSR[name]
        ids, _ = g.spanning_forest_csr(n, dev(off), dev(cols), g.make_variant(sample="kout", link="lt", lt=rules))
        g.gconn_sync()
        assert oracle.sf_check_arcs(n, off, cols, ids.cpu().numpy().astype(np.uint64), REF[name]) == 0


def test_forest_rejects_splice():
    import torch
    e = dev(np.array([[0, 1]], np.uint32))
    f = torch.empty(2, dtype=torch.int64, device="cuda")
    c = torch.empty(1, dtype=torch.int64, device="cuda")
    with pytest.raises(g.GconnError) as ex:
        g.gconn_spanning_forest(2, 1, e, f, c, None, g.make_variant(link="remcas", splice="splice"))
    assert ex.value.status == g.GCONN_E_UNSUPPORTED


def test_host_pointers_match():
    """Host (numpy) inputs and outputs go through the same kernels."""
    name, n, e = GRAPHS[0]
    lab = np.empty(n, np.uint32)
    g.gconn_cc(n, len(e), e, lab, g.make_variant(link="remcas", splice="splice"))
    assert (lab == REF[name]).all()
    off, cols = CSR[name]
    lab2 = np.empty(n, np.uint32)
    g.gconn_cc_csr(n, off, cols, lab2, g.make_variant(sample="kout"))
    assert (lab2 == REF[name]).all()
    forest = np.empty(n, np.uint64)
    cnt = np.zeros(1, np.uint64)
    g.gconn_spanning_forest(n, len(e), e, forest, cnt, None, None)
    assert oracle.sf_check(n, e, forest[: int(cnt[0])], REF[name]) == 0


@pytest.mark.parametrize("shape", ["rmat", "star", "ragged"])
def test_large_host_csr_inputs(shape):
    """Host (staged) CSR inputs with >= 8 Mi arcs and extreme row layouts (one
    row holding every arc, a huge row amid isolated stretches, self-loops)
    give exact labels."""
    if shape == "rmat":
        n = 1 << 19
        e = graphgen.rmat(19, 1 << 23, 21)
    elif shape == "star":          # one row holds every arc
        n = 1 << 20
        e = np.stack([np.zeros(1 << 22, np.uint32), graphgen.er(n, 1 << 22, 22)[:, 1]], axis=1)
    else:                          # isolated stretches, a huge row in the middle, self-loops
        n = (1 << 20) + 37
        e = graphgen.er(n, 1 << 22, 23)
        e[: 1 << 21, 0] = np.uint32(n // 2)
        e[-1000:, 1] = e[-1000:, 0]
    off, cols = graphgen.csr(n, e)
    assert off[-1] >= 1 << 23
    ref = oracle.cc_uf(n, e)
    for spec in ("kout/remcas/naive/split_one", "kout/async/naive/none", "kout/early/halve/none"):
        s, l, f, sp = spec.split("/")
        lab = np.empty(n, np.uint32)
        g.gconn_cc_csr(n, off, cols, lab, g.make_variant(sample=s, link=l, find=f, splice=sp))
        assert (lab == ref).all(), spec


@pytest.mark.parametrize("ablation", [1, 2, 3])
@pytest.mark.parametrize("spec", ["kout/remcas/naive/split_one", "kout/early/naive/none", "hb/async/halve/none",
                                  "none/remcas/naive/splice"])
def test_ablation_forms_exact(ablation, spec):
    """The measurement forms (plain k-out, finish without vertex gathering)
    reach the same canonical labels, and valid forests."""
    s, l, f, sp = spec.split("/")
    for name, n, e in GRAPHS[:4]:
        off, cols = CSR[name]
        v = g.make_variant(sample=s, link=l, find=f, splice=sp, ablation=ablation)
        lab = g.cc_csr(n, dev(off), dev(cols), v)
        g.gconn_sync()
        assert (host_u32(lab) == REF[name]).all(), (name, spec, ablation)
        if sp != "splice":
            ids, _ = g.spanning_forest_csr(n, dev(off), dev(cols), v)
            g.gconn_sync()
            assert oracle.sf_check_arcs(n, off, cols, ids.cpu().numpy().astype(np.uint64), REF[name]) == 0


def test_release_cached_then_rerun():
    """Scratch memory is cached between calls; releasing it leaves later calls exact."""
    import torch
    name, n, e = GRAPHS[0]
    off, cols = CSR[name]
    for _ in range(2):
        lab = np.empty(n, np.uint32)
        g.gconn_cc_csr(n, off, cols, lab, g.make_variant(sample="kout"))
        assert (lab == REF[name]).all()
        torch.cuda.synchronize()
        g.gconn_release_cached()


def test_repeated_runs_stay_valid():
    """Concurrent forests differ between runs; every one must be valid."""
    name, n, e = GRAPHS[2]
    de = dev(e)
    for _ in range(20):
        ids, _ = g.spanning_forest(n, de, g.make_variant(link="async"))
        g.gconn_sync()
        assert oracle.sf_check(n, e, ids.cpu().numpy().astype(np.uint64), REF[name]) == 0


# ------------------------------------------------------------------ errors

def test_endpoint_out_of_range_reported():
    import torch
    e = np.array([[0, 1], [2, 9]], np.uint32)
    lab = torch.empty(5, dtype=torch.int32, device="cuda")
    g.gconn_cc(5, 2, dev(e), lab)
    with pytest.raises(g.GconnError) as ex:
        g.gconn_sync()
    assert ex.value.status == g.GCONN_E_RANGE
    g.gconn_sync()                      # flag cleared
    with pytest.raises(g.GconnError) as ex:
        g.gconn_cc(5, 2, e, np.empty(5, np.uint32))   # host call returns it directly
    assert ex.value.status == g.GCONN_E_RANGE


def test_invalid_arguments():
    import torch
    lab = torch.empty(5, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GconnError) as ex:
        g.gconn_cc(5, 3, None, lab)
    assert ex.value.status == g.GCONN_E_INVAL
    with pytest.raises(g.GconnError) as ex:
        g.gconn_cc(5, 1, dev(np.array([[0, 1]], np.uint32)), lab, g.make_variant(sample="kout"))
    assert ex.value.status == g.GCONN_E_UNSUPPORTED
    with pytest.raises(g.GconnError) as ex:
        g.gconn_cc(0xFFFFFFFF, 0, None, lab)
    assert ex.value.status == g.GCONN_E_INVAL


def test_iteration_cap_reports_nonconverged():
    """A cap of one loop step on a contended star (every edge competes for
    the centre, the largest id) must stop with E_NONCONVERGED, not hang."""
    import torch
    n = 20001
    star = np.stack([np.full(n - 1, n - 1), np.arange(n - 1)], 1).astype(np.uint32)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    g.gconn_cc(n, n - 1, dev(star), lab, g.make_variant(link="async", iter_cap=1))
    with pytest.raises(g.GconnError) as ex:
        g.gconn_sync()
    assert ex.value.status == g.GCONN_E_NONCONVERGED
    # the context stays usable
    assert (_cc_coo(n, star, g.make_variant()) == oracle.cc_uf(n, star)).all()


def test_empty_and_zero_vertex_inputs():
    import torch
    lab = torch.empty(0, dtype=torch.int32, device="cuda")
    g.gconn_cc(0, 0, None, lab)
    g.gconn_sync()
    with pytest.raises(g.GconnError):
        g.gconn_cc(0, 1, dev(np.array([[0, 0]], np.uint32)), lab)
