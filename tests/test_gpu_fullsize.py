"""Parity at the full sizes of the five workloads, in the configuration the
benchmark times (RMAT scale 22) and the others: canonical labels bit-exact
with the oracle where it finishes in seconds, sampled graphs / prefixes and
size-independent invariants elsewhere."""
import numpy as np
import pytest

import graphgen
import oracle
import paper_2008_11839_gb300 as g
from gpu_util import UF_COMBOS, combo_id, dev, host_u32

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    g.build()


@pytest.fixture(scope="module")
def er_c1():
    n, m = 65_536, 1_048_576
    e = graphgen.er(n, m, 0x6C0A0001)
    return n, e, oracle.cc_uf(n, e)


@pytest.mark.parametrize("combo", UF_COMBOS, ids=combo_id)
def test_c1_er_full(er_c1, combo):
    n, e, ref = er_c1
    link, f, sp = combo
    lab = g.cc(n, dev(e), g.make_variant(link=link, find=f, splice=sp))
    g.gconn_sync()
    assert (host_u32(lab) == ref).all()


@pytest.fixture(scope="module")
def rmat_c2():
    n = 1 << 22
    e = graphgen.rmat(22, 1 << 26, 0x6C0A0002)
    off, cols = graphgen.csr(n, e)
    return n, e, off, cols, oracle.cc_uf(n, e)


@pytest.mark.parametrize("spec", ["kout/remcas/naive/split_one", "kout/async/compress/none",
                                  "hb/early/naive/none", "bfs/remcas/naive/split_one", "none/remcas/naive/split_one"])
def test_c2_rmat_s22_full(rmat_c2, spec):
    n, e, off, cols, ref = rmat_c2
    s, l, f, sp = spec.split("/")
    lab = g.cc_csr(n, dev(off), dev(cols), g.make_variant(sample=s, link=l, find=f, splice=sp))
    g.gconn_sync()
    assert (host_u32(lab) == ref).all()


@pytest.mark.parametrize("spec", ["kout/remcas/naive/split_one", "hb/remcas/naive/split_one",
                                  "bfs/async/naive/none"])
def test_c2_rmat_s22_full_offsets32(rmat_c2, spec):
    """The benchmark's configuration: uint32 offsets (2^27 arcs < 2^32)."""
    n, e, off, cols, ref = rmat_c2
    s, l, f, sp = spec.split("/")
    lab = g.cc_csr(n, dev(off.astype(np.uint32)), dev(cols), g.make_variant(sample=s, link=l, find=f, splice=sp))
    g.gconn_sync()
    assert (host_u32(lab) == ref).all()


def test_c2_forest_and_coo_full(rmat_c2):
    n, e, off, cols, ref = rmat_c2
    ids, lab = g.spanning_forest_csr(n, dev(off), dev(cols),
                                     g.make_variant(sample="kout", link="remcas", splice="split_one"), labels=True)
    g.gconn_sync()
    assert oracle.sf_check_arcs(n, off, cols, ids.cpu().numpy().astype(np.uint64), ref) == 0
    lab = g.cc(n, dev(e), g.make_variant(link="remcas", splice="split_one"))
    g.gconn_sync()
    assert (host_u32(lab) == ref).all()


@pytest.fixture(scope="module")
def grid_c3():
    n, e = graphgen.grid_paths(4096, 0.05, 64, 1 << 18, 0x6C0A0003)
    return n, e, oracle.cc_uf(n, e)


@pytest.mark.parametrize("kind,spec", [("coo", "none/remcas/naive/split_one"), ("coo", "none/async/halve/none"),
                                       ("coo", "none/sv/naive/none"), ("coo", "none/lt/PRF/none"),
                                       ("csr", "kout/remcas/naive/split_one"), ("csr", "bfs/async/naive/none")])
def test_c3_grid_paths_full(grid_c3, kind, spec):
    n, e, ref = grid_c3
    s, l, f, sp = spec.split("/")
    v = g.make_variant(sample=s, link=l, find=f if l != "lt" else "naive", splice=sp, lt=f if l == "lt" else "PRF")
    if kind == "coo":
        lab = g.cc(n, dev(e), v)
    else:
        off, cols = graphgen.csr(n, e)
        lab = g.cc_csr(n, dev(off), dev(cols), v)
    g.gconn_sync()
    got = host_u32(lab)
    assert (got == ref).all()
    # closed form: the 64 permuted paths are exactly 64 labels, each the path minimum
    pi = graphgen.path_permutation(64, 1 << 18, 0x6C0A0003).astype(np.int64) + 4096 * 4096
    for j in range(0, 64, 9):
        ids = pi[j << 18:(j + 1) << 18]
        assert (got[ids] == ids.min()).all()


def test_c4_batched_full():
    import torch
    G = 4096
    vo, eo, e = graphgen.batched(G, 0x6C0A0004)
    lab = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    de = dev(e)
    h = g.gconn_batch_create(G, vo, eo, de, lab)
    g.gconn_batch_run(h)
    g.gconn_sync()
    got = host_u32(lab)
    g.gconn_batch_destroy(h)
    ref = oracle.batched_cc(vo, eo, e)                    # O1 on every graph (a few seconds)
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, f"{bad.size} labels differ, first graph {int(np.searchsorted(vo, bad[0], 'right')) - 1}"


def test_c5_incremental_full():
    """The 2^28-insert stream: the first batches answer every query exactly as
    the replay does; after the whole stream the labels equal static
    components of everything inserted."""
    import torch
    n = 1 << 24
    seed = 0x6C0A0005
    h = graphgen.hash_fill(seed, 11, 0, 4096)
    sizes, tot = [], 0
    for x in h:
        b = min(int(10 ** (3 + 5 * ((int(x) >> 11) * 2.0 ** -53))), (1 << 28) - tot)
        sizes.append(b)
        tot += b
        if tot >= 1 << 28:
            break
    perm = graphgen.permutation(n, seed, 6)
    inc = g.Incremental(n, g.make_variant(link="async"))
    ref = oracle.Incremental(n)
    s = 0
    exact_batches = 0
    for b in sizes:
        ins = graphgen.rmat_range(24, s, b, seed, perm=perm)
        qs = graphgen.pairs_range(n, s, b, seed)
        inc.insert(dev(ins))
        out = inc.query(dev(qs))
        if s < (1 << 26):                                # replay the prefix exactly
            ref.insert(ins)
            assert (out.cpu().numpy() == ref.query(qs)).all()
            exact_batches += 1
        s += b
    g.gconn_sync()
    assert exact_batches >= 1
    allins = graphgen.rmat_range(24, 0, 1 << 28, seed, perm=perm)
    assert (host_u32(inc.labels()) == oracle.cc_uf(n, allins)).all()
    inc.close()
