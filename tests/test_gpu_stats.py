"""Sampling instrumentation (Section 4.3, Table 4): the counts reported by
gconn_cc_csr_stats equal the ones computed from the oracle's components of
the sampled subgraph, which is deterministic for k-out and HB."""
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


def _sampled_edges(n, off, cols, sample, k=2, N=4):
    out = []
    for v in range(n):
        lo, hi = int(off[v]), int(off[v + 1])
        if sample == "kout":
            out += [(v, int(cols[a])) for a in range(lo, min(hi, lo + k))]
        else:
            if hi > lo and cols[lo] < v:
                out.append((v, int(cols[lo])))           # step 1 hook
            else:                                        # still a root: first N edges
                out += [(v, int(cols[a])) for a in range(lo, min(hi, lo + N))]
    return np.array(out, np.uint32).reshape(-1, 2)


def _expected_lmax(n, lab0, seed):
    """GetMostFrequentLabel over the 1,024 seeded sample positions: position j
    is the upper 32 bits of SplitMix64 output j of the variant's seed, scaled
    to [0, n); the mode of the sampled labels there, ties to the smaller."""
    xs = np.array([((graphgen.splitmix64_at(seed, j) >> 32) * n) >> 32 for j in range(1024)], np.int64)
    vals, counts = np.unique(lab0[xs], return_counts=True)
    return int(vals[counts == counts.max()].min())


@pytest.mark.parametrize("seed", [0x6C0A0001, 0x1234567])
@pytest.mark.parametrize("sample", ["kout", "hb"])
@pytest.mark.parametrize("link", ["async", "remcas"])
def test_stats_match_sampled_components(sample, link, seed):
    import torch
    n = 6000
    e = graphgen.rmat(13, 30_000, 17) % np.uint32(n)
    off, cols = graphgen.csr(n, e)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    st = g.gconn_cc_csr_stats(n, dev(off), dev(cols), lab, g.make_variant(sample=sample, link=link, seed=seed))
    assert (host_u32(lab) == oracle.cc_uf(n, e)).all()
    lab0 = oracle.cc_uf(n, _sampled_edges(n, off, cols, sample))
    deg = np.diff(off).astype(np.int64)
    rows = np.repeat(np.arange(n), deg)
    d = st.as_dict()
    L = d["lmax"]
    assert d["n"] == n and d["arcs"] == off[-1]
    assert d["sampled_components"] == len(np.unique(lab0))
    assert d["lmax_vertices"] == int((lab0 == L).sum())
    assert d["inter_component_arcs"] == int((lab0[rows] != lab0[cols]).sum())
    act = (lab0 != L) & (deg > 0)
    assert d["active_vertices"] == int(act.sum()) and d["active_arcs"] == int(deg[act].sum())
    if sample == "kout":
        assert d["sample_arcs_inspected"] == int(np.minimum(deg, 2).sum())
    assert 0 < d["sample_ms"] <= d["total_ms"]
    # L_max is exactly the mode of the seeded samples' sampled labels
    assert L == _expected_lmax(n, lab0, seed)
    # and its component is the largest w.h.p.
    assert d["lmax_vertices"] == np.bincount(lab0).max()


@pytest.mark.parametrize("seed", [1, 2, 3, 0x6C0A0001])
def test_lmax_between_equal_components_follows_the_samples(seed):
    """Two equal components (even ids / odd ids): which one is L_max depends on
    the exact sampled positions and the tie rule, so this pins them."""
    import torch
    n = 8000
    h = n // 2
    ea = graphgen.er(h, 40_000, 31) * np.uint32(2)                 # even ids 0, 2, ...
    eb = graphgen.er(h, 40_000, 32) * np.uint32(2) + np.uint32(1)  # odd ids 1, 3, ...
    e = np.concatenate([ea, eb])
    off, cols = graphgen.csr(n, e)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    st = g.gconn_cc_csr_stats(n, dev(off), dev(cols), lab, g.make_variant(sample="kout", link="remcas", seed=seed))
    lab0 = oracle.cc_uf(n, _sampled_edges(n, off, cols, "kout"))
    assert st.as_dict()["lmax"] == _expected_lmax(n, lab0, seed)
    assert (host_u32(lab) == oracle.cc_uf(n, e)).all()


@pytest.mark.parametrize("link", ["remcas", "remlock"])
def test_deferred_splice_unions_keep_the_sampled_partition(link):
    """A k-out union that exceeds its step budget is finished later by the
    retry kernel.  With SpliceAtomic the abandoned climb may already have moved
    a subtree into the other tree, so it must resume from its current pair,
    not its endpoints; otherwise (rarely) part of a set is left behind and the
    sampled partition has an extra component.  Many repetitions make a
    resumption bug show."""
    import torch
    n = 6000
    e = graphgen.rmat(13, 30_000, 17) % np.uint32(n)
    off, cols = graphgen.csr(n, e)
    want = len(np.unique(oracle.cc_uf(n, _sampled_edges(n, off, cols, "kout"))))
    ref = oracle.cc_uf(n, e)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    d_off, d_cols = dev(off), dev(cols)
    v = g.make_variant(sample="kout", link=link, splice="splice")
    for _ in range(600):
        st = g.gconn_cc_csr_stats(n, d_off, d_cols, lab, v)
        assert st.as_dict()["sampled_components"] == want
    assert (host_u32(lab) == ref).all()
