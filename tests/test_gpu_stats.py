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


@pytest.mark.parametrize("sample", ["kout", "hb"])
@pytest.mark.parametrize("link", ["async", "remcas"])
def test_stats_match_sampled_components(sample, link):
    import torch
    n = 6000
    e = graphgen.rmat(13, 30_000, 17) % np.uint32(n)
    off, cols = graphgen.csr(n, e)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    st = g.gconn_cc_csr_stats(n, dev(off), dev(cols), lab, g.make_variant(sample=sample, link=link))
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
    # L_max is the mode of seeded samples: its component is the largest w.h.p.
    assert d["lmax_vertices"] == np.bincount(lab0).max()
