"""Captured plans (one CUDA graph per static pass): replays give the
oracle's labels, also after the input buffers are refilled."""
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


def _variant(spec):
    s, l, f, sp = spec.split("/")
    if l == "lt":
        return g.make_variant(sample=s, link=l, lt=f)
    return g.make_variant(sample=s, link=l, find=f, splice=sp)


# BFS sampling and the round-based finishes loop on the device, so they are
# captured like the rest
@pytest.mark.parametrize("spec", ["kout/remcas/naive/split_one", "hb/async/compress/none", "none/early/naive/none",
                                  "kout/jtb/twotrysplit/none", "kout/hooks/halve/none",
                                  "bfs/remcas/naive/split_one", "bfs/async/naive/none", "bfs/jtb/naive/none",
                                  "kout/sv/naive/none", "none/sv/naive/none", "hb/lt/PRF/none", "none/lt/CUSA/none",
                                  "kout/lp/naive/none", "none/stergiou/naive/none"])
def test_csr_plan_replay_and_refill(spec):
    import torch
    n = 30_011
    v = _variant(spec)
    e1 = graphgen.rmat(15, 90_000, 1) % np.uint32(n)
    e2 = graphgen.er(n, 90_000, 2)
    off1, cols1 = graphgen.csr(n, e1)
    off2, cols2 = graphgen.csr(n, e2)
    d_off, d_cols = dev(off1), dev(cols1)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    p = g.gconn_plan_create_cc_csr(n, d_off, d_cols, lab, v)
    for _ in range(2):
        lab.fill_(-1)
        g.gconn_plan_run(p)
        g.gconn_sync()
        assert (host_u32(lab) == oracle.cc_uf(n, e1)).all()
    d_off.copy_(dev(off2))                       # same n and arc count: new graph, same plan
    d_cols.copy_(dev(cols2))
    g.gconn_plan_run(p)
    g.gconn_sync()
    assert (host_u32(lab) == oracle.cc_uf(n, e2)).all()
    g.gconn_plan_destroy(p)


def test_coo_plans_incl_round_finishes():
    import torch
    n = 5000
    e = graphgen.er(n, 7000, 3)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    p = g.gconn_plan_create_cc(n, len(e), dev(e), lab, g.make_variant(link="remcas", splice="splice"))
    g.gconn_plan_run(p)
    g.gconn_sync()
    assert (host_u32(lab) == oracle.cc_uf(n, e)).all()
    g.gconn_plan_destroy(p)
    de = dev(e)
    ref = oracle.cc_uf(n, e)
    for kw in (dict(link="sv"), dict(link="lt", lt="PRF"), dict(link="lt", lt="EUSA"), dict(link="lp"),
               dict(link="stergiou")):
        p = g.gconn_plan_create_cc(n, len(e), de, lab, g.make_variant(**kw))
        for _ in range(2):
            lab.fill_(-1)
            g.gconn_plan_run(p)
            g.gconn_sync()
            assert (host_u32(lab) == ref).all(), kw
        g.gconn_plan_destroy(p)
    with pytest.raises(g.GconnError):
        g.gconn_plan_create_cc(n, len(e), e, lab)        # host edges cannot be captured


def test_profiled_plan_records_kernels():
    import torch
    n = 20_000
    e = graphgen.er(n, 50_000, 4)
    off, cols = graphgen.csr(n, e)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    g.gconn_profile_enable(True)
    p = g.gconn_plan_create_cc_csr(n, dev(off), dev(cols), lab, g.make_variant(sample="kout"))
    g.gconn_profile_enable(False)
    g.gconn_profile_reset()
    c0 = g.gconn_launch_count()
    for _ in range(3):
        g.gconn_plan_run(p)
        g.gconn_sync()
        g.gconn_profile_sync()
    prof = g.gconn_profile_get()
    assert prof["kout"][0] == 3 and prof["finalize"][0] == 3
    assert all(ms > 0 for _, ms in prof.values())          # the captured pairs really time each replay
    assert g.gconn_launch_count() - c0 == 3 * sum(1 for _ in prof) or g.gconn_launch_count() > c0
    assert (host_u32(lab) == oracle.cc_uf(n, e)).all()
    g.gconn_plan_destroy(p)


def test_profile_select_times_only_named_kernels():
    import torch
    n = 20_000
    e = graphgen.er(n, 50_000, 5)
    off, cols = graphgen.csr(n, e)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    g.gconn_profile_select("kout")
    g.gconn_profile_enable(True)
    p = g.gconn_plan_create_cc_csr(n, dev(off), dev(cols), lab, g.make_variant(sample="kout"))
    g.gconn_profile_enable(False)
    g.gconn_profile_select(None)
    g.gconn_profile_reset()
    for _ in range(2):
        g.gconn_plan_run(p)
        g.gconn_sync()
        g.gconn_profile_sync()
    prof = g.gconn_profile_get()
    assert set(prof) == {"kout"} and prof["kout"][0] == 2 and prof["kout"][1] > 0
    assert (host_u32(lab) == oracle.cc_uf(n, e)).all()
    g.gconn_plan_destroy(p)
    g.gconn_profile_reset()


@pytest.mark.parametrize("spec", ["kout/remcas/naive/split_one", "hb/early/naive/none", "none/async/halve/none",
                                  "bfs/remcas/naive/split_one", "none/sv/naive/none", "kout/lt/PRS/none"])
def test_forest_plan_replays_valid_forests(spec):
    import torch
    n = 25_013
    e = graphgen.rmat(15, 70_000, 9) % np.uint32(n)
    off, cols = graphgen.csr(n, e)
    ref = oracle.cc_uf(n, e)
    forest = torch.empty(n, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    p = g.gconn_plan_create_forest_csr(n, dev(off), dev(cols), forest, cnt, lab, _variant(spec))
    for _ in range(2):
        g.gconn_plan_run(p)
        g.gconn_sync()
        c = int(cnt.item())
        arcs = forest[:c].cpu().numpy().astype(np.uint64)
        assert oracle.sf_check_arcs(n, off, cols, arcs, ref) == 0
        assert (host_u32(lab) == ref).all()
    g.gconn_plan_destroy(p)
    with pytest.raises(g.GconnError) as ex:       # splice is not root-based: no forests
        g.gconn_plan_create_forest_csr(n, dev(off), dev(cols), forest, cnt, None,
                                       g.make_variant(sample="kout", link="remcas", splice="splice"))
    assert ex.value.status == g.GCONN_E_UNSUPPORTED
