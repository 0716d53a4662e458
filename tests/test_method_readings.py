"""Pins for the readings of the paper's rules (sequential restatements in
oracle/method_ref.py) against the oracle's definition.

Every sampling x linking x find (x splice) combination, Shiloach-Vishkin and
the 16 Liu-Tarjan variants must reach the component labels of the definition,
and every recorded spanning forest must pass the checker.  Planted wrong
readings show the checks have teeth.
"""
import numpy as np
import pytest

import graphgen
import oracle
from oracle import method_ref as mr


def _graphs():
    out = []
    for seed in range(3):
        n = 60
        out.append((n, graphgen.er(n, 45 + 20 * seed, 100 + seed)))
    out.append((128, graphgen.rmat(7, 300, 7)))
    n, e = graphgen.grid_paths(6, 0.2, 3, 12, 8)
    out.append((n, e))
    out.append((10, np.zeros((0, 2), np.uint32)))
    return out


GRAPHS = _graphs()

COMBOS = []
for link in ["async", "hooks", "early"]:
    for f in ["naive", "compress", "split", "halve"]:
        COMBOS.append((link, f, "splice"))
for f in ["naive", "split", "halve"]:
    for sp in ["split_one", "halve_one", "splice"]:
        COMBOS.append(("remcas", f, sp))
COMBOS += [("jtb", "naive", "splice"), ("jtb", "twotrysplit", "splice")]
for f in ["naive", "split", "halve"]:
    for sp in ["split_one", "halve_one", "splice"]:
        COMBOS.append(("remlock", f, sp))
COMBOS += [("afforest", "naive", "splice"), ("eclcc", "naive", "splice")]


@pytest.mark.parametrize("sample", ["none", "kout", "hb", "bfs"])
@pytest.mark.parametrize("link,find,splice", COMBOS)
def test_static_conn_reading(sample, link, find, splice):
    for n, e in GRAPHS:
        ref = oracle.cc_uf(n, e)
        off, cols = graphgen.csr(n, e)
        lab, sf = mr.static_conn_csr(off.tolist(), cols.tolist(), sample, link, find, splice)
        assert (np.array(lab, np.uint32) == ref).all()
        assert oracle.sf_check_arcs(n, off, cols, np.array(sf, np.uint64), ref) == 0


def test_coo_edge_order_irrelevant():
    n, e = GRAPHS[0]
    ref = oracle.cc_uf(n, e)
    rng = np.random.default_rng(3)
    for link, f, sp in COMBOS:
        uf = mr.UF(n, link, f, sp)
        sf = mr.finish_coo(e.tolist(), uf, order=rng.permutation(len(e)).tolist())
        assert (np.array(uf.labels(), np.uint32) == ref).all()
        assert oracle.sf_check(n, e, np.array(sf, np.uint64), ref) == 0


def test_shiloach_vishkin_reading():
    for n, e in GRAPHS:
        lab, rounds = mr.shiloach_vishkin(n, [tuple(x) for x in e.tolist()])
        assert (np.array(lab, np.uint32) == oracle.cc_uf(n, e)).all()


@pytest.mark.parametrize("variant", mr.LT_VARIANTS)
def test_liu_tarjan_reading(variant):
    for n, e in GRAPHS:
        lab, rounds = mr.liu_tarjan(n, [tuple(x) for x in e.tolist()], variant)
        assert (np.array(lab, np.uint32) == oracle.cc_uf(n, e)).all()


def test_most_frequent_label_tie_rule():
    assert mr.most_frequent_label([3, 3, 1, 1, 2]) == 1
    assert mr.most_frequent_label([5, 4, 4, 5, 5]) == 5


def test_wrong_skip_rule_is_caught():
    """Skipping edges of L_max vertices is only sound when every edge is seen
    from both endpoints (symmetric CSR).  Over a one-direction COO list the
    same rule drops edges: the definition catches it."""
    n = 6
    # sampled state: {0,1,2} merged (label 0 = L_max); edge (0, 5) listed once
    edges = [(0, 1), (1, 2), (0, 5), (3, 4)]
    uf = mr.UF(n)
    for u, v in edges[:2]:
        uf.union(u, v)
    mr.full_shortcut(uf.P)
    lmax = mr.most_frequent_label(uf.P)
    lab0 = list(uf.P)
    for u, v in edges:
        if lab0[u] == lmax:          # vertex-skip rule applied to one-direction COO
            continue
        uf.union(u, v)
    wrong = np.array(uf.labels(), np.uint32)
    ref = oracle.cc_uf(n, np.array(edges, np.uint32))
    assert not (wrong == ref).all()
    # the COO reading (skip an edge only when both endpoints are L_max) is right
    uf = mr.UF(n)
    for u, v in edges[:2]:
        uf.union(u, v)
    mr.full_shortcut(uf.P)
    lab0 = list(uf.P)
    for u, v in edges:
        if lab0[u] == lmax and lab0[v] == lmax:
            continue
        uf.union(u, v)
    assert (np.array(uf.labels(), np.uint32) == ref).all()


def test_parent_connect_to_endpoints_stalls():
    """Reading check for ParentConnect: if the parents of an edge's endpoints
    were sent to the endpoints themselves, root-only updates could never move a
    non-root endpoint, and PRS would stop with two components unmerged."""
    n = 4
    edges = [(0, 2), (1, 3), (2, 3)]
    P = [0, 1, 0, 1]                      # 2 -> 0 and 3 -> 1 already
    # wrong reading: 2 receives P[3] = 1, 3 receives P[2] = 0, both non-roots
    msg = {2: 1, 3: 0}
    newP = [min(P[x], msg.get(x, P[x])) if P[x] == x else P[x] for x in range(n)]
    assert newP == P                       # no progress: would end unmerged
    lab, _ = mr.liu_tarjan(n, edges, "PRS", labels=P)
    assert lab == [0, 0, 0, 0]


def test_label_propagation_and_stergiou_readings():
    for n, e in GRAPHS:
        el = [tuple(x) for x in e.tolist()]
        ref = oracle.cc_uf(n, e)
        lab, _ = mr.label_propagation(n, el)
        assert (np.array(lab, np.uint32) == ref).all()
        lab, _ = mr.stergiou(n, el)
        assert (np.array(lab, np.uint32) == ref).all()


def test_label_propagation_rounds_track_diameter():
    """LP needs about one round per hop of the longest shortest path: a path
    of k vertices with ids increasing along it takes k rounds (Section 4.2
    attributes LP's slowness on high-diameter graphs to this)."""
    k = 40
    path = [(i, i + 1) for i in reversed(range(k - 1))]   # far end first: one hop per round
    lab, rounds = mr.label_propagation(k, path)
    assert lab == [0] * k and rounds >= k - 1


def _same_set_lockstep(x, y, P):
    """The GPU query walk (query batches and serving query segments under the
    naive find): both endpoints climb one step per iteration, and a walk that
    stands on a root above the other walk's vertex answers "different"."""
    while x != y:
        px, py = P[x], P[y]
        rx, ry = px == x, py == y
        if (rx and (ry or y < x)) or (ry and x < y):
            return False
        x, y = px, py
    return True


def _same_set_lockstep_wrong(x, y, P):   # planted: the early exit tests the wrong side
    while x != y:
        px, py = P[x], P[y]
        rx, ry = px == x, py == y
        if (rx and (ry or y > x)) or (ry and x > y):
            return False
        x, y = px, py
    return True


LOCKSTEP_RULES = [("async", "naive", "splice"), ("hooks", "naive", "splice"), ("early", "naive", "splice"),
                  ("remcas", "naive", "split_one"), ("remcas", "naive", "splice"), ("remlock", "naive", "halve_one"),
                  ("afforest", "naive", "splice"), ("eclcc", "naive", "splice")]


@pytest.mark.parametrize("link,find,splice", LOCKSTEP_RULES)
def test_lockstep_query_equals_root_comparison(link, find, splice):
    """Every non-JTB rule keeps P[v] <= v, so a root is the smallest vertex of
    its tree; on the forests these rules build (whole graphs and prefixes of
    their edge lists), the lock-step walk answers exactly Find(u) == Find(v)
    for every pair, and the planted wrong early exit is caught."""
    caught = False
    for n, e in GRAPHS[:4]:
        for cut in (len(e) // 3, len(e)):
            uf = mr.UF(n, link=link, find=find, splice=splice)
            for u, v in e[:cut].tolist():
                if u != v:
                    uf.union(u, v)
            P = uf.P
            assert all(P[v] <= v for v in range(n))
            roots = [uf.root(v) for v in range(n)]
            for x in range(n):
                for y in range(n):
                    want = roots[x] == roots[y]
                    assert _same_set_lockstep(x, y, P) == want, (x, y)
                    caught |= _same_set_lockstep_wrong(x, y, P) != want
    assert caught


def _rem_cas_budget(u, v, P, splice, steps):
    """Union-Rem-CAS (Algorithm 11) that gives up after `steps` splice steps
    and returns the pair its climb stood on (None once linked or joined)."""
    ru, rv = u, v
    while P[ru] != P[rv]:
        if P[ru] < P[rv]:
            ru, rv = rv, ru
        if ru == P[ru] and mr.cas(P, ru, ru, P[rv]):
            return None
        ru = splice(ru, rv, P)
        steps -= 1
        if steps == 0:
            return ru, rv
    return None


def _labels_of(P):
    roots = [mr.find_naive(v, P) for v in range(len(P))]
    low = {}
    for v, r in enumerate(roots):
        low.setdefault(r, v)
    return np.array([low[r] for r in roots], np.uint32)


@pytest.mark.parametrize("splice", ["split_one", "halve_one", "splice"])
def test_abandoned_union_resumes_from_its_current_pair(splice):
    """R34: a union abandoned after a few steps and finished later must resume
    from the pair its climb stood on.  With SpliceAtomic, restarting from the
    endpoints can drop part of a set (the splice already moved a subtree of
    u's set into v's tree, so u and v look joined while the rest of u's set is
    not linked): the planted restart is caught there, and resuming is exact
    for every splice rule."""
    rng = np.random.default_rng(5)
    lost = False
    for trial in range(60):
        n = int(rng.integers(8, 40))
        e = rng.integers(0, n, size=(int(rng.integers(n, 3 * n)), 2)).astype(np.uint32)
        want = oracle.cc_uf(n, e)
        budgets = rng.integers(1, 3, size=len(e))
        for resume in (True, False):
            P = list(range(n))
            later = []
            for (u, v), b in zip(e.tolist(), budgets.tolist()):
                if u == v:
                    continue
                stop = _rem_cas_budget(u, v, P, mr.SPLICES[splice], b)
                if stop is not None:
                    later.append(stop if resume else (u, v))
            for u, v in later:
                mr.union_rem_cas(u, v, P, mr.find_naive, mr.SPLICES[splice])
            same = (_labels_of(P) == want).all()
            if resume:
                assert same, (trial, splice)
            else:
                lost |= not same
    assert lost == (splice == "splice")


def _chained_bfs(off, cols, s, hops, arcs_cap, bottom_up, rng):
    """A sequential run of BFS sampling in the chained form (the BFS reading):
    on a chained level a frontier vertex is expanded and then one of its
    fresh claims right away, up to `hops` vertices; a row longer than
    `arcs_cap` is not scanned in a chain but queued again (marked for the next
    level) and the next level expands whole frontier vertices; levels in
    `bottom_up` let every unreached vertex look for a neighbour marked with the
    current level.  Frontier order is shuffled to stand in for concurrency.
    Returns the level marks and each reached vertex's recorded arc."""
    n = len(off) - 1
    inf = -1
    dist, par = [inf] * n, [None] * n
    dist[s] = 0
    frontier, level, heavy = [s], 0, False
    while frontier:
        nxt, nheavy = [], False
        if level in bottom_up:
            for v in range(n):
                if dist[v] == inf:
                    for a in range(off[v], off[v + 1]):
                        if dist[cols[a]] == level:
                            dist[v], par[v] = level + 1, a
                            nxt.append(v)
                            break
        else:
            order = list(frontier)
            rng.shuffle(order)
            for x in order:
                for hop in range(hops if not heavy else 1):
                    if not heavy and off[x + 1] - off[x] > arcs_cap:
                        dist[x] = level + 1
                        nxt.append(x)
                        nheavy = True
                        break
                    nv = None
                    for a in range(off[x], off[x + 1]):
                        y = int(cols[a])
                        if dist[y] == inf:
                            dist[y], par[y] = level + 1, a
                            if nv is None and not heavy and hop + 1 < hops:
                                nv = y
                            else:
                                nxt.append(y)
                    if nv is None:
                        break
                    x = nv
        frontier, heavy, level = nxt, nheavy, level + 1
    return dist, par


@pytest.mark.parametrize("seed", range(12))
def test_chained_bfs_reaches_the_component_with_a_valid_tree(seed):
    """The BFS reading: chaining, re-queued long rows and bottom-up levels
    that take any vertex marked in the last level as a parent reach exactly
    the source's component, and the recorded arcs form a spanning tree of it."""
    rng = np.random.default_rng(seed)
    import random
    prng = random.Random(seed)
    graphs = GRAPHS[:5] + [(400, graphgen.ba(400, 3, 5 + seed)) if hasattr(graphgen, "ba") else GRAPHS[0]]
    for n, e in graphs:
        if n == 0 or len(e) == 0:
            continue
        off, cols = graphgen.csr(n, e)
        s = int(rng.integers(n))
        hops = int(rng.integers(1, 17))
        cap = int(rng.integers(1, 9))
        bottom_up = set(int(x) for x in rng.integers(0, 12, size=int(rng.integers(0, 4))))
        dist, par = _chained_bfs(off, cols, s, hops, cap, bottom_up, prng)
        lab = oracle.cc_uf(n, e)
        reached = {v for v in range(n) if dist[v] != -1}
        assert reached == {v for v in range(n) if lab[v] == lab[s]}
        # the recorded arcs: one per reached vertex but the source, each an arc
        # between two reached vertices, together acyclic
        owner = np.searchsorted(off, np.arange(len(cols)), side="right") - 1
        parent = list(range(n))

        def root(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x
        arcs = [par[v] for v in reached if v != s]
        assert None not in arcs and len(arcs) == len(reached) - 1
        for v in reached:
            if v == s:
                continue
            a = par[v]
            u, w = int(owner[a]), int(cols[a])
            assert v in (u, w) and u in reached and w in reached
            ru, rw = root(u), root(w)
            assert ru != rw
            parent[ru] = rw
