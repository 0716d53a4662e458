"""Pins for the CPU oracle: brute force, closed forms, hand-derived fixtures,
invariants, and planted mistakes that the pins must catch.

The oracle computes the definition of connected components (Section 2,
"Graph Connectivity Problems"); nothing here compares it with itself.
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from conftest import read_cc_golden, read_inc_golden

# --------------------------------------------------------------- brute force


def closure_labels(n, edges):
    """Min-id labels from the reflexive-transitive closure of the adjacency
    matrix (Warshall's algorithm), independent of union-find and BFS."""
    R = np.eye(n, dtype=bool)
    for u, v in edges:
        R[u, v] = R[v, u] = True
    for k in range(n):
        R |= R[:, k:k + 1] & R[k:k + 1, :]
    return np.array([int(np.flatnonzero(R[v])[0]) for v in range(n)], dtype=np.uint32)


PAIRS5 = list(itertools.combinations(range(5), 2))


@pytest.mark.parametrize("impl", [oracle.cc_uf, oracle.cc_bfs], ids=["O1", "O2"])
def test_all_simple_graphs_on_5_vertices(impl):
    for mask in range(1 << len(PAIRS5)):
        edges = [PAIRS5[i] for i in range(len(PAIRS5)) if mask >> i & 1]
        e = np.array(edges, dtype=np.uint32).reshape(-1, 2)
        assert (impl(5, e) == closure_labels(5, edges)).all(), edges


@pytest.mark.parametrize("impl", [oracle.cc_uf, oracle.cc_bfs], ids=["O1", "O2"])
def test_random_multigraphs_up_to_12(impl):
    rng = np.random.default_rng(1234)
    for _ in range(400):
        n = int(rng.integers(1, 13))
        m = int(rng.integers(0, 3 * n))
        e = rng.integers(0, n, size=(m, 2)).astype(np.uint32)
        assert (impl(n, e) == closure_labels(n, e.tolist())).all()


def test_o1_equals_o2_on_generated_graphs():
    cases = [(1 << 14, graphgen.er(1 << 14, 1 << 13, 3)),
             (1 << 14, graphgen.er(1 << 14, 1 << 16, 4)),
             (1 << 15, graphgen.rmat(15, 1 << 18, 5))]
    n, e = graphgen.grid_paths(64, 0.3, 8, 300, 6)
    cases.append((n, e))
    for n, e in cases:
        assert (oracle.cc_uf(n, e) == oracle.cc_bfs(n, e)).all()


# -------------------------------------------------------------- closed forms


def test_empty_graph_is_identity():
    for n in (0, 1, 7, 1000):
        e = np.zeros((0, 2), np.uint32)
        assert (oracle.cc_uf(n, e) == np.arange(n)).all()
        assert (oracle.cc_bfs(n, e) == np.arange(n)).all()


def test_paths_stars_cliques_selfloops():
    n = 257
    path = np.stack([np.arange(n - 1), np.arange(1, n)], 1).astype(np.uint32)
    rng = np.random.default_rng(0)
    for e in (path, path[::-1].copy(), path[rng.permutation(n - 1)], path[:, ::-1].copy()):
        assert (oracle.cc_uf(n, e) == 0).all()
    star = np.stack([np.full(n - 2, n - 1), np.arange(1, n - 1)], 1).astype(np.uint32)
    lab = oracle.cc_uf(n, star)
    assert lab[0] == 0 and (lab[1:] == 1).all()
    clique = np.array(list(itertools.combinations(range(40), 2)), np.uint32)
    assert (oracle.cc_uf(40, clique) == 0).all()
    loops = np.stack([np.arange(n), np.arange(n)], 1).astype(np.uint32)
    assert (oracle.cc_uf(n, loops) == np.arange(n)).all()


def test_permuted_paths_closed_form():
    """64-style permuted paths (the high-diameter workload): the labels are the
    minimum id on each path, computed straight from the generator's layout."""
    side, npaths, plen, seed = 32, 16, 500, 11
    n, e = graphgen.grid_paths(side, 0.0, npaths, plen, seed)
    pi = graphgen.path_permutation(npaths, plen, seed).astype(np.int64) + side * side
    lab = oracle.cc_uf(n, e)
    assert (lab[: side * side] == 0).all()          # full grid is connected
    for j in range(npaths):
        ids = pi[j * plen:(j + 1) * plen]
        assert (lab[ids] == ids.min()).all()
    assert len(np.unique(lab)) == 1 + npaths


def test_grid_row_cut_closed_form():
    """A side x side grid whose vertical edges between rows 9 and 10 are all
    removed splits into two components labelled 0 and 10*side."""
    side = 20
    ids = np.arange(side * side).reshape(side, side)
    h = np.stack([ids[:, :-1].ravel(), ids[:, 1:].ravel()], 1)
    v = np.stack([ids[:-1, :].ravel(), ids[1:, :].ravel()], 1)
    keep = ids[:-1, :].ravel() // side != 9
    e = np.concatenate([h, v[keep]]).astype(np.uint32)
    lab = oracle.cc_uf(side * side, e)
    assert (lab[: 10 * side] == 0).all() and (lab[10 * side:] == 10 * side).all()


@pytest.mark.parametrize("name", ["cc_two_triangles.txt", "cc_reversed_path.txt",
                                  "cc_multigraph.txt", "cc_star_high_center.txt", "cc_empty.txt"])
def test_golden_fixtures(name):
    n, edges, labels = read_cc_golden(name)
    e = np.array(edges, np.uint32).reshape(-1, 2)
    assert oracle.cc_uf(n, e).tolist() == labels
    assert oracle.cc_bfs(n, e).tolist() == labels


def test_out_of_range_endpoint_rejected():
    with pytest.raises(ValueError):
        oracle.cc_uf(3, np.array([[0, 3]], np.uint32))
    with pytest.raises(ValueError):
        oracle.cc_bfs(3, np.array([[5, 1]], np.uint32))


def test_labels_are_min_id_invariant():
    n = 5000
    e = graphgen.er(n, 3000, 9)
    lab = oracle.cc_uf(n, e)
    assert (lab <= np.arange(n)).all()
    assert (lab[lab] == lab).all()                   # a label is its own label
    for u, v in e:
        assert lab[u] == lab[v]


# ---------------------------------------------------- spanning-forest checker


def _bfs_tree_ids(n, e):
    adj = [[] for _ in range(n)]
    for i, (u, v) in enumerate(e.tolist()):
        adj[u].append((v, i))
        adj[v].append((u, i))
    seen = [False] * n
    ids = []
    for s in range(n):
        if seen[s]:
            continue
        seen[s] = True
        stack = [s]
        while stack:
            x = stack.pop()
            for y, i in adj[x]:
                if not seen[y]:
                    seen[y] = True
                    ids.append(i)
                    stack.append(y)
    return np.array(ids, np.uint64)


def test_sf_checker_accepts_valid_forests():
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = int(rng.integers(1, 60))
        e = rng.integers(0, n, size=(int(rng.integers(0, 2 * n)), 2)).astype(np.uint32)
        ref = oracle.cc_uf(n, e)
        assert oracle.sf_check(n, e, oracle.kruskal_forest(n, e), ref) == 0
        assert oracle.sf_check(n, e, _bfs_tree_ids(n, e), ref) == 0


def test_sf_checker_rejects_planted_mistakes():
    n = 30
    e = graphgen.er(n, 60, 17)
    ref = oracle.cc_uf(n, e)
    good = oracle.kruskal_forest(n, e)
    assert oracle.sf_check(n, e, good, ref) == 0
    # an edge id outside the input
    assert oracle.sf_check(n, e, np.append(good[:-1], 60), ref) == 1
    # the same edge twice
    assert oracle.sf_check(n, e, np.append(good[:-1], good[0]), ref) == 2
    # a dropped edge: one component too many
    assert oracle.sf_check(n, e, good[:-1], ref) in (5, 6)
    # an extra non-tree edge closes a cycle
    extra = [i for i in range(60) if i not in set(good.tolist()) and e[i, 0] != e[i, 1]][0]
    assert oracle.sf_check(n, e, np.append(good, extra), ref) in (4, 5)
    # a self-loop edge
    e2 = e.copy()
    e2[good[0]] = [3, 3]
    assert oracle.sf_check(n, e2, good, oracle.cc_uf(n, e)) == 3
    # a forest of another graph: right count, wrong partition
    other = graphgen.er(n, 60, 18)
    ref_o = oracle.cc_uf(n, other)
    if len(np.unique(ref_o)) == len(np.unique(ref)) and not (ref_o == ref).all():
        assert oracle.sf_check(n, other, oracle.kruskal_forest(n, other), ref) == 6


def test_sf_arc_checker():
    n = 200
    e = graphgen.er(n, 150, 21)
    off, cols = graphgen.csr(n, e)
    ref = oracle.cc_uf(n, e)
    # build a forest of arcs by Kruskal over arcs in row order
    arcs_u = np.repeat(np.arange(n), np.diff(off).astype(np.int64)).astype(np.uint32)
    arc_edges = np.stack([arcs_u, cols], 1)
    ids = oracle.kruskal_forest(n, arc_edges)
    assert oracle.sf_check_arcs(n, off, cols, ids, ref) == 0
    # both arcs of one undirected edge form a 2-cycle
    a = int(ids[0])
    u, v = int(arcs_u[a]), int(cols[a])
    rev = [b for b in range(int(off[v]), int(off[v + 1])) if cols[b] == u][0]
    assert oracle.sf_check_arcs(n, off, cols, np.append(ids, rev), ref) in (4, 5)
    assert oracle.sf_check_arcs(n, off, cols, np.append(ids[:-1], off[-1]), ref) == 1


# ------------------------------------------------------ incremental replay


def test_incremental_golden_stream():
    n, ops, labels = read_inc_golden("inc_stream.txt")
    inc = oracle.Incremental(n)
    for op in ops:
        if op[0] == "insert":
            inc.insert(np.array([[op[1], op[2]]], np.uint32))
        else:
            assert int(inc.query(np.array([[op[1], op[2]]], np.uint32))[0]) == op[3], op
    assert inc.labels().tolist() == labels


def test_incremental_matches_static_and_brute_force():
    rng = np.random.default_rng(77)
    n = 40
    inc = oracle.Incremental(n)
    inserted = np.zeros((0, 2), np.uint32)
    prev = None
    for _ in range(12):
        b = rng.integers(0, n, size=(int(rng.integers(0, 6)), 2)).astype(np.uint32)
        inc.insert(b)
        inserted = np.concatenate([inserted, b])
        q = rng.integers(0, n, size=(30, 2)).astype(np.uint32)
        ans = inc.query(q)
        ref = closure_labels(n, inserted.tolist())
        assert (ans == (ref[q[:, 0]] == ref[q[:, 1]])).all()
        if prev is not None:   # monotone: connected pairs stay connected
            pq, pa = prev
            assert (inc.query(pq) >= pa).all()
        prev = (q, ans)
    assert (inc.labels() == oracle.cc_uf(n, inserted)).all()


def test_batched_oracle_is_per_graph():
    vo, eo, e = graphgen.batched(6, 3, nmin=16, nmax=200)
    lab = oracle.batched_cc(vo, eo, e)
    for g in range(6):
        n = int(vo[g + 1] - vo[g])
        sub = e[int(eo[g]):int(eo[g + 1])]
        assert (lab[int(vo[g]):int(vo[g + 1])] == closure_labels(n, sub.tolist())).all()


# ------------------------------------------- planted mistakes must be caught
# Each mutant is a plausible bug in an implementation of the definition; the
# pins above (brute force on small graphs, closed forms) must reject it.


def _mutant_drop_last_edge(n, e):
    return oracle.cc_uf(n, e[:-1]) if len(e) else oracle.cc_uf(n, e)


def _mutant_root_not_min(n, e):
    """Union-find that links the smaller root under the larger one and returns
    roots without canonicalising."""
    p = list(range(n))

    def f(x):
        while p[x] != x:
            x = p[x]
        return x
    for u, v in e.tolist():
        a, b = f(u), f(v)
        if a != b:
            p[min(a, b)] = max(a, b)
    return np.array([f(v) for v in range(n)], np.uint32)


def _mutant_one_direction(n, e):
    """Traversal that follows edges only from their first endpoint."""
    adj = [[] for _ in range(n)]
    for u, v in e.tolist():
        adj[u].append(v)
    lab = [None] * n
    for s in range(n):
        if lab[s] is None:
            lab[s] = s
            st = [s]
            while st:
                x = st.pop()
                for y in adj[x]:
                    if lab[y] is None:
                        lab[y] = s
                        st.append(y)
    return np.array(lab, np.uint32)


@pytest.mark.parametrize("mutant", [_mutant_drop_last_edge, _mutant_root_not_min, _mutant_one_direction])
def test_pins_catch_planted_mistakes(mutant):
    caught = False
    for mask in range(1 << len(PAIRS5)):
        edges = [PAIRS5[i] for i in range(len(PAIRS5)) if mask >> i & 1]
        e = np.array(edges, dtype=np.uint32).reshape(-1, 2)
        if not (mutant(5, e) == closure_labels(5, edges)).all():
            caught = True
            break
    assert caught
