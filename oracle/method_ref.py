"""Sequential restatement of the paper's per-step rules (TEST INFRASTRUCTURE ONLY).

Each function follows one algorithm of the paper, in its order and notation,
executed by a single thread: a compare-and-swap always sees the value it just
read, so these functions pin the *readings* of the rules (what each step
computes and that the two-phase method reaches the right labels), not the
concurrent behaviour.  They are for small inputs (pure Python loops).

The arrays are Python lists: ``P`` is the parent/label array, ``H`` the hooks
array of Union-Hooks, ``W`` the (rank, parent) words of Union-JTB.
Edge lists are lists of (u, v) pairs; CSR is (offsets, cols) with sorted rows.
"""
from __future__ import annotations

import random
from collections import Counter, deque

INF = 0xFFFFFFFF


def cas(arr, i, old, new) -> bool:
    """Compare-and-swap (Section 2, "Compare-and-Swap")."""
    if arr[i] == old:
        arr[i] = new
        return True
    return False


# ---------------------------------------------------------------- find rules
# Algorithm 5 ("Find Algorithms").

def find_naive(u, P):
    v = u
    while v != P[v]:
        v = P[v]
    return v


def find_compress(u, P):
    r = u
    if P[r] == r:
        return r
    while r != P[r]:
        r = P[r]
    # second pass: every vertex on the path whose parent is above r points at r
    while True:
        j = P[u]
        if not j > r:
            break
        P[u] = r
        u = j
    return r


def find_split(u, P):
    while True:
        v = P[u]
        w = P[v]
        if v == w:
            return v
        cas(P, u, v, w)
        u = v


def find_halve(u, P):
    while True:
        v = P[u]
        w = P[v]
        if v == w:
            return v
        cas(P, u, v, w)
        u = P[u]


FINDS = {"naive": find_naive, "compress": find_compress, "split": find_split, "halve": find_halve}


# --------------------------------------------------------------- splice rules
# Algorithm 6 ("Splice Algorithms"); the argument named u in the listing is
# the current vertex r_u of Rem's loop.

def split_atomic_one(ru, rv, P):
    v = P[ru]
    w = P[v]
    if v != w:
        cas(P, ru, v, w)
    return v


def halve_atomic_one(ru, rv, P):
    v = P[ru]
    w = P[v]
    if v != w:
        cas(P, ru, v, w)
    return w


def splice_atomic(ru, rv, P):
    pu = P[ru]
    cas(P, ru, pu, P[rv])
    return pu


SPLICES = {"split_one": split_atomic_one, "halve_one": halve_atomic_one, "splice": splice_atomic}


# ---------------------------------------------------------------- union rules
# Each returns the vertex that stopped being a root (the spanning-forest slot
# of Section 3.2), or None when u and v were already connected.

def union_async(u, v, P, find):
    """Algorithm 7: find both roots; CAS the larger root onto the smaller."""
    pu, pv = find(u, P), find(v, P)
    while pu != pv:
        if pu < pv:
            pu, pv = pv, pu
        if pu == P[pu] and cas(P, pu, pu, pv):
            return pu
        pu, pv = find(u, P), find(v, P)
    return None


def union_hooks(u, v, P, H, find):
    """Algorithm 8: claim the larger root through H, then write P uncontended."""
    pu, pv = find(u, P), find(v, P)
    while pu != pv:
        if pu < pv:
            pu, pv = pv, pu
        if pu == P[pu] and cas(H, pu, INF, pv):
            P[pu] = pv
            return pu
        pu, pv = find(u, P), find(v, P)
    return None


def union_early(u, v, P, find):
    """Algorithm 9: climb both paths together, hook as soon as one is a root."""
    pu, pv = u, v
    linked = None
    while pu != pv:
        if pu < pv:
            pu, pv = pv, pu
        if pu == P[pu] and cas(P, pu, pu, pv):
            linked = pu
            break
        z = P[pu]
        w = P[z]
        cas(P, pu, z, w)
        pu = w
    if find is not find_naive:
        find(u, P)
        find(v, P)
    return linked


def union_rem_cas(u, v, P, compress, splice):
    """Algorithm 11: Rem's algorithm with a CAS link and a splice step."""
    ru, rv = u, v
    while P[ru] != P[rv]:
        if P[ru] < P[rv]:
            ru, rv = rv, ru
        if ru == P[ru] and cas(P, ru, ru, P[rv]):
            if compress is not find_naive:
                compress(u, P)
                compress(v, P)
            return ru
        ru = splice(ru, rv, P)
    return None


def union_rem_lock(u, v, P, compress, splice, locks):
    """Algorithm 10 (Rem's algorithm with a lock per root).  Reading: after
    the lock is taken, r_u is linked only if it is still a root above P[r_v];
    otherwise the loop continues (one thread: the lock is always free)."""
    ru, rv = u, v
    while P[ru] != P[rv]:
        if P[ru] < P[rv]:
            ru, rv = rv, ru
        if ru == P[ru]:
            locks[ru] = 1
            pv = P[rv]
            linked = ru == P[ru] and ru > pv
            if linked:
                P[ru] = pv
            locks[ru] = 0
            if linked:
                if compress is not find_naive:
                    compress(u, P)
                    compress(v, P)
                return ru
        else:
            ru = splice(ru, rv, P)
    return None


def union_afforest(u, v, P):
    """The finish rule of Afforest (Sutton, Ben-Nun, Bar-Noy 2018): compare the
    parents, hook the higher one onto the lower when it is a root, otherwise
    climb the higher side by two levels and the lower by one."""
    p1, p2 = P[u], P[v]
    while p1 != p2:
        high, low = max(p1, p2), min(p1, p2)
        ph = P[high]
        if ph == low:
            return None
        if ph == high and cas(P, high, high, low):
            return high
        p1, p2 = P[P[high]], P[low]
    return None


def label_propagation(n, edges, labels=None):
    """Label Propagation (Section 3.4): every round the larger label of each
    edge takes the smaller one, until a round changes nothing."""
    lab = list(range(n)) if labels is None else list(labels)
    rounds = 0
    changed = True
    while changed:
        changed = False
        rounds += 1
        for (u, v) in edges:
            lo = min(lab[u], lab[v])
            if lab[u] > lo:
                lab[u] = lo
                changed = True
            if lab[v] > lo:
                lab[v] = lo
                changed = True
    return lab, rounds


def stergiou(n, edges, labels=None):
    """Stergiou's algorithm as described in Section 3.4: like a Liu-Tarjan
    ParentConnect round but with two label arrays -- messages are computed
    from the previous round's array and applied to the current one -- then
    one shortcut; until a round changes nothing."""
    prev = list(range(n)) if labels is None else list(labels)
    rounds = 0
    while True:
        rounds += 1
        cur = list(prev)
        for (u, v) in edges:
            pu, pv = prev[u], prev[v]
            if pv < cur[pu]:
                cur[pu] = pv
            if pu < cur[pv]:
                cur[pv] = pu
        cur = [cur[cur[x]] for x in range(n)]
        if cur == prev:
            break
        prev = cur
    full_shortcut(prev)
    return prev, rounds


def jtb_priority(v, seed):
    """Random priority of a vertex for Union-JTB tie-breaking (SplitMix64 finaliser)."""
    z = (seed * 0x9E3779B97F4A7C15 + v + 1) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return (z ^ (z >> 31)) >> 32


def jtb_find(u, W, two_try):
    """FindSimple or FindTwoTrySplit over (rank, parent) words."""
    while True:
        rk, v = W[u]
        if v == u:
            return u
        w = W[v][1]
        if w == v:
            return v
        if two_try:
            for _ in range(2):
                if W[u][1] == v:
                    W[u] = (W[u][0], w)
                    break
        u = v


def union_jtb(u, v, W, seed, two_try):
    """Union-JTB reading: randomized linking by rank (ties by a random
    priority, then id) with (rank, parent) updated as one word."""
    ru, rv = jtb_find(u, W, two_try), jtb_find(v, W, two_try)
    while ru != rv:
        ku = (W[ru][0], jtb_priority(ru, seed), ru)
        kv = (W[rv][0], jtb_priority(rv, seed), rv)
        if ku > kv:
            ru, rv = rv, ru
            ku, kv = kv, ku
        if W[ru] == (ku[0], ru) and W[rv][1] == rv:
            W[ru] = (ku[0], rv)
            if ku[0] == kv[0]:
                W[rv] = (kv[0] + 1, rv)
            return ru
        ru, rv = jtb_find(ru, W, two_try), jtb_find(rv, W, two_try)
    return None


# ------------------------------------------------------------- whole-array ops

def full_shortcut(P):
    """FullShortcut: P[v] <- P[P[v]] for all v until nothing changes."""
    changed = True
    while changed:
        changed = False
        for v in range(len(P)):
            if P[v] != P[P[v]]:
                P[v] = P[P[v]]
                changed = True


def most_frequent_label(P):
    """GetMostFrequentLabel (Algorithm 1): exact mode, ties to the smaller label."""
    if not P:
        return None
    cnt = Counter(P)
    best = max(cnt.values())
    return min(l for l, c in cnt.items() if c == best)


# ------------------------------------------------------------------ sampling
# Each sampler returns the spanning-forest edges it used as CSR arc positions.

class UF:
    """Union-find configuration for the sampling and finish phases."""

    def __init__(self, n, link="async", find="naive", splice="splice", seed=1):
        self.link, self.seed = link, seed
        self.find = FINDS.get(find, find_naive)
        self.splice = SPLICES.get(splice, splice_atomic)
        self.P = list(range(n))
        self.H = [INF] * n
        self.W = [(0, v) for v in range(n)] if link == "jtb" else None
        self.two_try = find == "twotrysplit"
        self.locks = [0] * n

    def union(self, u, v):
        if self.link == "remlock":
            return union_rem_lock(u, v, self.P, self.find, self.splice, self.locks)
        if self.link == "afforest":
            return union_afforest(u, v, self.P)
        if self.link == "eclcc":
            return union_async(u, v, self.P, find_split)
        if self.link == "async":
            return union_async(u, v, self.P, self.find)
        if self.link == "hooks":
            return union_hooks(u, v, self.P, self.H, self.find)
        if self.link == "early":
            return union_early(u, v, self.P, self.find)
        if self.link == "remcas":
            return union_rem_cas(u, v, self.P, self.find, self.splice)
        if self.link == "jtb":
            return union_jtb(u, v, self.W, self.seed, self.two_try)
        raise ValueError(self.link)

    def root(self, v):
        if self.W is not None:
            return jtb_find(v, self.W, False)
        return find_naive(v, self.P)

    def labels(self):
        """LabelFinalization, then min-id canonicalisation for JTB roots."""
        n = len(self.P)
        roots = [self.root(v) for v in range(n)]
        if self.W is None:
            return roots
        minid = {}
        for v in range(n):
            minid.setdefault(roots[v], v)
        return [minid[r] for r in roots]

    def compress_all(self):
        if self.W is not None:
            for v in range(len(self.W)):
                self.W[v] = (self.W[v][0], jtb_find(v, self.W, False))
        else:
            full_shortcut(self.P)


def kout_sample(off, cols, uf, k=2):
    """Algorithm 2 (k-out), reading: the first k edges of every vertex."""
    sf = []
    n = len(off) - 1
    for v in range(n):
        for j in range(min(k, off[v + 1] - off[v])):
            a = off[v] + j
            if uf.union(v, cols[a]) is not None:
                sf.append(a)
    uf.compress_all()
    return sf


def hb_sample(off, cols, uf, N=4):
    """Algorithm 3 (HB).  Step 1: labels[v] = min(v, w) for the smallest
    neighbour w (no contention).  Step 2: vertices that are still roots
    (labels[v] == v, the reading of the prose) union their first N edges.
    Then full compression.  For Union-JTB the step-1 trees are first flattened
    and their roots given rank 1, so every parent outranks its children."""
    n = len(off) - 1
    sf = []
    P = uf.P
    for v in range(n):
        if off[v + 1] > off[v]:
            w = cols[off[v]]
            if w < v:
                P[v] = w
                sf.append(off[v])
    roots = [v for v in range(n) if P[v] == v]
    if uf.W is not None:
        full_shortcut(P)
        for v in range(n):
            uf.W[v] = (1 if P[v] == v else 0, P[v])
    for v in roots:
        for j in range(min(N, off[v + 1] - off[v])):
            a = off[v] + j
            if uf.union(v, cols[a]) is not None:
                sf.append(a)
    uf.compress_all()
    return sf


def bfs_sample(off, cols, uf, n_samples=1024, seed=1):
    """Algorithm 4 (BFS): source = max degree over a seeded sample (ties to the
    smaller id); label the reached set; relabel it to its minimum id so that
    parents never exceed their vertex."""
    n = len(off) - 1
    if n == 0:
        return []
    rng = random.Random(seed)
    sample = [rng.randrange(n) for _ in range(min(n_samples, n))]
    s = min(sample, key=lambda x: (-(off[x + 1] - off[x]), x))
    seen = {s: None}
    q = deque([s])
    while q:
        x = q.popleft()
        for a in range(off[x], off[x + 1]):
            y = cols[a]
            if y not in seen:
                seen[y] = a
                q.append(y)
    r = min(seen)
    sf = [a for y, a in seen.items() if a is not None]
    for v in seen:
        if uf.W is not None:
            uf.W[v] = (1 if v == r else 0, r)
        else:
            uf.P[v] = r
    return sf


# -------------------------------------------------------------- finish phase

def finish_csr(off, cols, uf, lmax, skip=True):
    """Union-find meta-algorithm: every vertex whose label is not L_max unions
    all of its edges (the two-phase skip rule of Section 3.1)."""
    n = len(off) - 1
    lab0 = [uf.root(v) for v in range(n)]
    sf = []
    for u in range(n):
        if skip and lab0[u] == lmax:
            continue
        for a in range(off[u], off[u + 1]):
            if uf.union(u, cols[a]) is not None:
                sf.append(a)
    return sf


def finish_coo(edges, uf, order=None):
    sf = []
    idx = range(len(edges)) if order is None else order
    for i in idx:
        u, v = edges[i]
        if uf.union(u, v) is not None:
            sf.append(i)
    return sf


def static_conn_csr(off, cols, sample="kout", link="async", find="naive", splice="splice",
                    k=2, N=4, seed=1):
    """Algorithm 1 over CSR: InitLabel, SamplePhase, GetMostFrequentLabel,
    FinishPhase, LabelFinalization.  Returns (labels, forest arcs)."""
    n = len(off) - 1
    uf = UF(n, link, find, splice, seed)
    sf = []
    if sample == "kout":
        sf += kout_sample(off, cols, uf, k)
    elif sample == "hb":
        sf += hb_sample(off, cols, uf, N)
    elif sample == "bfs":
        sf += bfs_sample(off, cols, uf, seed=seed)
    lmax = most_frequent_label([uf.root(v) for v in range(n)]) if sample != "none" else None
    sf += finish_csr(off, cols, uf, lmax, skip=sample != "none")
    return uf.labels(), sf


# ------------------------------------------------------ Shiloach-Vishkin rounds

def shiloach_vishkin(n, edges, labels=None, frequent=None):
    """Algorithm 12 (root-based SV): writeMin of the smaller label onto the
    larger one when that one was a root at the start of the round, then full
    shortcut, until a round changes nothing.  Returns (labels, rounds)."""
    lab = list(range(n)) if labels is None else list(labels)
    cand = [e for e in edges if frequent is None or not (lab[e[0]] == frequent and lab[e[1]] == frequent)]
    prev = list(lab)
    rounds = 0
    changed = True
    while changed:
        changed = False
        rounds += 1
        for (u, v) in cand:
            pu, pv = lab[u], lab[v]
            lo, hi = min(pu, pv), max(pu, pv)
            if lo != hi and prev[hi] == hi:
                lab[hi] = min(lab[hi], lo)
                changed = True
        full_shortcut(lab)
        prev = list(lab)
    return lab, rounds


# ----------------------------------------------------------- Liu-Tarjan rounds
# Variant names follow the appendix list: connect rule C / P / E, update rule
# U (all vertices) / R (roots only), shortcut S (one step) / F (to fixpoint),
# optional A (alter).

LT_VARIANTS = ["CUSA", "CRSA", "PUSA", "PRSA", "PUS", "PRS", "EUSA", "EUS",
               "CUFA", "CRFA", "PUFA", "PRFA", "PUF", "PRF", "EUFA", "EUF"]
LT_ROOT_BASED = ["CRSA", "PRSA", "PRS", "CRFA", "PRFA", "PRF"]


def liu_tarjan(n, edges, variant, labels=None, max_rounds=100000):
    """One Liu-Tarjan variant, synchronous rounds: every message of a round is
    computed from the parents at the start of the round.

    Reading of the connect rules:
      C (Connect)         u receives v and v receives u;
      P (ParentConnect)   P[u] receives P[v] and P[v] receives P[u];
      E (ExtendedConnect) u, v, P[u] and P[v] all receive min(P[u], P[v]).
    Update: P[x] <- min(P[x], smallest message to x); RootUpdate: the same but
    only for x with P[x] == x at the start of the round.  Shortcut: one step
    P[x] <- P[P[x]]; FullShortcut: to the fixpoint.  Alter: every edge (u, v)
    becomes (P[u], P[v]) and is dropped when both are equal.  The loop ends
    after a round that changes neither P nor the edge list.
    Returns (labels, rounds)."""
    conn, upd, sc = variant[0], variant[1], variant[2]
    alter = variant.endswith("A")
    P = list(range(n)) if labels is None else list(labels)
    E = [tuple(e) for e in edges]
    rounds = 0
    while rounds < max_rounds:
        rounds += 1
        msg = [INF] * n

        def send(x, val):
            if val < msg[x]:
                msg[x] = val

        for (u, v) in E:
            if conn == "C":
                send(u, v)
                send(v, u)
            elif conn == "P":
                send(P[u], P[v])
                send(P[v], P[u])
            else:
                lo = min(P[u], P[v])
                for x in (u, v, P[u], P[v]):
                    send(x, lo)
        newP = list(P)
        for x in range(n):
            if upd == "R" and P[x] != x:
                continue
            if msg[x] < newP[x]:
                newP[x] = msg[x]
        if sc == "S":
            newP = [newP[newP[x]] for x in range(n)]
        else:
            full_shortcut(newP)
        changed = newP != P
        P = newP
        if alter:
            E2 = [(P[u], P[v]) for (u, v) in E]
            E2 = [e for e in E2 if e[0] != e[1]]
            changed = changed or E2 != E
            E = E2
        if not changed:
            break
    full_shortcut(P)
    return P, rounds
