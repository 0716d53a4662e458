// uf_device.cuh -- concurrent union-find rules on a uint32 parent array P.
//
// Section 2 fixes the invariant every rule here keeps: a vertex points to
// itself (a root) or to a vertex with a smaller id, so parent chains strictly
// decrease and can never close a cycle.  All rules are root-based: only a
// root is ever re-pointed into another tree (by one CAS), while compression
// only moves a non-root pointer to one of its ancestors.
//
// Memory model: P lives in global memory and is shared by all threads.
// Plain loads go through L2 only (ld.global.cg), so a retry loop always sees
// other threads' CAS results; CAS is atomicCAS (performed at L2).  Every loop
// is bounded by Spin: after `cap` steps the operation gives up and raises
// ERR_NONCONV in the device error word, and every other operation gives up
// soon after seeing that flag.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gc {

enum { LK_ASYNC = 0, LK_HOOKS = 1, LK_EARLY = 2, LK_REMCAS = 3, LK_JTB = 4, LK_REMLOCK = 7, LK_AFFOREST = 9 };
enum { FD_NAIVE = 0, FD_COMPRESS = 1, FD_SPLIT = 2, FD_HALVE = 3, FD_TWOTRY = 4 };
enum { SP_NONE = 0, SP_SPLIT_ONE = 1, SP_HALVE_ONE = 2, SP_SPLICE = 3 };

#define GC_DINF 0xFFFFFFFFu
#define GC_DERR_RANGE 1u
#define GC_DERR_NONCONV 2u
#define GC_DERR_OVERFLOW 4u

typedef unsigned long long u64w;

struct UFState {
    uint32_t* P;      // parents (all min-linking rules)
    uint32_t* H;      // hooks, INF-initialised (Union-Hooks)
    u64w* W;          // (rank << 32) | parent words (Union-JTB)
    uint32_t* sf;     // spanning-forest slot per vertex (edge / arc id), INF = none
    uint32_t* err;    // device error word
    uint32_t* Lk;     // per-vertex locks, 0 = free (Union-Rem-Lock)
    uint32_t n;
    uint32_t cap;     // per-operation loop cap
    uint32_t seed;    // Union-JTB priority seed
};

__device__ __forceinline__ uint32_t ldp(const uint32_t* P, uint32_t i) { return __ldcg(P + i); }
// L1-allowed parent load.  Every P[x] only ever decreases (roots are linked to
// smaller ids, compression moves a pointer to an ancestor, a splice only to a
// smaller parent), so a stale value is an older, larger parent of x in the
// same set: walks through stale values still strictly descend, and every
// decision is validated by a CAS whose returned value (always fresh) is what
// the loops continue from.  Rules that retry by re-loading (Union-Hooks,
// Union-JTB) use the L2-only ldp instead.
template <bool L1>
__device__ __forceinline__ uint32_t ldq(const uint32_t* P, uint32_t i) { return L1 ? __ldca(P + i) : __ldcg(P + i); }
__device__ __forceinline__ void stp(uint32_t* P, uint32_t i, uint32_t v) { __stcg(P + i, v); }
__device__ __forceinline__ u64w ldw(const u64w* W, uint32_t i) { return __ldcg(W + i); }
__device__ __forceinline__ uint32_t wpar(u64w w) { return (uint32_t)w; }
__device__ __forceinline__ uint32_t wrank(u64w w) { return (uint32_t)(w >> 32); }
__device__ __forceinline__ u64w wmake(uint32_t rank, uint32_t par) { return ((u64w)rank << 32) | par; }

struct Spin {
    uint32_t left;
    bool dead;
    bool soft;   // a soft budget gives up quietly (the caller defers the operation)
    // Where an abandoned union must resume (GC_DINF: from its endpoints).  A
    // Rem climb records its current pair: SpliceAtomic may already have moved
    // a non-root subtree into the other tree, so the two endpoints can look
    // joined while the rest of the first set is not yet linked.
    uint32_t at_u, at_v;
    __device__ __forceinline__ explicit Spin(uint32_t cap, bool soft_ = false)
        : left(cap), dead(false), soft(soft_), at_u(GC_DINF), at_v(GC_DINF) {}
    // One loop step; false once the operation must give up.
    __device__ __forceinline__ bool step(const UFState& s) {
        if (dead) return false;
        if (--left == 0) {
            if (!soft) atomicOr(s.err, GC_DERR_NONCONV);
            dead = true;
            return false;
        }
        if ((left & 4095u) == 0 && (__ldcg(s.err) & GC_DERR_NONCONV)) {
            dead = true;
            return false;
        }
        return true;
    }
};

// ------------------------------------------------------------ find rules
// Algorithm 5.  Each returns the root reached (or, after giving up, the last
// vertex visited with sp.dead set).

template <int F, bool L1 = false>
__device__ __forceinline__ uint32_t uf_find(const UFState& s, uint32_t u, Spin& sp) {
    uint32_t* P = s.P;
    if (F == FD_NAIVE) {
        uint32_t v = u;
        while (true) {
            uint32_t p = ldq<L1>(P, v);
            if (p == v) return v;
            v = p;
            if (!sp.step(s)) return v;
        }
    } else if (F == FD_COMPRESS) {
        uint32_t r = u, p = ldq<L1>(P, r);
        if (p == r) return r;
        while (p != r) {
            r = p;
            p = ldq<L1>(P, r);
            if (!sp.step(s)) return r;
        }
        // every vertex on the path whose parent is above the root points at it
        uint32_t x = u;
        while (true) {
            uint32_t j = ldq<L1>(P, x);
            if (!(j > r)) break;
            stp(P, x, r);
            x = j;
            if (!sp.step(s)) break;
        }
        return r;
    } else if (F == FD_SPLIT) {
        while (true) {
            uint32_t v = ldq<L1>(P, u), w = ldq<L1>(P, v);
            if (v == w) return v;
            atomicCAS(P + u, v, w);
            u = v;
            if (!sp.step(s)) return u;
        }
    } else {  // FD_HALVE
        while (true) {
            uint32_t v = ldq<L1>(P, u), w = ldq<L1>(P, v);
            if (v == w) return v;
            uint32_t old = atomicCAS(P + u, v, w);
            u = (old == v) ? w : old;  // the value P[u] holds right after the CAS
            if (!sp.step(s)) return u;
        }
    }
}

// ----------------------------------------------------------- union rules
// Each returns true iff this call re-pointed a root, and then records the
// edge id in that root's spanning-forest slot (Section 3.2).

// Union-Async (Algorithm 7).  The CAS target is P[p_u]: only a root is
// linked, from the larger root id to the smaller.  Retries re-run the find
// from the previous roots, which are ancestors of the endpoints.
template <int F, bool SF>
__device__ __forceinline__ bool union_async(const UFState& s, uint32_t u, uint32_t v, uint32_t eid, Spin& sp) {
    uint32_t pu = uf_find<F, true>(s, u, sp), pv = uf_find<F, true>(s, v, sp);
    while (pu != pv && !sp.dead) {
        if (pu < pv) { uint32_t t = pu; pu = pv; pv = t; }
        uint32_t p = ldq<true>(s.P, pu);
        if (p == pu) {
            p = atomicCAS(s.P + pu, pu, pv);
            if (p == pu) {
                if (SF) s.sf[pu] = eid;
                return true;
            }
        }
        if (!sp.step(s)) break;
        pu = uf_find<F, true>(s, p, sp);     // p is a (possibly older) parent of pu: strictly smaller
        pv = uf_find<F, true>(s, pv, sp);
    }
    return false;
}

// Union-Hooks (Algorithm 8): the CAS claims H[p_u]; the winner then writes
// P[p_u] with an uncontended store followed by a memory fence.
template <int F, bool SF>
__device__ __forceinline__ bool union_hooks(const UFState& s, uint32_t u, uint32_t v, uint32_t eid, Spin& sp) {
    uint32_t pu = uf_find<F>(s, u, sp), pv = uf_find<F>(s, v, sp);
    while (pu != pv && !sp.dead) {
        if (pu < pv) { uint32_t t = pu; pu = pv; pv = t; }
        if (ldp(s.P, pu) == pu && atomicCAS(s.H + pu, GC_DINF, pv) == GC_DINF) {
            stp(s.P, pu, pv);
            __threadfence();
            if (SF) s.sf[pu] = eid;
            return true;
        }
        if (!sp.step(s)) break;
        pu = uf_find<F>(s, pu, sp);
        pv = uf_find<F>(s, pv, sp);
    }
    return false;
}

// Union-Early (Algorithm 9): climb both paths together with a halving step
// and hook the larger side as soon as it is a root.  Hooking a root p_u under
// any p_v < p_u is safe: every member of p_u's tree has an id >= p_u.
template <int F, bool SF>
__device__ __forceinline__ bool union_early(const UFState& s, uint32_t u, uint32_t v, uint32_t eid, Spin& sp) {
    uint32_t pu = u, pv = v;
    bool linked = false;
    while (pu != pv) {
        if (pu < pv) { uint32_t t = pu; pu = pv; pv = t; }
        uint32_t z = ldq<true>(s.P, pu);
        if (z == pu) {
            uint32_t old = atomicCAS(s.P + pu, pu, pv);
            if (old == pu) {
                if (SF) s.sf[pu] = eid;
                linked = true;
                break;
            }
            z = old;
        }
        uint32_t w = ldq<true>(s.P, z);
        if (w != z) atomicCAS(s.P + pu, z, w);
        pu = w;
        if (!sp.step(s)) break;
    }
    if (F != FD_NAIVE && !sp.dead) {
        uf_find<F, true>(s, u, sp);
        uf_find<F, true>(s, v, sp);
    }
    return linked;
}

// Union-Rem-CAS (Algorithm 11) with the splice step of Algorithm 6 applied to
// the current r_u.  The loop carries the parent values it has loaded instead
// of re-reading them: P[r_u] after a step is the value the step just read (or
// the CAS returned).  Carried values may be older than memory; every P[x]
// only decreases and sets only merge while unions run, so "equal parents"
// still means "same set", and a link happens only through a CAS that checks
// r_u is still a root.
template <int F, int S, bool SF>
__device__ __forceinline__ bool union_remcas(const UFState& s, uint32_t u, uint32_t v, uint32_t eid, Spin& sp) {
    uint32_t* P = s.P;
    uint32_t ru = u, rv = v;
    uint32_t pu = ldq<true>(P, ru), pv = ldq<true>(P, rv);
    while (true) {
        if (pu == pv) return false;
        if (pu < pv) {
            uint32_t t = ru; ru = rv; rv = t;
            t = pu; pu = pv; pv = t;
        }
        if (ru == pu) {
            uint32_t old = atomicCAS(P + ru, ru, pv);
            if (old == ru) {
                if (SF) s.sf[ru] = eid;
                if (F != FD_NAIVE) {
                    uf_find<F, true>(s, u, sp);
                    uf_find<F, true>(s, v, sp);
                }
                return true;
            }
            pu = old;                       // r_u was linked meanwhile: its fresh parent
        } else if (S == SP_SPLICE) {        // P[r_u] <- P[r_v], continue from the old parent
            atomicCAS(P + ru, pu, pv);
            ru = pu;
            pu = ldq<true>(P, ru);
        } else {                            // one split (return the parent) or halve (grandparent)
            uint32_t w = ldq<true>(P, pu);
            if (w != pu) atomicCAS(P + ru, pu, w);
            if (S == SP_SPLIT_ONE) {
                ru = pu;
                pu = w;
            } else {
                ru = w;
                pu = ldq<true>(P, w);
            }
        }
        if (!sp.step(s)) {
            sp.at_u = ru;
            sp.at_v = rv;
            return false;
        }
    }
}

// Union-Rem-Lock (Algorithm 10): Rem's climb, but a root is linked under a
// lock on it (a plain store while holding the lock) instead of by CAS.  A
// thread holds at most one lock and never waits for another lock while
// holding it, so lock waits always end; each wait is one bounded Spin step.
// After taking the lock, r_u is linked only if it is still a root above the
// current P[r_v]; otherwise the climb continues from the fresh values.
template <int F, int S, bool SF>
__device__ __forceinline__ bool union_remlock(const UFState& s, uint32_t u, uint32_t v, uint32_t eid, Spin& sp) {
    uint32_t* P = s.P;
    uint32_t ru = u, rv = v;
    uint32_t pu = ldq<true>(P, ru), pv = ldq<true>(P, rv);
    while (true) {
        if (pu == pv) return false;
        if (pu < pv) {
            uint32_t t = ru; ru = rv; rv = t;
            t = pu; pu = pv; pv = t;
        }
        if (ru == pu) {
            if (atomicCAS(s.Lk + ru, 0u, 1u) == 0u) {
                uint32_t cur = ldp(P, ru), pvf = ldp(P, rv);
                bool linked = cur == ru && ru > pvf;
                if (linked) {
                    stp(P, ru, pvf);
                    if (SF) s.sf[ru] = eid;
                }
                __threadfence();
                atomicExch(s.Lk + ru, 0u);
                if (linked) {
                    if (F != FD_NAIVE) {
                        uf_find<F, true>(s, u, sp);
                        uf_find<F, true>(s, v, sp);
                    }
                    return true;
                }
                pu = cur;
                pv = pvf;
            } else {                        // lock held by another thread: re-read
                pu = ldp(P, ru);
                pv = ldp(P, rv);
            }
        } else if (S == SP_SPLICE) {
            atomicCAS(P + ru, pu, pv);
            ru = pu;
            pu = ldq<true>(P, ru);
        } else {
            uint32_t w = ldq<true>(P, pu);
            if (w != pu) atomicCAS(P + ru, pu, w);
            if (S == SP_SPLIT_ONE) {
                ru = pu;
                pu = w;
            } else {
                ru = w;
                pu = ldq<true>(P, w);
            }
        }
        if (!sp.step(s)) {
            sp.at_u = ru;
            sp.at_v = rv;
            return false;
        }
    }
}

// The finish rule of Afforest (Sutton, Ben-Nun, Bar-Noy, IPDPS 2018):
// compare the two parents; if the higher one's parent is the lower one they
// are joined; if the higher one is a root, CAS it onto the lower one; else
// climb the higher side two levels and the lower side one.
template <bool SF>
__device__ __forceinline__ bool union_afforest(const UFState& s, uint32_t u, uint32_t v, uint32_t eid, Spin& sp) {
    uint32_t* P = s.P;
    uint32_t p1 = ldq<true>(P, u), p2 = ldq<true>(P, v);
    while (p1 != p2) {
        uint32_t high = p1 > p2 ? p1 : p2, low = p1 > p2 ? p2 : p1;
        uint32_t ph = ldq<true>(P, high);
        if (ph == low) return false;
        if (ph == high) {
            uint32_t old = atomicCAS(P + high, high, low);
            if (old == high) {
                if (SF) s.sf[high] = eid;
                return true;
            }
            ph = old;
        }
        p1 = ldq<true>(P, ph);
        p2 = ldq<true>(P, low);
        if (!sp.step(s)) return false;
    }
    return false;
}

// ----------------------------------------------------------- Union-JTB
// Randomized linking by rank on 64-bit (rank, parent) words: the root with
// the smaller key (rank, priority, id) is linked under the other; on equal
// ranks the new parent's rank is raised by a second CAS.  Keys strictly
// increase along every parent pointer, so no cycle can form.

__device__ __forceinline__ uint32_t jtb_priority(uint32_t seed, uint32_t v) {
    unsigned long long z = (unsigned long long)seed * 0x9E3779B97F4A7C15ull + v + 1;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (uint32_t)((z ^ (z >> 31)) >> 32);
}

template <int F>
__device__ __forceinline__ uint32_t jtb_find(const UFState& s, uint32_t u, Spin& sp) {
    u64w* W = s.W;
    if constexpr (F != FD_TWOTRY) {  // FindSimple
        while (true) {
            uint32_t p = wpar(ldw(W, u));
            if (p == u) return u;
            u = p;
            if (!sp.step(s)) return u;
        }
    } else {
        while (true) {  // FindTwoTrySplit: up to two split attempts per step
            u64w wu = ldw(W, u);
            uint32_t v = wpar(wu);
            if (v == u) return u;
            uint32_t w = wpar(ldw(W, v));
            if (w == v) return v;
            for (int t = 0; t < 2; ++t) {
                u64w old = atomicCAS(W + u, wu, wmake(wrank(wu), w));
                if (old == wu) break;
                wu = old;
                v = wpar(wu);
                w = wpar(ldw(W, v));
                if (w == v) break;
            }
            u = v;
            if (!sp.step(s)) return u;
        }
    }
}

template <int F, bool SF>
__device__ __forceinline__ bool union_jtb(const UFState& s, uint32_t u, uint32_t v, uint32_t eid, Spin& sp) {
    uint32_t ru = jtb_find<F>(s, u, sp), rv = jtb_find<F>(s, v, sp);
    while (ru != rv && !sp.dead) {
        u64w wu = ldw(s.W, ru), wv = ldw(s.W, rv);
        if (wpar(wu) != ru || wpar(wv) != rv) {
            if (!sp.step(s)) break;
            ru = jtb_find<F>(s, ru, sp);
            rv = jtb_find<F>(s, rv, sp);
            continue;
        }
        uint32_t ku = wrank(wu), kv = wrank(wv);
        bool u_low;
        if (ku != kv) {
            u_low = ku < kv;
        } else {
            uint32_t qu = jtb_priority(s.seed, ru), qv = jtb_priority(s.seed, rv);
            u_low = (qu != qv) ? (qu < qv) : (ru < rv);
        }
        if (!u_low) {
            uint32_t t = ru; ru = rv; rv = t;
            u64w tw = wu; wu = wv; wv = tw;
            t = ku; ku = kv; kv = t;
        }
        if (atomicCAS(s.W + ru, wu, wmake(ku, rv)) == wu) {
            if (ku == kv) atomicCAS(s.W + rv, wv, wmake(kv + 1, rv));
            if (SF) s.sf[ru] = eid;
            return true;
        }
        if (!sp.step(s)) break;
        ru = jtb_find<F>(s, ru, sp);
        rv = jtb_find<F>(s, rv, sp);
    }
    return false;
}

// ----------------------------------------------------------- same set
// Connectivity query that stays exact while unions run concurrently.  Two
// roots found at different times may differ although the sets have merged in
// between, so "different" is answered only after both are confirmed to still
// be roots by fresh (L2) reads: a non-root never becomes a root again, so at
// that instant the two vertices are in different sets.  Otherwise the walk
// continues from the fresh parent.
template <int L, int F>
__device__ __forceinline__ bool same_set(const UFState& s, uint32_t x, uint32_t y, Spin& sp) {
    if (L == LK_JTB) {
        uint32_t a = jtb_find<F>(s, x, sp), b = jtb_find<F>(s, y, sp);
        while (!sp.dead) {
            if (a == b) return true;
            uint32_t pa = wpar(ldw(s.W, a));
            if (pa != a) { a = jtb_find<F>(s, pa, sp); continue; }
            uint32_t pb = wpar(ldw(s.W, b));
            if (pb != b) { b = jtb_find<F>(s, pb, sp); continue; }
            return false;
        }
        return false;
    }
    uint32_t a = uf_find<F, true>(s, x, sp), b = uf_find<F, true>(s, y, sp);
    while (!sp.dead) {
        if (a == b) return true;
        uint32_t pa = ldp(s.P, a);
        if (pa != a) { a = uf_find<F, true>(s, pa, sp); if (!sp.step(s)) break; continue; }
        uint32_t pb = ldp(s.P, b);
        if (pb != b) { b = uf_find<F, true>(s, pb, sp); if (!sp.step(s)) break; continue; }
        return false;
    }
    return false;
}

// Both endpoints' walks in lock step, for queries under the naive find while
// nothing links or compresses the forest (query batches, query segments).
// Every rule but JTB keeps P[v] <= v, so each tree's root is its smallest
// vertex: a walk that reaches a root above the other walk's current vertex
// proves the two sets differ without walking the other path to its end.  One
// dependent load per step pair instead of the two walks one after the other.
__device__ __forceinline__ bool same_root_lockstep(const UFState& s, uint32_t x, uint32_t y, Spin& sp) {
    while (x != y) {
        uint32_t px = ldq<true>(s.P, x), py = ldq<true>(s.P, y);
        bool rx = px == x, ry = py == y;
        if ((rx && (ry || y < x)) || (ry && x < y)) return false;
        x = px;
        y = py;
        if (!sp.step(s)) return false;
    }
    return true;
}

// ----------------------------------------------------------- dispatcher
template <int L, int F, int S, bool SF>
__device__ __forceinline__ bool uf_union(const UFState& s, uint32_t u, uint32_t v, uint32_t eid, Spin& sp) {
    if (L == LK_ASYNC) return union_async<F, SF>(s, u, v, eid, sp);
    if (L == LK_HOOKS) return union_hooks<F, SF>(s, u, v, eid, sp);
    if (L == LK_EARLY) return union_early<F, SF>(s, u, v, eid, sp);
    if (L == LK_REMCAS) return union_remcas<F, S, SF>(s, u, v, eid, sp);
    if (L == LK_REMLOCK) return union_remlock<F, S, SF>(s, u, v, eid, sp);
    if (L == LK_AFFOREST) return union_afforest<SF>(s, u, v, eid, sp);
    return union_jtb<F, SF>(s, u, v, eid, sp);
}

// Root of v with no compression (parent array or JTB words).  A chain has
// at most n vertices; a longer walk means a corrupted forest and raises
// ERR_NONCONV instead of looping.
template <int L, bool L1 = false>
__device__ __forceinline__ uint32_t uf_root(const UFState& s, uint32_t v) {
    for (uint32_t i = 0; i <= s.n; ++i) {
        uint32_t p = (L == LK_JTB) ? wpar(ldw(s.W, v)) : ldq<L1>(s.P, v);
        if (p == v) return v;
        v = p;
    }
    atomicOr(s.err, GC_DERR_NONCONV);
    return v;
}

}  // namespace gc
