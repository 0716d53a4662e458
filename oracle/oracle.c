/*
 * oracle.c -- plain sequential CPU oracle for connected components, spanning
 * forests and incremental connectivity.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code with the GPU library.
 *
 * What it computes is the plain definition of each problem (Section 2, "Graph
 * Connectivity Problems"):
 *   - connected components: labels(u) == labels(v) iff u and v are joined by a
 *     path; the canonical labelling used everywhere is the minimum vertex id
 *     of the component;
 *   - connectivity query: true iff both vertices are in one component;
 *   - spanning forest: one spanning tree per component, made of input edges.
 *
 * Two independent routes to the same labels:
 *   O1  sequential union-find with union by rank and full path compression
 *       (Cormen, Leiserson, Rivest, Stein, Introduction to Algorithms, ch. 21),
 *       then one ascending sweep that maps every root to the smallest id seen;
 *   O2  breadth-first search from every still-unlabelled vertex in increasing
 *       id order, over an adjacency structure built here.
 * Self-loops and duplicate edges are accepted and change nothing.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NONE 0xFFFFFFFFu

/* ---------------- O1: union by rank + path compression ---------------- */

static uint32_t or_find(uint32_t* parent, uint32_t x) {
    uint32_t r = x;
    while (parent[r] != r) r = parent[r];
    while (parent[x] != r) { uint32_t nx = parent[x]; parent[x] = r; x = nx; }
    return r;
}

/* Returns 1 when x and y were in different sets (and are now joined). */
static int or_union(uint32_t* parent, uint8_t* rank, uint32_t x, uint32_t y) {
    uint32_t rx = or_find(parent, x), ry = or_find(parent, y);
    if (rx == ry) return 0;
    if (rank[rx] < rank[ry]) { uint32_t t = rx; rx = ry; ry = t; }
    parent[ry] = rx;
    if (rank[rx] == rank[ry]) rank[rx]++;
    return 1;
}

/* Canonical min-id labels from a union-find state: the first vertex reached
 * in ascending order for each root is the smallest member of its set. */
static void or_canonical(uint32_t n, uint32_t* parent, uint32_t* labels) {
    uint32_t* minid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    for (uint32_t v = 0; v < n; ++v) minid[v] = OR_NONE;
    for (uint32_t v = 0; v < n; ++v) {
        uint32_t r = or_find(parent, v);
        if (minid[r] == OR_NONE) minid[r] = v;
        labels[v] = minid[r];
    }
    free(minid);
}

/* O1.  Returns 0, or 2 when an endpoint is >= n (labels untouched). */
int oracle_cc_uf(uint32_t n, uint64_t m, const uint32_t* edges, uint32_t* labels) {
    for (uint64_t i = 0; i < m; ++i)
        if (edges[2 * i] >= n || edges[2 * i + 1] >= n) return 2;
    uint32_t* parent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    uint8_t* rank = (uint8_t*)calloc(n ? n : 1, 1);
    for (uint32_t v = 0; v < n; ++v) parent[v] = v;
    for (uint64_t i = 0; i < m; ++i) or_union(parent, rank, edges[2 * i], edges[2 * i + 1]);
    or_canonical(n, parent, labels);
    free(parent); free(rank);
    return 0;
}

/* ---------------- O2: BFS over an adjacency structure ---------------- */

int oracle_cc_bfs(uint32_t n, uint64_t m, const uint32_t* edges, uint32_t* labels) {
    for (uint64_t i = 0; i < m; ++i)
        if (edges[2 * i] >= n || edges[2 * i + 1] >= n) return 2;
    uint64_t* start = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    for (uint64_t i = 0; i < m; ++i) { start[edges[2 * i] + 1]++; start[edges[2 * i + 1] + 1]++; }
    for (uint32_t v = 0; v < n; ++v) start[v + 1] += start[v];
    uint64_t* fill = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    memcpy(fill, start, sizeof(uint64_t) * ((size_t)n + 1));
    uint32_t* adj = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(2 * m + 1));
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t u = edges[2 * i], v = edges[2 * i + 1];
        adj[fill[u]++] = v;
        adj[fill[v]++] = u;
    }
    free(fill);
    uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    for (uint32_t v = 0; v < n; ++v) labels[v] = OR_NONE;
    for (uint32_t s = 0; s < n; ++s) {
        if (labels[s] != OR_NONE) continue;
        /* every vertex of s's component is unlabelled and has id >= s */
        uint32_t head = 0, tail = 0;
        labels[s] = s; queue[tail++] = s;
        while (head < tail) {
            uint32_t x = queue[head++];
            for (uint64_t j = start[x]; j < start[x + 1]; ++j) {
                uint32_t y = adj[j];
                if (labels[y] == OR_NONE) { labels[y] = s; queue[tail++] = y; }
            }
        }
    }
    free(queue); free(adj); free(start);
    return 0;
}

/* ---------------- spanning-forest checker ----------------
 * A spanning forest is not unique, so the oracle checks one instead of
 * producing one.  Given the chosen edge endpoints (eu[k], ev[k]) for k < count
 * and the reference canonical labels, it returns
 *   0 valid
 *   3 a chosen edge is a self-loop
 *   4 the chosen edges contain a cycle
 *   5 count != n - (number of components)
 *   6 the chosen edges connect a different partition than the reference
 * Membership of each edge in the input and distinctness of ids are checked by
 * the callers below, which know the id space. */
static int or_forest_check(uint32_t n, uint64_t count, const uint32_t* eu, const uint32_t* ev,
                           const uint32_t* ref_labels) {
    uint64_t comps = 0;
    for (uint32_t v = 0; v < n; ++v) comps += (ref_labels[v] == v);
    uint32_t* parent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    uint8_t* rank = (uint8_t*)calloc(n ? n : 1, 1);
    uint32_t* lab = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    for (uint32_t v = 0; v < n; ++v) parent[v] = v;
    int rc = 0;
    for (uint64_t k = 0; k < count && rc == 0; ++k) {
        if (eu[k] == ev[k]) { rc = 3; break; }
        if (!or_union(parent, rank, eu[k], ev[k])) rc = 4;
    }
    if (rc == 0 && count != (uint64_t)n - comps) rc = 5;
    if (rc == 0) {
        or_canonical(n, parent, lab);
        for (uint32_t v = 0; v < n; ++v) if (lab[v] != ref_labels[v]) { rc = 6; break; }
    }
    free(parent); free(rank); free(lab);
    return rc;
}

/* Forest given as COO edge indices.  Extra codes: 1 id >= m, 2 duplicate id. */
int oracle_sf_check(uint32_t n, uint64_t m, const uint32_t* edges, const uint64_t* ids,
                    uint64_t count, const uint32_t* ref_labels) {
    if (count > (uint64_t)n) return 5;
    uint8_t* seen = (uint8_t*)calloc(m ? m : 1, 1);
    uint32_t* eu = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(count + 1));
    uint32_t* ev = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(count + 1));
    int rc = 0;
    for (uint64_t k = 0; k < count; ++k) {
        if (ids[k] >= m) { rc = 1; break; }
        if (seen[ids[k]]) { rc = 2; break; }
        seen[ids[k]] = 1;
        eu[k] = edges[2 * ids[k]]; ev[k] = edges[2 * ids[k] + 1];
        if (eu[k] >= n || ev[k] >= n) { rc = 1; break; }
    }
    if (rc == 0) rc = or_forest_check(n, count, eu, ev, ref_labels);
    free(seen); free(eu); free(ev);
    return rc;
}

/* Forest given as CSR arc positions a (0 <= a < offsets[n]); arc a joins the
 * row that contains it to cols[a].  Extra codes: 1 position out of range,
 * 2 duplicate position. */
int oracle_sf_check_arcs(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                         const uint64_t* ids, uint64_t count, const uint32_t* ref_labels) {
    if (count > (uint64_t)n) return 5;
    uint64_t narcs = offsets[n];
    uint8_t* seen = (uint8_t*)calloc(narcs ? narcs : 1, 1);
    uint32_t* eu = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(count + 1));
    uint32_t* ev = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(count + 1));
    int rc = 0;
    for (uint64_t k = 0; k < count; ++k) {
        uint64_t a = ids[k];
        if (a >= narcs) { rc = 1; break; }
        if (seen[a]) { rc = 2; break; }
        seen[a] = 1;
        /* row = largest r with offsets[r] <= a (binary search) */
        uint32_t lo = 0, hi = n;   /* offsets[lo] <= a < offsets[hi] */
        while (hi - lo > 1) {
            uint32_t mid = lo + (hi - lo) / 2;
            if (offsets[mid] <= a) lo = mid; else hi = mid;
        }
        eu[k] = lo; ev[k] = cols[a];
        if (ev[k] >= n) { rc = 1; break; }
    }
    if (rc == 0) rc = or_forest_check(n, count, eu, ev, ref_labels);
    free(seen); free(eu); free(ev);
    return rc;
}

/* Diagnostic forest: scan edges in input order and keep every edge that joins
 * two different trees (Kruskal's rule with unit weights).  Returns the count. */
uint64_t oracle_kruskal_forest(uint32_t n, uint64_t m, const uint32_t* edges, uint64_t* ids) {
    uint32_t* parent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    uint8_t* rank = (uint8_t*)calloc(n ? n : 1, 1);
    for (uint32_t v = 0; v < n; ++v) parent[v] = v;
    uint64_t c = 0;
    for (uint64_t i = 0; i < m; ++i)
        if (or_union(parent, rank, edges[2 * i], edges[2 * i + 1])) ids[c++] = i;
    free(parent); free(rank);
    return c;
}

/* ---------------- incremental replay (Section 3.5) ----------------
 * Insert batches apply unions; a query batch answers find(u) == find(v)
 * against every edge inserted before it.  The state persists across calls. */
typedef struct { uint32_t n; uint32_t* parent; uint8_t* rank; } oracle_inc;

void* oracle_inc_new(uint32_t n) {
    oracle_inc* s = (oracle_inc*)malloc(sizeof(oracle_inc));
    s->n = n;
    s->parent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    s->rank = (uint8_t*)calloc(n ? n : 1, 1);
    for (uint32_t v = 0; v < n; ++v) s->parent[v] = v;
    return s;
}

int oracle_inc_insert(void* h, uint64_t b, const uint32_t* edges) {
    oracle_inc* s = (oracle_inc*)h;
    for (uint64_t i = 0; i < b; ++i)
        if (edges[2 * i] >= s->n || edges[2 * i + 1] >= s->n) return 2;
    for (uint64_t i = 0; i < b; ++i) or_union(s->parent, s->rank, edges[2 * i], edges[2 * i + 1]);
    return 0;
}

int oracle_inc_query(void* h, uint64_t q, const uint32_t* pairs, uint8_t* out) {
    oracle_inc* s = (oracle_inc*)h;
    for (uint64_t i = 0; i < q; ++i)
        if (pairs[2 * i] >= s->n || pairs[2 * i + 1] >= s->n) return 2;
    for (uint64_t i = 0; i < q; ++i)
        out[i] = or_find(s->parent, pairs[2 * i]) == or_find(s->parent, pairs[2 * i + 1]);
    return 0;
}

void oracle_inc_labels(void* h, uint32_t* labels) {
    oracle_inc* s = (oracle_inc*)h;
    or_canonical(s->n, s->parent, labels);
}

void oracle_inc_free(void* h) {
    oracle_inc* s = (oracle_inc*)h;
    if (!s) return;
    free(s->parent); free(s->rank); free(s);
}
