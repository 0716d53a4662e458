// mt_cc.c -- multicore CPU connected components, for comparison with the GPU
// library: the two-phase method of Algorithm 1 (k-out sampling, L_max by
// sampling, finish over the vertices outside L_max) on the host cores, with
// OpenMP threads and a lock-free min-linking union-find (Union-Rem-CAS with
// SplitAtomicOne, Algorithm 11 and Algorithm 6) on GCC atomics -- the shape of
// the multicore framework the paper compares against (Section 4.8).
//
// It is a measured baseline, not a parity reference (the oracle is); its
// labels are still checked against the oracle by the CPU tests.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#define RLX __ATOMIC_RELAXED

static inline uint32_t ldp(const uint32_t* P, uint32_t i) { return __atomic_load_n(P + i, RLX); }

static inline int casp(uint32_t* P, uint32_t i, uint32_t* expect, uint32_t want) {
    return __atomic_compare_exchange_n(P + i, expect, want, 0, RLX, RLX);
}

// Parent values only decrease (a root is linked under a smaller value, a split
// moves a pointer to its grandparent), so the climb ends.
static void unite(uint32_t* P, uint32_t u, uint32_t v) {
    uint32_t ru = u, rv = v, pu = ldp(P, u), pv = ldp(P, v);
    for (;;) {
        if (pu == pv) return;
        if (pu < pv) {
            uint32_t t = ru; ru = rv; rv = t;
            t = pu; pu = pv; pv = t;
        }
        if (ru == pu) {
            uint32_t e = ru;
            if (casp(P, ru, &e, pv)) return;
            pu = e;                          // linked meanwhile: its fresh parent
        } else {
            uint32_t w = ldp(P, pu);
            if (w != pu) {
                uint32_t e = pu;
                casp(P, ru, &e, w);
            }
            ru = pu;
            pu = w;
        }
    }
}

static inline uint32_t root(const uint32_t* P, uint32_t x) {
    for (;;) {
        uint32_t p = ldp(P, x);
        if (p == x) return x;
        x = p;
    }
}

static inline uint64_t mix64(uint64_t z) {   // SplitMix64 finaliser (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : x > y;
}

// labels[v] = smallest vertex id of v's component.  Returns 0, or 1 when a
// column entry is >= n (labels are then unspecified).
int mt_cc_csr(uint32_t n, const uint64_t* off, const uint32_t* cols, uint32_t* labels, int k, int threads,
              uint64_t seed) {
    if (n == 0) return 0;
    if (threads > 0) omp_set_num_threads(threads);
    uint32_t* P = labels;
    int bad = 0;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < (int64_t)n; ++v) P[v] = (uint32_t)v;
    // sampling: the first k arcs of every vertex
#pragma omp parallel for schedule(dynamic, 4096) reduction(| : bad)
    for (int64_t v = 0; v < (int64_t)n; ++v) {
        uint64_t lo = off[v], hi = off[v + 1];
        uint64_t end = lo + (uint64_t)k < hi ? lo + (uint64_t)k : hi;
        for (uint64_t a = lo; a < end; ++a) {
            uint32_t w = cols[a];
            if (w >= n) { bad = 1; continue; }
            if (w != (uint32_t)v) unite(P, (uint32_t)v, w);
        }
    }
    if (bad) return 1;
    // full compression, then L_max = the most frequent of 1,024 sampled labels
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < (int64_t)n; ++v) P[v] = root(P, (uint32_t)v);
    uint32_t smp[1024];
    for (int i = 0; i < 1024; ++i) smp[i] = P[(uint32_t)(((mix64(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull) >> 32) * n) >> 32)];
    qsort(smp, 1024, sizeof(uint32_t), cmp_u32);
    uint32_t lmax = smp[0], best = 0;
    for (int i = 0, j; i < 1024; i = j) {
        for (j = i; j < 1024 && smp[j] == smp[i]; ++j) {}
        if ((uint32_t)(j - i) > best) { best = (uint32_t)(j - i); lmax = smp[i]; }
    }
    // finish over the vertices outside L_max; each undirected edge once: from
    // its larger endpoint when both are active, else from the active one
    uint8_t* act = (uint8_t*)malloc(n);
    if (!act) return 2;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < (int64_t)n; ++v) act[v] = P[v] != lmax;
#pragma omp parallel for schedule(dynamic, 1024) reduction(| : bad)
    for (int64_t v = 0; v < (int64_t)n; ++v) {
        if (!act[v]) continue;
        for (uint64_t a = off[v]; a < off[v + 1]; ++a) {
            uint32_t u = cols[a];
            if (u >= n) { bad = 1; continue; }
            if (u < (uint32_t)v || !act[u]) unite(P, (uint32_t)v, u);
        }
    }
    free(act);
    if (bad) return 1;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < (int64_t)n; ++v) labels[v] = root(P, (uint32_t)v);
    return 0;
}

int mt_max_threads(void) { return omp_get_max_threads(); }
