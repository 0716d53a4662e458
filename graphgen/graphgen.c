/*
 * graphgen.c -- seeded synthetic graph generators and the COO -> CSR builder.
 *
 * This module only produces inputs.  It holds none of the connectivity
 * method's arithmetic: no union, find, linking or labelling.  Both the CPU
 * oracle (tests only) and the GPU library consume what it writes.
 *
 * Randomness is counter based.  Every draw is the i-th output of a SplitMix64
 * generator (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): state_i = base + (i + 1) * 0x9E3779B97F4A7C15,
 * output = mix(state_i).  Each generator stream gets its own base, derived
 * from the user seed and a stream number, so any draw can be computed
 * independently of the others and in parallel.
 *
 * Integer-only sampling:
 *   uniform integer in [0, n)   : ((h >> 32) * n) >> 32            (n <= 2^32)
 *   event of probability p      : (h >> 32) < p * 2^32  (threshold precomputed
 *                                 by the caller as an integer)
 *
 * Graph shapes follow the workloads the paper evaluates (Section 4, Table 2):
 * Erdos-Renyi multigraphs, RMAT/Kronecker graphs with Graph500 parameters,
 * high-diameter grids and long paths, and a many-small-graphs batch.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (i = 0, 1, ...) of a SplitMix64 generator whose state starts at base. */
static inline uint64_t gg_at(uint64_t base, uint64_t i) { return gg_mix(base + (i + 1) * GG_GAMMA); }

static inline uint64_t gg_stream(uint64_t seed, uint64_t stream) {
    return gg_mix(seed ^ (stream * 0xD1B54A32D192ED03ULL));
}

static inline uint32_t gg_uniform(uint64_t h, uint32_t n) {
    return (uint32_t)(((h >> 32) * (uint64_t)n) >> 32);
}

/* ---- exported primitives (also used by the tests to pin the hash) ---- */

uint64_t gg_splitmix64_at(uint64_t base, uint64_t i) { return gg_at(base, i); }
uint64_t gg_stream_base(uint64_t seed, uint64_t stream) { return gg_stream(seed, stream); }

void gg_hash_fill(uint64_t seed, uint64_t stream, uint64_t start, uint64_t count, uint64_t* out) {
    uint64_t base = gg_stream(seed, stream);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; ++i) out[i] = gg_at(base, start + (uint64_t)i);
}

/* Seeded Fisher-Yates permutation of [0, n) (Knuth, TAOCP vol. 2, Algorithm P). */
void gg_permutation(uint32_t n, uint64_t seed, uint64_t stream, uint32_t* perm) {
    uint64_t base = gg_stream(seed, stream);
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    for (uint32_t i = n; i > 1; --i) {
        uint32_t j = gg_uniform(gg_at(base, i - 1), i);
        uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
    }
}

/* Barabasi-Albert preferential attachment, d edges per new vertex, by the
 * endpoint-copying method of Batagelj and Brandes ("Efficient generation of
 * large random networks", Phys. Rev. E 71, 036113, 2005): the edge list itself
 * is the list of all endpoints so far, and the far end of edge e (vertex
 * v = e / d) is a uniformly chosen earlier entry, i.e. a vertex picked with
 * probability proportional to its degree.  Entry 2e + 1 copies entry r, r
 * uniform in [0, 2e] (r = 2e is v itself: a self-loop, kept, as are
 * duplicates).  Draw e is output e of stream 9.  Sequential by nature. */
void gg_ba(uint32_t n, uint32_t d, uint64_t seed, uint32_t* edges) {
    uint64_t base = gg_stream(seed, 9);
    uint64_t m = (uint64_t)n * d;
    for (uint64_t e = 0; e < m; ++e) {
        edges[2 * e] = (uint32_t)(e / d);
        uint64_t r = (uint64_t)(((unsigned __int128)gg_at(base, e) * (2 * e + 1)) >> 64);
        edges[2 * e + 1] = edges[r];
    }
}

/* Erdos-Renyi G(n, m) multigraph: edge i has endpoints uniform in [0, n), drawn
 * from outputs 2i and 2i+1 of stream 1.  Self-loops and duplicates are kept. */
void gg_er(uint32_t n, uint64_t m, uint64_t seed, uint32_t* edges) {
    uint64_t base = gg_stream(seed, 1);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        edges[2 * i]     = gg_uniform(gg_at(base, 2 * (uint64_t)i), n);
        edges[2 * i + 1] = gg_uniform(gg_at(base, 2 * (uint64_t)i + 1), n);
    }
}

/* One RMAT endpoint pair at the given scale: `scale` quadrant draws, each from
 * its own counter value; quadrant (row bit, column bit) is (0,0) with
 * probability a, (0,1) with b, (1,0) with c and (1,1) with d = 1-a-b-c. */
static inline void gg_rmat_pair(uint64_t base, uint64_t idx, int scale,
                                uint32_t ta, uint32_t tab, uint32_t tabc,
                                uint32_t* pu, uint32_t* pv) {
    uint32_t u = 0, v = 0;
    for (int l = 0; l < scale; ++l) {
        uint32_t r = (uint32_t)(gg_at(base, idx * 64 + (uint64_t)l) >> 32);
        uint32_t bu = r >= tab;                       /* c or d */
        uint32_t bv = (r >= ta && r < tab) || r >= tabc; /* b or d */
        u = (u << 1) | bu;
        v = (v << 1) | bv;
    }
    *pu = u; *pv = v;
}

/* RMAT graph with m edges on 2^scale vertices (Chakrabarti, Zhan, Faloutsos,
 * SDM 2004), no noise.  Thresholds are a, a+b, a+b+c scaled by 2^32.  When
 * perm is non-NULL every endpoint x is replaced by perm[x]. */
void gg_rmat(int scale, uint64_t m, uint32_t ta, uint32_t tab, uint32_t tabc,
             uint64_t seed, const uint32_t* perm, uint32_t* edges) {
    uint64_t base = gg_stream(seed, 2);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        uint32_t u, v;
        gg_rmat_pair(base, (uint64_t)i, scale, ta, tab, tabc, &u, &v);
        if (perm) { u = perm[u]; v = perm[v]; }
        edges[2 * i] = u; edges[2 * i + 1] = v;
    }
}

/* Same stream as gg_rmat, but for edge indices [start, start + count): lets a
 * long insertion stream be produced in pieces. */
void gg_rmat_range(int scale, uint64_t start, uint64_t count, uint32_t ta, uint32_t tab,
                   uint32_t tabc, uint64_t seed, const uint32_t* perm, uint32_t* edges) {
    uint64_t base = gg_stream(seed, 2);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; ++i) {
        uint32_t u, v;
        gg_rmat_pair(base, start + (uint64_t)i, scale, ta, tab, tabc, &u, &v);
        if (perm) { u = perm[u]; v = perm[v]; }
        edges[2 * i] = u; edges[2 * i + 1] = v;
    }
}

/* Uniform random vertex pairs (connectivity queries), stream 7. */
void gg_pairs_range(uint32_t n, uint64_t start, uint64_t count, uint64_t seed, uint32_t* pairs) {
    uint64_t base = gg_stream(seed, 7);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; ++i) {
        uint64_t k = start + (uint64_t)i;
        pairs[2 * i]     = gg_uniform(gg_at(base, 2 * k), n);
        pairs[2 * i + 1] = gg_uniform(gg_at(base, 2 * k + 1), n);
    }
}

/* Shuffle an edge list in place (Fisher-Yates over pairs), stream `stream`. */
void gg_shuffle_edges(uint64_t m, uint64_t seed, uint64_t stream, uint32_t* edges) {
    uint64_t base = gg_stream(seed, stream);
    for (uint64_t i = m; i > 1; --i) {
        uint64_t h = gg_at(base, i - 1);
        uint64_t j = (uint64_t)(((unsigned __int128)h * (unsigned __int128)i) >> 64);
        uint32_t a = edges[2 * (i - 1)], b = edges[2 * (i - 1) + 1];
        edges[2 * (i - 1)] = edges[2 * j]; edges[2 * (i - 1) + 1] = edges[2 * j + 1];
        edges[2 * j] = a; edges[2 * j + 1] = b;
    }
}

/* ---- high-diameter input: 2D grid with random edge removal plus long paths ----
 * Grid: side x side vertices, row-major ids.  Horizontal edge (r,c)-(r,c+1) has
 * index r*(side-1)+c; vertical edge (r,c)-(r+1,c) has index
 * side*(side-1) + r*side + c.  An edge is kept iff the draw at its index
 * (stream 3) is >= keep_threshold (the removal probability times 2^32).
 * Paths: a seeded permutation (stream 4) of the npaths*plen ids that follow the
 * grid; path j visits pi[j*plen], ..., pi[(j+1)*plen - 1] in order.
 * The combined list is shuffled (stream 5).  Returns the number of edges
 * written (call with edges == NULL to get the count only). */
uint64_t gg_grid_paths(uint32_t side, uint32_t remove_threshold, uint32_t npaths, uint32_t plen,
                       uint64_t seed, uint32_t* edges) {
    uint64_t nh = (uint64_t)side * (side - 1), ngrid = 2 * nh;
    uint64_t base = gg_stream(seed, 3);
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    uint64_t nchunks = (uint64_t)nthreads * 8;
    uint64_t chunk = (ngrid + nchunks - 1) / nchunks;
    uint64_t* cnt = (uint64_t*)calloc(nchunks + 1, sizeof(uint64_t));
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < (int64_t)nchunks; ++c) {
        uint64_t lo = (uint64_t)c * chunk, hi = lo + chunk < ngrid ? lo + chunk : ngrid, k = 0;
        for (uint64_t e = lo; e < hi; ++e)
            if ((uint32_t)(gg_at(base, e) >> 32) >= remove_threshold) ++k;
        cnt[c + 1] = k;
    }
    for (uint64_t c = 0; c < nchunks; ++c) cnt[c + 1] += cnt[c];
    uint64_t kept = cnt[nchunks];
    uint64_t npath_edges = (uint64_t)npaths * (plen > 0 ? plen - 1 : 0);
    if (!edges) { free(cnt); return kept + npath_edges; }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < (int64_t)nchunks; ++c) {
        uint64_t lo = (uint64_t)c * chunk, hi = lo + chunk < ngrid ? lo + chunk : ngrid, k = cnt[c];
        for (uint64_t e = lo; e < hi; ++e) {
            if ((uint32_t)(gg_at(base, e) >> 32) < remove_threshold) continue;
            uint32_t u, v;
            if (e < nh) {
                uint32_t r = (uint32_t)(e / (side - 1)), col = (uint32_t)(e % (side - 1));
                u = r * side + col; v = u + 1;
            } else {
                uint64_t f = e - nh;
                uint32_t r = (uint32_t)(f / side), col = (uint32_t)(f % side);
                u = r * side + col; v = u + side;
            }
            edges[2 * k] = u; edges[2 * k + 1] = v; ++k;
        }
    }
    free(cnt);
    uint32_t np = npaths * plen;
    uint32_t* pi = (uint32_t*)malloc((size_t)np * sizeof(uint32_t) + 4);
    gg_permutation(np, seed, 4, pi);
    uint32_t off = side * side;
    uint64_t k = kept;
    for (uint32_t j = 0; j < npaths; ++j)
        for (uint32_t t = 0; t + 1 < plen; ++t) {
            edges[2 * k] = off + pi[(uint64_t)j * plen + t];
            edges[2 * k + 1] = off + pi[(uint64_t)j * plen + t + 1];
            ++k;
        }
    free(pi);
    gg_shuffle_edges(k, seed, 5, edges);
    return k;
}

/* ---- many small graphs ----
 * Sizes: n_i = floor(nmin * (nmax/nmin)^U) (log-uniform), average degree
 * d_i = dmin + (dmax-dmin) * U', m_i = round(n_i * d_i / 2); U, U' from stream 8
 * outputs 2i and 2i+1 (53-bit fractions).  Even i: Erdos-Renyi on local ids;
 * odd i: RMAT at scale ceil(log2 n_i), an endpoint pair with either id >= n_i
 * is rejected and redrawn from the next counter value. */
void gg_batched_sizes(uint32_t G, uint32_t nmin, uint32_t nmax, double dmin, double dmax,
                      uint64_t seed, uint64_t* vtx_off, uint64_t* edge_off) {
    uint64_t base = gg_stream(seed, 8);
    vtx_off[0] = 0; edge_off[0] = 0;
    double ratio = (double)nmax / (double)nmin;
    for (uint32_t i = 0; i < G; ++i) {
        double U = (double)(gg_at(base, 2 * (uint64_t)i) >> 11) * 0x1.0p-53;
        double V = (double)(gg_at(base, 2 * (uint64_t)i + 1) >> 11) * 0x1.0p-53;
        uint64_t ni = (uint64_t)floor((double)nmin * pow(ratio, U));
        if (ni < nmin) ni = nmin;
        if (ni > nmax) ni = nmax;
        double d = dmin + (dmax - dmin) * V;
        uint64_t mi = (uint64_t)llround((double)ni * d / 2.0);
        vtx_off[i + 1] = vtx_off[i] + ni;
        edge_off[i + 1] = edge_off[i] + mi;
    }
}

void gg_batched_fill(uint32_t G, const uint64_t* vtx_off, const uint64_t* edge_off,
                     uint32_t ta, uint32_t tab, uint32_t tabc, uint64_t seed, uint32_t* edges) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t g = 0; g < (int64_t)G; ++g) {
        uint32_t ni = (uint32_t)(vtx_off[g + 1] - vtx_off[g]);
        uint64_t mi = edge_off[g + 1] - edge_off[g];
        uint32_t* e = edges + 2 * edge_off[g];
        uint64_t gb = gg_stream(seed ^ ((uint64_t)g * 0x9E3779B97F4A7C15ULL), 9);
        if ((g & 1) == 0) {
            for (uint64_t j = 0; j < mi; ++j) {
                e[2 * j] = gg_uniform(gg_at(gb, 2 * j), ni);
                e[2 * j + 1] = gg_uniform(gg_at(gb, 2 * j + 1), ni);
            }
        } else {
            int scale = 0;
            while ((1ULL << scale) < ni) ++scale;
            uint64_t ctr = 0;
            for (uint64_t j = 0; j < mi; ++j) {
                uint32_t u, v;
                do { gg_rmat_pair(gb, ctr++, scale, ta, tab, tabc, &u, &v); } while (u >= ni || v >= ni);
                e[2 * j] = u; e[2 * j + 1] = v;
            }
        }
    }
}

/* ---- COO -> symmetric CSR ----
 * Every undirected edge {u,v} becomes the arcs u->v and v->u (a self-loop gives
 * two arcs u->u); duplicates are kept.  Rows are sorted ascending, so the
 * first entry of a row is the smallest neighbour (the CSR layout of Section 2).
 * offsets has n+1 entries, cols 2m entries. */
static int gg_cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

int gg_coo_to_csr(uint32_t n, uint64_t m, const uint32_t* edges, uint64_t* offsets, uint32_t* cols) {
    uint64_t* cur = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!cur) return 1;
    for (uint64_t i = 0; i < m; ++i) {
        if (edges[2 * i] >= n || edges[2 * i + 1] >= n) { free(cur); return 2; }
    }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        __atomic_fetch_add(&cur[edges[2 * i] + 1], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&cur[edges[2 * i + 1] + 1], 1, __ATOMIC_RELAXED);
    }
    offsets[0] = 0;
    for (uint32_t v = 0; v < n; ++v) offsets[v + 1] = offsets[v] + cur[v + 1];
    memcpy(cur, offsets, sizeof(uint64_t) * ((size_t)n + 1));
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        uint32_t u = edges[2 * i], v = edges[2 * i + 1];
        cols[__atomic_fetch_add(&cur[u], 1, __ATOMIC_RELAXED)] = v;
        cols[__atomic_fetch_add(&cur[v], 1, __ATOMIC_RELAXED)] = u;
    }
    free(cur);
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < (int64_t)n; ++v) {
        uint64_t lo = offsets[v], hi = offsets[v + 1];
        if (hi - lo > 1) qsort(cols + lo, hi - lo, sizeof(uint32_t), gg_cmp_u32);
    }
    return 0;
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
