// gconn_bfs.cu -- BFS sampling (Algorithm 4): a direction-optimising BFS
// (Beamer, Asanovic, Patterson, SC 2012) from the highest-degree vertex of a
// seeded sample labels that vertex's component; the reached set is then
// relabelled to its smallest id, which becomes L_max.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gc_internal.h"
#include "gc_static.h"
#include "static_kernels.cuh"

namespace gc {

constexpr int BFS_SAMPLES = 1024;
constexpr uint64_t BEAMER_ALPHA = 14;   // top-down -> bottom-up when m_f > m_u / alpha
constexpr uint64_t BEAMER_BETA = 24;    // bottom-up -> top-down when n_f < n / beta

struct BfsCounters {
    uint32_t qlen;                 // next-frontier length
    uint32_t src;                  // BFS source
    unsigned long long degsum;     // arcs out of the next frontier
    uint32_t rmin;                 // smallest reached id
    uint32_t pad;
};

// Source: the largest degree over a seeded sample, ties to the smaller id.
__global__ void __launch_bounds__(BFS_SAMPLES) k_bfs_source(const uint64_t* off, uint32_t n, uint64_t seed,
                                                            uint32_t* dist, uint32_t* queue, BfsCounters* c) {
    __shared__ unsigned long long best;
    if (threadIdx.x == 0) best = 0;
    __syncthreads();
    uint32_t x = (uint32_t)(((uint64_t)hash_u32(seed ^ 0xB5ull, threadIdx.x) * n) >> 32);
    uint64_t deg = off[x + 1] - off[x];
    if (deg > 0xFFFFFFFFull) deg = 0xFFFFFFFFull;
    atomicMax(&best, (deg << 32) | (uint32_t)(~x));
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = ~(uint32_t)best;
        c->src = s;
        c->qlen = 1;
        c->degsum = off[s + 1] - off[s];
        c->rmin = s;
        dist[s] = 0;
        queue[0] = s;
    }
}

__device__ __forceinline__ void warp_append(bool has, uint32_t val, uint64_t deg, uint32_t* q, BfsCounters* c) {
    unsigned m = __ballot_sync(0xFFFFFFFFu, has);
    if (!m) return;
    unsigned lane = threadIdx.x & 31u;
    unsigned leader = __ffs(m) - 1;
    unsigned long long dsum = has ? deg : 0;
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xFFFFFFFFu, dsum, o);
    dsum = __shfl_sync(0xFFFFFFFFu, dsum, 0);
    uint32_t base = 0;
    if (lane == leader) {
        base = atomicAdd(&c->qlen, (uint32_t)__popc(m));
        atomicAdd(&c->degsum, dsum);
    }
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (has) q[base + __popc(m & ((1u << lane) - 1))] = val;
}

// Top-down step: one warp per frontier vertex claims unvisited neighbours.
__global__ void __launch_bounds__(256) k_bfs_td(const uint64_t* __restrict__ off, const uint32_t* __restrict__ cols,
                                                uint32_t n, const uint32_t* frontier, uint32_t flen, uint32_t level,
                                                uint32_t* dist, uint32_t* next, BfsCounters* c, uint32_t* sf,
                                                uint32_t* err) {
    uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    unsigned lane = threadIdx.x & 31u;
    for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; i < flen; i += nw) {
        uint32_t u = frontier[i];
        uint64_t lo = off[u], hi = off[u + 1];
        for (uint64_t base = lo; base < hi; base += 32) {
            uint64_t a = base + lane;
            bool claimed = false;
            uint32_t y = 0;
            uint64_t dy = 0;
            if (a < hi) {
                y = cols[a];
                if (y >= n) {
                    atomicOr(err, GC_DERR_RANGE);
                } else if (__ldcg(dist + y) == GC_DINF && atomicCAS(dist + y, GC_DINF, level + 1) == GC_DINF) {
                    claimed = true;
                    if (sf) sf[y] = (uint32_t)a;
                    dy = off[y + 1] - off[y];
                }
            }
            warp_append(claimed, y, dy, next, c);
        }
    }
}

// Block-wide append (blocks of BFS_BU_BLOCK threads, every thread calling):
// one reservation on the shared queue counters per block instead of one per
// warp -- a bottom-up level can discover millions of vertices, and per-warp
// atomics on the same two counters serialise at their L2 slice.
constexpr int BFS_BU_BLOCK = 256;

__device__ __forceinline__ void block_append(bool has, uint32_t val, uint64_t deg, uint32_t* q, BfsCounters* c) {
    __shared__ uint32_t wcnt[BFS_BU_BLOCK / 32];
    __shared__ unsigned long long wdeg[BFS_BU_BLOCK / 32];
    __shared__ uint32_t bbase;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x / 32;
    unsigned m = __ballot_sync(0xFFFFFFFFu, has);
    unsigned long long dsum = has ? deg : 0;
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xFFFFFFFFu, dsum, o);
    if (lane == 0) {
        wcnt[warp] = __popc(m);
        wdeg[warp] = dsum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        unsigned long long dtot = 0;
        for (int i = 0; i < BFS_BU_BLOCK / 32; ++i) {
            uint32_t x = wcnt[i];
            wcnt[i] = tot;                 // exclusive prefix over the warps
            tot += x;
            dtot += wdeg[i];
        }
        bbase = tot ? atomicAdd(&c->qlen, tot) : 0;
        if (dtot) atomicAdd(&c->degsum, dtot);
    }
    __syncthreads();
    if (has) q[bbase + wcnt[warp] + __popc(m & ((1u << lane) - 1))] = val;
    __syncthreads();                       // wcnt / bbase are reused by the next round
}

// Bottom-up step: every unvisited vertex looks for a parent in the frontier.
__global__ void __launch_bounds__(BFS_BU_BLOCK) k_bfs_bu(const uint64_t* __restrict__ off,
                                                         const uint32_t* __restrict__ cols, uint32_t n,
                                                         uint32_t level, uint32_t* dist, uint32_t* next,
                                                         BfsCounters* c, uint32_t* sf, uint32_t* err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t start = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t rounds = ((uint64_t)n + stride - 1) / stride;
    for (uint64_t r = 0; r < rounds; ++r) {     // uniform trip count for the block-wide append
        uint64_t v = start + r * stride;
        bool found = false;
        uint64_t deg = 0;
        if (v < n && __ldcg(dist + v) == GC_DINF) {
            uint64_t lo = off[v], hi = off[v + 1];
            for (uint64_t a = lo; a < hi; ++a) {
                uint32_t y = cols[a];
                if (y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
                if (__ldcg(dist + y) == level) {
                    dist[v] = level + 1;
                    if (sf) sf[v] = (uint32_t)a;
                    found = true;
                    deg = hi - lo;
                    break;
                }
            }
        }
        block_append(found, (uint32_t)v, deg, next, c);
    }
}

__global__ void k_bfs_min(uint32_t n, const uint32_t* dist, BfsCounters* c) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t best = GC_DINF;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (dist[v] != GC_DINF && (uint32_t)v < best) best = (uint32_t)v;
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xFFFFFFFFu, best, o));
    if ((threadIdx.x & 31u) == 0 && best != GC_DINF) atomicMin(&c->rmin, best);
}

// Reached vertices point at the smallest reached id r (a root), so parents
// never exceed their vertex; for Union-JTB r gets rank 1.
__global__ void k_bfs_label(uint32_t n, const uint32_t* dist, const BfsCounters* c, uint32_t* P, u64w* W,
                            uint32_t* lmax) {
    uint32_t r = c->rmin;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (first == 0) *lmax = r;
    for (uint64_t v = first; v < n; v += stride) {
        if (dist[v] == GC_DINF) continue;
        if (W) W[v] = wmake((uint32_t)v == r ? 1u : 0u, r);
        else P[v] = r;
    }
}

gconn_status bfs_sample(const Variant& v, const UFState& s, const uint64_t* off, const uint32_t* cols,
                        uint32_t* lmax_dev, cudaStream_t st) {
    uint32_t n = s.n;
    DevBuf dbuf, q0, q1, cbuf;
    GC_TRY(dbuf.alloc(sizeof(uint32_t) * (size_t)n, st));
    GC_TRY(q0.alloc(sizeof(uint32_t) * (size_t)n, st));
    GC_TRY(q1.alloc(sizeof(uint32_t) * (size_t)n, st));
    GC_TRY(cbuf.alloc(sizeof(BfsCounters), st));
    uint32_t* dist = dbuf.as<uint32_t>();
    uint32_t* qa = q0.as<uint32_t>();
    uint32_t* qb = q1.as<uint32_t>();
    BfsCounters* c = cbuf.as<BfsCounters>();
    // The per-level counter read-back goes through a pinned buffer kept per
    // host thread (a pinned allocation per call would cost more than a level).
    struct PinnedCounters {
        BfsCounters* p = nullptr;
        ~PinnedCounters() {
            if (p) cudaFreeHost(p);
        }
    };
    static thread_local PinnedCounters pinned;
    if (!pinned.p) GC_CUDA(cudaMallocHost(&pinned.p, sizeof(BfsCounters)));
    BfsCounters* hc = pinned.p;

    uint64_t narcs = 0;
    GC_CUDA(cudaMemcpyAsync(&narcs, off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    GC_TRY(launch("bfs_fill", k_fill, grid_for(k_fill, 256, n), 256, 0, st, n, dist, INF));
    GC_TRY(launch("bfs_source", k_bfs_source, 1, BFS_SAMPLES, 0, st, off, n, v.seed, dist, qa, c));
    GC_CUDA(cudaMemcpyAsync(hc, c, sizeof(BfsCounters), cudaMemcpyDeviceToHost, st));
    GC_CUDA(cudaStreamSynchronize(st));
    uint32_t flen = hc->qlen;
    uint64_t mf = hc->degsum, mu = narcs > mf ? narcs - mf : 0;
    bool topdown = true;
    unsigned gtd = grid_for(k_bfs_td, 256, (uint64_t)n * 32);
    unsigned gbu = grid_for(k_bfs_bu, 256, n);
    for (uint32_t level = 0; flen > 0; ++level) {
        if (level > n) return GCONN_E_NONCONVERGED;
        if (topdown && mf > mu / BEAMER_ALPHA) topdown = false;
        else if (!topdown && (uint64_t)flen < (uint64_t)n / BEAMER_BETA) topdown = true;
        GC_CUDA(cudaMemsetAsync(c, 0, offsetof(BfsCounters, rmin), st));   // qlen, src, degsum
        if (topdown)
            GC_TRY(launch("bfs_td", k_bfs_td, gtd, 256, 0, st, off, cols, n, qa, flen, level, dist, qb, c, s.sf,
                          s.err));
        else
            GC_TRY(launch("bfs_bu", k_bfs_bu, gbu, 256, 0, st, off, cols, n, level, dist, qb, c, s.sf, s.err));
        GC_CUDA(cudaMemcpyAsync(hc, c, sizeof(BfsCounters), cudaMemcpyDeviceToHost, st));
        GC_CUDA(cudaStreamSynchronize(st));
        flen = hc->qlen;
        mf = hc->degsum;
        mu = mu > mf ? mu - mf : 0;
        uint32_t* t = qa; qa = qb; qb = t;
    }
    GC_TRY(launch("bfs_min", k_bfs_min, grid_for(k_bfs_min, 256, n), 256, 0, st, n, dist, c));
    return launch("bfs_label", k_bfs_label, grid_for(k_bfs_label, 256, n), 256, 0, st, n, dist, c, s.P, s.W,
                  lmax_dev);
}

}  // namespace gc
