// gconn_bfs.cu -- BFS sampling (Algorithm 4): a direction-optimising BFS
// (Beamer, Asanovic, Patterson, SC 2012) from the highest-degree vertex of a
// seeded sample labels that vertex's component; the reached set is then
// relabelled to its smallest id, which becomes L_max.
//
// The whole BFS is one cooperative launch (every block resident): the levels
// are separated by grid barriers and every block takes the same top-down /
// bottom-up decision from the level's frontier counters, so no level needs a
// host round trip (the paper blames BFS sampling's cost on high-diameter
// graphs on exactly these per-level steps, Section 4.3) and the pass can be
// captured into a CUDA graph.  Counters rotate through three slots: a level
// reads slot L % 3, appends to slot (L + 1) % 3 and clears slot (L + 2) % 3,
// which every block finished reading a level earlier.  On small frontiers of
// low mean degree a level chains: a thread expands one of its own fresh
// claims right away instead of queueing it (the sampling needs the reached
// set, not exact levels), so such a level advances several hops.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gc_internal.h"
#include "gc_static.h"
#include "static_kernels.cuh"

namespace gc {

constexpr int BFS_SAMPLES = 1024;
constexpr int BFS_BLOCK = 256;
constexpr uint64_t BEAMER_ALPHA = 14;   // top-down -> bottom-up when m_f > m_u / alpha
constexpr uint64_t BEAMER_BETA = 24;    // bottom-up -> top-down when n_f < n / beta

struct alignas(128) BfsSlot {    // a line per slot: appends to one do not slow reads of another
    uint32_t qlen;                 // frontier length
    uint32_t heavy;                // a chained level queued a row too long to chain
    unsigned long long degsum;     // arcs out of the frontier
};

struct BfsCtl {
    GridBar bar;
    uint32_t src;                  // BFS source
    uint32_t rmin;                 // smallest reached id
    BfsSlot slot[3];
};

// Top-down claims of one level, staged per block in shared memory: a warp
// reserves its claims with a shared atomic, and the block reserves space on
// the queue once, at the end of the level (stage_flush).  A high-diameter
// graph runs thousands of levels with small frontiers, where one reservation
// per warp on the same two counters costs more than the level's own work.
constexpr uint32_t BFS_STAGE = 1024;
constexpr uint32_t BFS_PROBE_MIN = 16384;   // frontier size from which claims probe first
// Chained expansion on small, low-degree frontiers: a thread expands its
// frontier vertex, then goes on to expand one of the vertices it just claimed
// instead of queueing it, up to BFS_CHAIN_HOPS vertices per level.
constexpr uint32_t BFS_CHAIN_MAX = 1u << 18;  // frontier size up to which levels chain
constexpr uint64_t BFS_CHAIN_DEG = 8;         // ... when the frontier's mean degree is at most this
constexpr uint32_t BFS_CHAIN_HOPS = 16;
constexpr uint32_t BFS_CHAIN_ARCS = 64;       // a row longer than this is left to a warp-per-vertex level
struct BfsStage {
    uint32_t cnt;                  // claims staged (may pass BFS_STAGE: the rest went to the queue)
    uint32_t base;                 // the block's reservation on the queue
    unsigned long long deg;        // arcs out of the staged and overflowed claims
    uint32_t q[BFS_STAGE];
};

__device__ __forceinline__ void warp_stage(bool has, uint32_t val, uint64_t deg, uint32_t* q, BfsSlot* c,
                                           BfsStage& sg) {
    unsigned m = __ballot_sync(0xFFFFFFFFu, has);
    if (!m) return;
    const unsigned lane = threadIdx.x & 31u, leader = __ffs(m) - 1;
    unsigned long long dsum = has ? deg : 0;
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xFFFFFFFFu, dsum, o);
    if (lane == 0 && dsum) atomicAdd(&sg.deg, dsum);
    const uint32_t cnt = __popc(m);
    uint32_t base = 0, gbase = 0;
    if (lane == leader) {
        base = atomicAdd(&sg.cnt, cnt);
        uint32_t room = base < BFS_STAGE ? BFS_STAGE - base : 0;
        if (cnt > room) gbase = atomicAdd(&c->qlen, cnt - room);   // what does not fit goes to the queue now
    }
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    gbase = __shfl_sync(0xFFFFFFFFu, gbase, leader);
    const uint32_t room = base < BFS_STAGE ? BFS_STAGE - base : 0;
    const uint32_t rank = __popc(m & ((1u << lane) - 1));
    if (has) {
        if (rank < room) sg.q[base + rank] = val;
        else q[gbase + rank - room] = val;
    }
}

// One thread's claim, staged in the block's shared list (a shared atomic;
// what does not fit goes to the queue at once).
__device__ __forceinline__ void thread_stage(uint32_t val, uint64_t deg, uint32_t* q, BfsSlot* c, BfsStage& sg) {
    if (deg) atomicAdd(&sg.deg, (unsigned long long)deg);
    const uint32_t p = atomicAdd(&sg.cnt, 1u);
    if (p < BFS_STAGE) sg.q[p] = val;
    else q[atomicAdd(&c->qlen, 1u)] = val;
}

// Every thread of the block, at the end of a top-down level: one reservation
// for the staged claims, copied out coalesced; the staged degree sum is added
// once.  The counters are reset for the next level, which starts after a
// grid barrier (a block synchronisation).
__device__ __forceinline__ void stage_flush(uint32_t* q, BfsSlot* c, BfsStage& sg) {
    __syncthreads();
    const uint32_t k = sg.cnt < BFS_STAGE ? sg.cnt : BFS_STAGE;
    if (threadIdx.x == 0) {
        if (k) sg.base = atomicAdd(&c->qlen, k);
        if (sg.deg) atomicAdd(&c->degsum, sg.deg);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) q[sg.base + i] = sg.q[i];
    if (threadIdx.x == 0) {
        sg.cnt = 0;
        sg.deg = 0;
    }
}

// Block-wide append (every thread of the block calling): one reservation on
// the shared queue counters per block instead of one per warp -- a bottom-up
// level can discover millions of vertices, and per-warp atomics on the same
// two counters serialise at their L2 slice.
__device__ __forceinline__ void block_append(bool has, uint32_t val, uint64_t deg, uint32_t* q, BfsSlot* c) {
    __shared__ uint32_t wcnt[BFS_BLOCK / 32];
    __shared__ unsigned long long wdeg[BFS_BLOCK / 32];
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
        for (int i = 0; i < BFS_BLOCK / 32; ++i) {
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

// Source: the largest degree over BFS_SAMPLES seeded samples, ties to the
// smaller id (one block).
template <class OffT>
__device__ void bfs_pick_source(const OffT* off, uint32_t n, uint64_t seed, BfsCtl* c, uint32_t* dist,
                                uint32_t* queue) {
    __shared__ unsigned long long best;
    if (threadIdx.x == 0) best = 0;
    __syncthreads();
    unsigned long long mine = 0;
    for (unsigned j = threadIdx.x; j < BFS_SAMPLES; j += blockDim.x) {
        uint32_t x = (uint32_t)(((uint64_t)hash_u32(seed ^ 0xB5ull, j) * n) >> 32);
        uint64_t deg = (uint64_t)off[x + 1] - (uint64_t)off[x];
        if (deg > 0xFFFFFFFFull) deg = 0xFFFFFFFFull;
        unsigned long long key = (deg << 32) | (uint32_t)(~x);
        mine = key > mine ? key : mine;
    }
    atomicMax(&best, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = ~(uint32_t)best;
        c->src = s;
        c->rmin = s;
        c->slot[0].qlen = 1;
        c->slot[0].degsum = (uint64_t)off[s + 1] - (uint64_t)off[s];
        dist[s] = 0;
        queue[0] = s;
    }
}

template <class OffT>
__global__ void __launch_bounds__(BFS_BLOCK, 8) k_bfs(const OffT* __restrict__ off, const uint32_t* __restrict__ cols,
                                                   uint32_t n, uint64_t seed, uint32_t* dist, uint32_t* qa,
                                                   uint32_t* qb, BfsCtl* c, uint32_t* P, u64w* W, uint32_t* sf,
                                                   uint32_t* lmax, uint32_t* err) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gw = tid / 32, nw = stride / 32;
    const unsigned lane = threadIdx.x & 31u;
    __shared__ BfsStage sg;
    __shared__ uint32_t s_flen;
    __shared__ unsigned long long s_mf;
    __shared__ uint32_t s_heavy;
    if (threadIdx.x == 0) {
        sg.cnt = 0;
        sg.deg = 0;
    }
    for (uint64_t v = tid; v < n; v += stride) dist[v] = GC_DINF;
    if (!grid_sync(&c->bar, err)) return;
    if (blockIdx.x == 0) bfs_pick_source(off, n, seed, c, dist, qa);
    if (!grid_sync(&c->bar, err)) return;
    const uint64_t narcs = off[n];
    uint64_t mu = 0;
    bool topdown = true;
    uint32_t* q = qa;
    uint32_t* nq = qb;
    for (uint32_t level = 0;; ++level) {
        BfsSlot* cur = &c->slot[level % 3];
        BfsSlot* nxt = &c->slot[(level + 1) % 3];
        if (threadIdx.x == 0) {            // one read of the level's counters per block
            s_flen = __ldcg(&cur->qlen);
            s_mf = __ldcg(&cur->degsum);
            s_heavy = __ldcg(&cur->heavy);
        }
        __syncthreads();
        const uint32_t flen = s_flen;
        const uint64_t mf = s_mf;
        const bool heavy = s_heavy != 0;
        if (flen == 0) break;
        if (level > n) {
            if (tid == 0) atomicOr(err, GC_DERR_NONCONV);
            return;
        }
        mu = level == 0 ? (narcs > mf ? narcs - mf : 0) : (mu > mf ? mu - mf : 0);
        if (topdown && mf > mu / BEAMER_ALPHA) topdown = false;
        else if (!topdown && (uint64_t)flen < (uint64_t)n / BEAMER_BETA) topdown = true;
        if (tid == 0) {                    // the slot every block read a level ago
            BfsSlot* clr = &c->slot[(level + 2) % 3];
            clr->qlen = 0;
            clr->degsum = 0;
            clr->heavy = 0;
        }
        if (topdown && !heavy && flen <= BFS_CHAIN_MAX && mf <= BFS_CHAIN_DEG * (uint64_t)flen) {
            // a thread per frontier vertex, chained: BFS sampling needs the
            // reached set, not exact levels, so a vertex claimed here may be
            // expanded at once (its neighbours are claimed with the same
            // level mark); every claimed vertex is either expanded in the
            // chain or queued, so the reached set is complete when the queue
            // runs dry, and any claimed neighbour is a valid forest parent
            for (uint64_t i = tid; i < flen; i += stride) {
                uint32_t x = __ldcg(q + i);
                for (uint32_t hop = 0; hop < BFS_CHAIN_HOPS; ++hop) {
                    const uint64_t lo = off[x], hi = off[x + 1];
                    if (hi - lo > BFS_CHAIN_ARCS) {
                        // no thread scans a long row alone: queue the vertex
                        // again, marked as a member of the next frontier (a
                        // bottom-up level looks for exactly that mark), and
                        // keep the next level warp-per-vertex
                        dist[x] = level + 1;
                        thread_stage(x, hi - lo, nq, nxt, sg);
                        nxt->heavy = 1;
                        break;
                    }
                    uint32_t next = GC_DINF;
                    for (uint64_t a0 = lo; a0 < hi; a0 += 4) {
                        // four arcs at a time: their columns, then their
                        // claims and degrees, each group of loads in flight together
                        uint32_t y[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) y[k] = a0 + k < hi ? cols[a0 + k] : GC_DINF;
                        uint32_t deg[4];
                        bool got[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            got[k] = false;
                            deg[k] = 0;
                            if (y[k] == GC_DINF) continue;
                            if (y[k] >= n) {
                                atomicOr(err, GC_DERR_RANGE);
                                continue;
                            }
                            const uint64_t dk = (uint64_t)off[y[k] + 1] - (uint64_t)off[y[k]];
                            deg[k] = dk < 0xFFFFFFFFull ? (uint32_t)dk : 0xFFFFFFFFu;
                            got[k] = atomicCAS(dist + y[k], GC_DINF, level + 1) == GC_DINF;
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (!got[k]) continue;
                            if (sf) sf[y[k]] = (uint32_t)(a0 + k);
                            if (next == GC_DINF && hop + 1 < BFS_CHAIN_HOPS) next = y[k];
                            else thread_stage(y[k], deg[k], nq, nxt, sg);
                        }
                    }
                    if (next == GC_DINF) break;
                    x = next;
                }
            }
            stage_flush(nq, nxt, sg);
        } else if (topdown) {              // one warp per frontier vertex claims unvisited neighbours
            // a large frontier reads a neighbour's distance before trying to
            // claim it (most are taken: a load is cheaper than a failed CAS);
            // a small one, latency-bound, goes straight to the CAS
            const bool probe = flen >= BFS_PROBE_MIN;
            for (uint64_t i = gw; i < flen; i += nw) {
                uint32_t u = __ldcg(q + i);
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
                        } else {
                            // y's degree is loaded with the claim, not after it
                            const uint64_t ylo = off[y], yhi = off[y + 1];
                            if ((!probe || __ldcg(dist + y) == GC_DINF) &&
                                atomicCAS(dist + y, GC_DINF, level + 1) == GC_DINF) {
                                claimed = true;
                                if (sf) sf[y] = (uint32_t)a;
                                dy = yhi - ylo;
                            }
                        }
                    }
                    warp_stage(claimed, y, dy, nq, nxt, sg);
                }
            }
            stage_flush(nq, nxt, sg);
        } else {                           // every unvisited vertex looks for a parent in the frontier
            const uint64_t rounds = ((uint64_t)n + stride - 1) / stride;
            for (uint64_t r = 0; r < rounds; ++r) {     // uniform trip count for the block-wide append
                uint64_t v = tid + r * stride;
                bool found = false;
                uint64_t deg = 0;
                if (v < n && __ldcg(dist + v) == GC_DINF) {
                    uint64_t lo = off[v], hi = off[v + 1];
                    for (uint64_t a = lo; a < hi; ++a) {
                        uint32_t y = cols[a];
                        if (y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
                        if (__ldcg(dist + y) == level) {
                            __stcg(dist + v, level + 1);
                            if (sf) sf[v] = (uint32_t)a;
                            found = true;
                            deg = hi - lo;
                            break;
                        }
                    }
                }
                block_append(found, (uint32_t)v, deg, nq, nxt);
            }
        }
        if (!grid_sync(&c->bar, err)) return;
        uint32_t* t = q; q = nq; nq = t;
    }
    // the reached set's smallest id r, then every reached vertex points at r
    // (a root, so parents never exceed their vertex; rank 1 for Union-JTB)
    uint32_t best = GC_DINF;
    for (uint64_t v = tid; v < n; v += stride)
        if (__ldcg(dist + v) != GC_DINF && (uint32_t)v < best) best = (uint32_t)v;
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xFFFFFFFFu, best, o));
    if (lane == 0 && best != GC_DINF) atomicMin(&c->rmin, best);
    if (!grid_sync(&c->bar, err)) return;
    const uint32_t r = __ldcg(&c->rmin);
    if (tid == 0) *lmax = r;
    for (uint64_t v = tid; v < n; v += stride) {
        if (__ldcg(dist + v) == GC_DINF) continue;
        if (W) W[v] = wmake((uint32_t)v == r ? 1u : 0u, r);
        else P[v] = r;
    }
}

template <class OffT>
gconn_status bfs_sample(const Variant& v, const UFState& s, const OffT* off, const uint32_t* cols,
                        uint32_t* lmax_dev, cudaStream_t st) {
    uint32_t n = s.n;
    DevBuf dbuf, q0, q1, cbuf;
    GC_TRY(dbuf.alloc(sizeof(uint32_t) * (size_t)n, st));
    GC_TRY(q0.alloc(sizeof(uint32_t) * (size_t)n, st));
    GC_TRY(q1.alloc(sizeof(uint32_t) * (size_t)n, st));
    GC_TRY(cbuf.alloc(sizeof(BfsCtl), st));
    GC_CUDA(cudaMemsetAsync(cbuf.p, 0, sizeof(BfsCtl), st));
    auto k = k_bfs<OffT>;
    return launch_coop("bfs", k, grid_for(k, BFS_BLOCK, n), BFS_BLOCK, 0, st, off, cols, n, v.seed,
                       dbuf.as<uint32_t>(), q0.as<uint32_t>(), q1.as<uint32_t>(), cbuf.as<BfsCtl>(), s.P, s.W, s.sf,
                       lmax_dev, s.err);
}

template gconn_status bfs_sample<uint32_t>(const Variant&, const UFState&, const uint32_t*, const uint32_t*,
                                          uint32_t*, cudaStream_t);
template gconn_status bfs_sample<uint64_t>(const Variant&, const UFState&, const uint64_t*, const uint32_t*,
                                          uint32_t*, cudaStream_t);

}  // namespace gc
