// gconn_rounds.cu -- round-based finish algorithms: root-based
// Shiloach-Vishkin (Algorithm 12), the 16 Liu-Tarjan rule sets (appendix
// list), label propagation and Stergiou's algorithm, over a COO edge list,
// and the gather step that feeds them the arcs of the active CSR vertices.
//
// Each algorithm runs as ONE cooperative launch (every block resident) that
// loops over its rounds on the device: the phases of a round (an edge pass,
// vertex passes) are separated by grid barriers, a round that changes
// anything records its number in a control word, and every block reads that
// word after the round's last barrier to decide, identically, whether to run
// another round.  No host round trip per round, so these finishes can also be
// captured into a CUDA graph.  Arrays that other blocks wrote earlier in the
// same launch are read through L2 (ld.global.cg): L1 is not coherent
// between blocks.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "gc_internal.h"
#include "gc_static.h"
#include "static_kernels.cuh"

namespace gc {

constexpr unsigned long long NOMSG = 0xFFFFFFFFFFFFFFFFull;
constexpr uint32_t MAX_ROUNDS = 1u << 16;   // round cap: E_NONCONVERGED beyond it
constexpr int RB = 256;                     // block size of the round kernels

// Control words of one round kernel, zeroed before its launch.  chg only
// grows: after round r's last barrier every block reads it, and it is at
// least r + 1 exactly when round r changed something (a block that already
// went on to round r + 1 can only have raised it further).
struct RoundCtl {
    GridBar bar;
    uint32_t chg;      // 1 + the last round in which something changed
    uint32_t rounds;   // rounds run (written once, at the end)
    uint32_t pad[4];
};

__device__ __forceinline__ uint64_t gtid() { return (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ uint64_t gstride() { return (uint64_t)gridDim.x * blockDim.x; }

// Records that round r changed something (one atomic per block); called by
// every thread of a block at the same point.
__device__ __forceinline__ void mark_changed(bool ch, uint32_t* chg, uint32_t r) {
    if (__syncthreads_or(ch) && threadIdx.x == 0) atomicMax(chg, r + 1);
}

// Whether round r changed anything, read after the round's last barrier:
// thread 0 reads the word once for the block.  The next round reaches
// another barrier (which synchronises the block) before it reads again.
__device__ __forceinline__ bool round_changed(const RoundCtl* ctl, uint32_t r) {
    __shared__ uint32_t s_chg;
    if (threadIdx.x == 0) s_chg = __ldcg(&ctl->chg);
    __syncthreads();
    return s_chg >= r + 1;
}

__device__ __forceinline__ uint64_t edge_count(uint64_t m_host, const unsigned long long* m_dev) {
    if (!m_dev) return m_host;
    unsigned long long m = __ldcg(m_dev);
    return m < m_host ? m : m_host;
}

// FullShortcut while nothing links: every vertex points at its root (a walk
// through L2), and prev (optional) receives the same value.
__device__ __forceinline__ void compress_copy(uint32_t n, uint32_t* P, uint32_t* prev, uint32_t* err) {
    for (uint64_t v = gtid(); v < n; v += gstride()) {
        uint32_t p = __ldcg(P + v), r = p;
        for (uint32_t i = 0;; ++i) {
            uint32_t q = __ldcg(P + r);
            if (q == r) break;
            r = q;
            if (i == n) { atomicOr(err, GC_DERR_NONCONV); break; }
        }
        if (r != p) __stcg(P + v, r);
        if (prev) __stcg(prev + v, r);
    }
}

// The round cap: every block reaches it in the same round.
__device__ __forceinline__ bool over_cap(uint32_t r, uint32_t* err) {
    if (r < MAX_ROUNDS) return false;
    if (gtid() == 0) atomicOr(err, GC_DERR_NONCONV);
    return true;
}

__device__ __forceinline__ void finish_rounds(RoundCtl* ctl, uint32_t r) {
    if (gtid() == 0) ctl->rounds = r;
}

// --------------------------------------------------------------------- SV
// Shiloach-Vishkin (Algorithm 12), root-based.  Per round: the hook pass --
// for each edge the larger of its two current labels is writeMin'ed with the
// smaller when it was a root at round start (prev); forest form: each
// round-start root keeps the smallest (label, edge id) message, applied in a
// vertex pass -- then full compression, which also copies the labels into
// prev.  Stop after a round that hooked nothing.
template <bool SF>
__global__ void __launch_bounds__(RB) k_sv(const uint2* __restrict__ E, const uint32_t* eids, uint64_t m_host,
                                           const unsigned long long* m_dev, uint32_t n, uint32_t* P, uint32_t* prev,
                                           unsigned long long* msg, uint32_t* sf, uint32_t* err, RoundCtl* ctl) {
    const uint64_t m = edge_count(m_host, m_dev);
    compress_copy(n, P, prev, err);
    if (SF)
        for (uint64_t x = gtid(); x < n; x += gstride()) msg[x] = NOMSG;
    if (!grid_sync(&ctl->bar, err)) return;
    for (uint32_t r = 0;; ++r) {
        if (over_cap(r, err)) return;
        bool ch = false;
        for (uint64_t i = gtid(); i < m; i += gstride()) {
            uint2 e = E[i];
            if (e.x >= n || e.y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
            if (SF) {
                uint32_t pu = __ldcg(prev + e.x), pv = __ldcg(prev + e.y);
                if (pu == pv) continue;
                uint32_t lo = min(pu, pv), hi = max(pu, pv);
                uint32_t id = eids ? eids[i] : (uint32_t)i;
                atomicMin(msg + hi, ((unsigned long long)lo << 32) | id);
            } else {
                uint32_t pu = __ldcg(P + e.x), pv = __ldcg(P + e.y);
                uint32_t lo = min(pu, pv), hi = max(pu, pv);
                if (lo != hi && __ldcg(prev + hi) == hi) {
                    atomicMin(P + hi, lo);
                    ch = true;
                }
            }
        }
        if (!SF) mark_changed(ch, &ctl->chg, r);
        if (!grid_sync(&ctl->bar, err)) return;
        if (SF) {   // apply the winning messages to round-start roots
            for (uint64_t x = gtid(); x < n; x += gstride()) {
                unsigned long long mv = __ldcg(msg + x);
                if (mv == NOMSG) continue;
                msg[x] = NOMSG;
                uint32_t val = (uint32_t)(mv >> 32);
                if (__ldcg(P + x) == (uint32_t)x && val < (uint32_t)x) {
                    __stcg(P + x, val);
                    sf[x] = (uint32_t)mv;
                    ch = true;
                }
            }
            mark_changed(ch, &ctl->chg, r);
            if (!grid_sync(&ctl->bar, err)) return;
        }
        compress_copy(n, P, prev, err);
        if (!grid_sync(&ctl->bar, err)) return;
        if (!round_changed(ctl, r)) {   // no change in round r (chg only grows)
            finish_rounds(ctl, r + 1);
            return;
        }
    }
}

// --------------------------------------------------------------------- LT
// One Liu-Tarjan rule set per launch (runtime flags).  Per round: Connect
// messages from the round-start parents go to msg by atomicMin (packed with
// the edge id for forests):
//   C: u receives v, v receives u
//   P: P[u] receives P[v], P[v] receives P[u]
//   E: u, v, P[u], P[v] all receive min(P[u], P[v])
// then Update (all vertices) or RootUpdate (round-start roots only), then one
// Shortcut jump per vertex or FullShortcut, then Alter (edge <- (P[u], P[v]),
// dropped when the ends meet).  Stop after a round that changes neither a
// parent nor an edge; then full compression.
__global__ void __launch_bounds__(RB) k_lt(const uint2* __restrict__ E_in, uint2* Ew, const uint32_t* eids,
                                           uint64_t m_host, const unsigned long long* m_dev, uint32_t n, uint32_t* P,
                                           unsigned long long* msg, uint32_t* sf, int conn, int root_only, int full,
                                           uint32_t* err, RoundCtl* ctl) {
    const uint64_t m = edge_count(m_host, m_dev);
    const bool alter = Ew != nullptr;
    for (uint64_t x = gtid(); x < n; x += gstride()) msg[x] = NOMSG;
    if (!grid_sync(&ctl->bar, err)) return;
    for (uint32_t r = 0;; ++r) {
        if (over_cap(r, err)) return;
        bool ch = false;
        for (uint64_t i = gtid(); i < m; i += gstride()) {      // Connect
            uint2 e = alter ? __ldcg(Ew + i) : E_in[i];
            if (e.x == GC_DINF) continue;                       // dropped by Alter
            if (e.x >= n || e.y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
            if (e.x == e.y) continue;
            unsigned long long id = eids ? eids[i] : (uint32_t)i;
            if (conn == GCONN_LT_CONNECT) {
                atomicMin(msg + e.x, ((unsigned long long)e.y << 32) | id);
                atomicMin(msg + e.y, ((unsigned long long)e.x << 32) | id);
            } else {
                uint32_t pu = __ldcg(P + e.x), pv = __ldcg(P + e.y);
                if (pu == pv) continue;
                if (conn == GCONN_LT_PARENT) {
                    atomicMin(msg + pu, ((unsigned long long)pv << 32) | id);
                    atomicMin(msg + pv, ((unsigned long long)pu << 32) | id);
                } else {
                    unsigned long long lo = ((unsigned long long)min(pu, pv) << 32) | id;
                    atomicMin(msg + e.x, lo);
                    atomicMin(msg + e.y, lo);
                    atomicMin(msg + pu, lo);
                    atomicMin(msg + pv, lo);
                }
            }
        }
        if (!grid_sync(&ctl->bar, err)) return;
        for (uint64_t x = gtid(); x < n; x += gstride()) {      // Update / RootUpdate
            unsigned long long mv = __ldcg(msg + x);
            if (mv == NOMSG) continue;
            msg[x] = NOMSG;
            uint32_t p = __ldcg(P + x), val = (uint32_t)(mv >> 32);
            if (root_only && p != (uint32_t)x) continue;
            if (val < p) {
                __stcg(P + x, val);
                if (sf) sf[x] = (uint32_t)mv;
                ch = true;
            }
        }
        mark_changed(ch, &ctl->chg, r);
        if (!grid_sync(&ctl->bar, err)) return;
        ch = false;
        if (full) {
            compress_copy(n, P, nullptr, err);
        } else {                                                // one jump, in place
            for (uint64_t x = gtid(); x < n; x += gstride()) {
                uint32_t p = __ldcg(P + x), g2 = __ldcg(P + p);
                if (g2 != p) {
                    __stcg(P + x, g2);
                    ch = true;
                }
            }
            mark_changed(ch, &ctl->chg, r);
        }
        if (!grid_sync(&ctl->bar, err)) return;
        if (alter) {
            ch = false;
            for (uint64_t i = gtid(); i < m; i += gstride()) {
                uint2 e = __ldcg(Ew + i);
                if (e.x == GC_DINF) continue;
                uint2 f = make_uint2(__ldcg(P + e.x), __ldcg(P + e.y));
                if (f.x == f.y) f = make_uint2(GC_DINF, GC_DINF);
                if (f.x != e.x || f.y != e.y) {
                    __stcg(Ew + i, f);
                    ch = true;
                }
            }
            mark_changed(ch, &ctl->chg, r);
            if (!grid_sync(&ctl->bar, err)) return;
        }
        if (!round_changed(ctl, r)) {   // no change in round r (chg only grows)
            finish_rounds(ctl, r + 1);
            break;
        }
    }
    compress_copy(n, P, nullptr, err);
}

// --------------------------------------------------------------------- LP
// Label Propagation: per round, for each edge the larger endpoint label takes
// the smaller (atomicMin on both ends); stop after a round that changes
// nothing; then full compression.
__global__ void __launch_bounds__(RB) k_lp(const uint2* __restrict__ E, uint64_t m_host,
                                           const unsigned long long* m_dev, uint32_t n, uint32_t* P, uint32_t* err,
                                           RoundCtl* ctl) {
    const uint64_t m = edge_count(m_host, m_dev);
    for (uint32_t r = 0; m; ++r) {
        if (over_cap(r, err)) return;
        bool ch = false;
        for (uint64_t i = gtid(); i < m; i += gstride()) {
            uint2 e = E[i];
            if (e.x >= n || e.y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
            uint32_t a = __ldcg(P + e.x), b = __ldcg(P + e.y);
            if (a == b) continue;
            uint32_t lo = min(a, b);
            if (a > lo) atomicMin(P + e.x, lo);
            if (b > lo) atomicMin(P + e.y, lo);
            ch = true;
        }
        mark_changed(ch, &ctl->chg, r);
        if (!grid_sync(&ctl->bar, err)) return;
        if (!round_changed(ctl, r)) {   // no change in round r (chg only grows)
            finish_rounds(ctl, r + 1);
            break;
        }
    }
    compress_copy(n, P, nullptr, err);
}

// ---------------------------------------------------------------- Stergiou
// Per round: for each edge the entry of the larger of prev[u], prev[v]
// receives the smaller (atomicMin into the current labels), then one
// shortcut jump per vertex; the round changed something if a jump moved or a
// label differs from prev.  The shortcut pass also writes the next round's
// prev (each entry is written there by its own thread only).
__global__ void __launch_bounds__(RB) k_stergiou(const uint2* __restrict__ E, uint64_t m_host,
                                                 const unsigned long long* m_dev, uint32_t n, uint32_t* P,
                                                 uint32_t* prev, uint32_t* err, RoundCtl* ctl) {
    const uint64_t m = edge_count(m_host, m_dev);
    for (uint64_t x = gtid(); x < n; x += gstride()) prev[x] = __ldcg(P + x);
    if (!grid_sync(&ctl->bar, err)) return;
    for (uint32_t r = 0; m; ++r) {
        if (over_cap(r, err)) return;
        for (uint64_t i = gtid(); i < m; i += gstride()) {
            uint2 e = E[i];
            if (e.x >= n || e.y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
            uint32_t a = __ldcg(prev + e.x), b = __ldcg(prev + e.y);
            if (a == b) continue;
            if (b < a) atomicMin(P + a, b);
            else atomicMin(P + b, a);
        }
        if (!grid_sync(&ctl->bar, err)) return;
        bool ch = false;
        for (uint64_t x = gtid(); x < n; x += gstride()) {
            uint32_t p = __ldcg(P + x), g2 = __ldcg(P + p);
            if (g2 != p) {
                __stcg(P + x, g2);
                ch = true;
            }
            if (__ldcg(prev + x) != g2) ch = true;
            __stcg(prev + x, g2);
        }
        mark_changed(ch, &ctl->chg, r);
        if (!grid_sync(&ctl->bar, err)) return;
        if (!round_changed(ctl, r)) {   // no change in round r (chg only grows)
            finish_rounds(ctl, r + 1);
            break;
        }
    }
    compress_copy(n, P, nullptr, err);
}

// ------------------------------------------------------------- CSR gather
struct Gather {
    uint2* E;
    uint32_t* ids;
    unsigned long long* cnt;
    unsigned long long cap;
};

__device__ __forceinline__ void gather_arc(const Gather& g, uint32_t u, uint32_t v, uint32_t a) {
    unsigned long long k = atomicAdd(g.cnt, 1ull);
    if (k < g.cap) {
        g.E[k] = make_uint2(u, v);
        g.ids[k] = a;
    }
}

template <class OffT>
__global__ void k_gather_small(const OffT* off, const uint32_t* cols, uint32_t n, const uint32_t* active,
                               const uint32_t* small, const uint32_t* nsmall, Gather g, uint32_t* err) {
    uint32_t cnt = *nsmall;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
        uint32_t u = small[i];
        for (uint64_t a = off[u]; a < off[u + 1]; ++a) {
            uint32_t v = cols[a];
            if (v >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
            if (arc_needed(active, u, v)) gather_arc(g, u, v, (uint32_t)a);
        }
    }
}

template <class OffT>
__global__ void k_gather_tasks(const OffT* off, const uint32_t* cols, uint32_t n, const uint32_t* active,
                               const unsigned long long* tasks, const uint32_t* ntasks, uint32_t task_cap, Gather g,
                               uint32_t* err) {
    uint32_t cnt = min(*ntasks, task_cap);
    uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    unsigned lane = threadIdx.x & 31u;
    for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; t < cnt; t += nw) {
        unsigned long long task = tasks[t];
        uint32_t u = (uint32_t)(task >> 32);
        uint64_t lo = off[u] + (task & 0xFFFFFFFFull) * TASK_ARCS, hi = off[u + 1];
        if (lo + TASK_ARCS < hi) hi = lo + TASK_ARCS;
        for (uint64_t a = lo + lane; a < hi; a += 32) {
            uint32_t v = cols[a];
            if (v >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
            if (arc_needed(active, u, v)) gather_arc(g, u, v, (uint32_t)a);
        }
    }
}

template <class OffT>
__global__ void k_gather_over(const OffT* off, const uint32_t* cols, uint32_t n, const uint32_t* active,
                              const uint32_t* over, const uint32_t* nover, Gather g, uint32_t* err) {
    uint64_t cnt = *nover;
    for (uint64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
        uint32_t u = over[i];
        for (uint64_t a = off[u] + threadIdx.x; a < off[u + 1]; a += blockDim.x) {
            uint32_t v = cols[a];
            if (v >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
            if (arc_needed(active, u, v)) gather_arc(g, u, v, (uint32_t)a);
        }
    }
}

// ------------------------------------------------------------------ drivers
// Scratch for one round kernel: its control words (zeroed on the stream).
struct RoundLaunch {
    DevBuf ctlb;
    RoundCtl* ctl = nullptr;
    gconn_status init(cudaStream_t st) {
        GC_TRY(ctlb.alloc(sizeof(RoundCtl), st));
        ctl = ctlb.as<RoundCtl>();
        GC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(RoundCtl), st));
        return GCONN_OK;
    }
    // Rounds run, for the edge-pass count (waits for the stream).
    gconn_status rounds(cudaStream_t st, uint32_t* out) {
        uint32_t r = 0;
        GC_CUDA(cudaMemcpyAsync(&r, &ctl->rounds, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        GC_CUDA(cudaStreamSynchronize(st));
        *out = r;
        return GCONN_OK;
    }
};

template <class K>
unsigned round_grid(K kernel, uint64_t m, uint32_t n) {
    return grid_for(kernel, RB, std::max<uint64_t>(m, n));
}

static gconn_status run_sv(const UFState& s, const uint2* E, const uint32_t* eids, uint64_t m,
                           const unsigned long long* m_dev, cudaStream_t st, uint32_t* rounds) {
    uint32_t n = s.n;
    DevBuf prevb, msgb;
    GC_TRY(prevb.alloc(sizeof(uint32_t) * (size_t)n, st));
    unsigned long long* msg = nullptr;
    bool sf = s.sf != nullptr;
    if (sf) {
        GC_TRY(msgb.alloc(sizeof(unsigned long long) * (size_t)n, st));
        msg = msgb.as<unsigned long long>();
    }
    RoundLaunch rl;
    GC_TRY(rl.init(st));
    auto k = sf ? k_sv<true> : k_sv<false>;
    GC_TRY(launch_coop("sv", k, round_grid(k, m, n), RB, 0, st, E, eids, m, m_dev, n, s.P, prevb.as<uint32_t>(), msg,
                       s.sf, s.err, rl.ctl));
    return rounds ? rl.rounds(st, rounds) : GCONN_OK;
}

static gconn_status run_lt(const Variant& v, const UFState& s, const uint2* E_in, const uint32_t* eids, uint64_t m,
                           const unsigned long long* m_dev, cudaStream_t st, uint32_t* rounds) {
    uint32_t n = s.n;
    int conn = v.lt_rules & 3;
    bool root_only = (v.lt_rules & GCONN_LT_ROOTUPDATE) != 0;
    bool full = (v.lt_rules & GCONN_LT_FULLSHORTCUT) != 0;
    bool alter = (v.lt_rules & GCONN_LT_ALTER) != 0;
    DevBuf msgb, eb;
    GC_TRY(msgb.alloc(sizeof(unsigned long long) * (size_t)n, st));
    uint2* Ew = nullptr;
    if (alter && m) {   // Alter rewrites the edges: work on a copy
        GC_TRY(eb.alloc(sizeof(uint2) * m, st));
        Ew = eb.as<uint2>();
        GC_CUDA(cudaMemcpyAsync(Ew, E_in, sizeof(uint2) * m, cudaMemcpyDeviceToDevice, st));
    }
    RoundLaunch rl;
    GC_TRY(rl.init(st));
    GC_TRY(launch_coop("lt", k_lt, round_grid(k_lt, m, n), RB, 0, st, E_in, Ew, eids, m, m_dev, n, s.P,
                       msgb.as<unsigned long long>(), s.sf, conn, (int)root_only, (int)full, s.err, rl.ctl));
    if (!rounds) return GCONN_OK;
    GC_TRY(rl.rounds(st, rounds));
    *rounds *= (m ? 1u : 0u) + (alter && m ? 1u : 0u);   // connect (+ alter) read every edge
    return GCONN_OK;
}

static gconn_status run_lp(const UFState& s, const uint2* E, uint64_t m, const unsigned long long* m_dev,
                           cudaStream_t st, uint32_t* rounds) {
    RoundLaunch rl;
    GC_TRY(rl.init(st));
    GC_TRY(launch_coop("lp", k_lp, round_grid(k_lp, m, s.n), RB, 0, st, E, m, m_dev, s.n, s.P, s.err, rl.ctl));
    return rounds ? rl.rounds(st, rounds) : GCONN_OK;
}

static gconn_status run_stergiou(const UFState& s, const uint2* E, uint64_t m, const unsigned long long* m_dev,
                                 cudaStream_t st, uint32_t* rounds) {
    DevBuf prevb;
    GC_TRY(prevb.alloc(sizeof(uint32_t) * (size_t)s.n, st));
    RoundLaunch rl;
    GC_TRY(rl.init(st));
    GC_TRY(launch_coop("stergiou", k_stergiou, round_grid(k_stergiou, m, s.n), RB, 0, st, E, m, m_dev, s.n, s.P,
                       prevb.as<uint32_t>(), s.err, rl.ctl));
    return rounds ? rl.rounds(st, rounds) : GCONN_OK;
}

gconn_status rounds_coo(const Variant& v, const UFState& s, const uint32_t* edges, const uint32_t* eids, uint64_t m,
                        cudaStream_t st, uint32_t* edge_passes, const unsigned long long* m_dev) {
    uint32_t passes = 0;
    uint32_t* pp = edge_passes ? &passes : nullptr;
    gconn_status r = GCONN_OK;
    const uint2* E = (const uint2*)edges;
    if (s.n == 0) r = GCONN_OK;
    else if (v.link == GCONN_LINK_SV) r = run_sv(s, E, eids, m, m_dev, st, pp);
    else if (v.link == GCONN_LINK_LP) r = run_lp(s, E, m, m_dev, st, pp);
    else if (v.link == GCONN_LINK_STERGIOU) r = run_stergiou(s, E, m, m_dev, st, pp);
    else r = run_lt(v, s, E, eids, m, m_dev, st, pp);
    if (edge_passes) *edge_passes = passes;
    return r;
}

template <class OffT>
gconn_status rounds_csr(const Variant& v, const UFState& s, const OffT* off, const uint32_t* cols,
                        const uint32_t* active, const uint32_t* small, const uint32_t* nsmall,
                        const unsigned long long* tasks, const uint32_t* ntasks, uint32_t task_cap,
                        const uint32_t* over, const uint32_t* nover, cudaStream_t st) {
    uint32_t n = s.n;
    // the gathered arcs are at most all arcs: the host needs offsets[n] to
    // size the list (known in advance while a plan is being captured)
    uint64_t narcs = csr_arcs_hint();
    if (narcs == UINT64_MAX) {
        OffT last = 0;
        GC_CUDA(cudaMemcpyAsync(&last, off + n, sizeof(OffT), cudaMemcpyDeviceToHost, st));
        GC_CUDA(cudaStreamSynchronize(st));
        narcs = last;
    }
    DevBuf eb, ib, cb;
    uint64_t cap = narcs ? narcs : 1;
    GC_TRY(eb.alloc(sizeof(uint2) * cap, st));
    GC_TRY(ib.alloc(sizeof(uint32_t) * cap, st));
    GC_TRY(cb.alloc(sizeof(unsigned long long), st));
    Gather g{eb.as<uint2>(), ib.as<uint32_t>(), cb.as<unsigned long long>(), cap};
    GC_CUDA(cudaMemsetAsync(g.cnt, 0, sizeof(unsigned long long), st));
    GC_TRY(launch("gather_small", k_gather_small<OffT>, grid_for(k_gather_small<OffT>, 256, n), 256, 0, st, off,
                  cols, n, active, small, nsmall, g, s.err));
    GC_TRY(launch("gather_tasks", k_gather_tasks<OffT>, grid_for(k_gather_tasks<OffT>, 256, (uint64_t)n * 32), 256,
                  0, st, off, cols, n, active, tasks, ntasks, task_cap, g, s.err));
    GC_TRY(launch("gather_over", k_gather_over<OffT>, grid_for(k_gather_over<OffT>, 256, (uint64_t)n * 256), 256, 0,
                  st, off, cols, n, active, over, nover, g, s.err));
    // the rounds read the gathered count on the device
    return rounds_coo(v, s, (const uint32_t*)g.E, g.ids, cap, st, nullptr, g.cnt);
}

template gconn_status rounds_csr<uint32_t>(const Variant&, const UFState&, const uint32_t*, const uint32_t*,
                                          const uint32_t*, const uint32_t*, const uint32_t*,
                                          const unsigned long long*, const uint32_t*, uint32_t, const uint32_t*,
                                          const uint32_t*, cudaStream_t);
template gconn_status rounds_csr<uint64_t>(const Variant&, const UFState&, const uint64_t*, const uint32_t*,
                                          const uint32_t*, const uint32_t*, const uint32_t*,
                                          const unsigned long long*, const uint32_t*, uint32_t, const uint32_t*,
                                          const uint32_t*, cudaStream_t);

}  // namespace gc
