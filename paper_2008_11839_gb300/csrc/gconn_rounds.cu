// gconn_rounds.cu -- round-based finish algorithms: root-based
// Shiloach-Vishkin (Algorithm 12) and the 16 Liu-Tarjan rule sets (appendix
// list), over a COO edge list, and the gather step that feeds them the arcs
// of the active CSR vertices.
//
// Each round is a few grid-stride kernels; a device flag records whether the
// round changed anything and the host reads it (one small copy per round).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gc_internal.h"
#include "gc_static.h"
#include "static_kernels.cuh"

namespace gc {

constexpr unsigned long long NOMSG = 0xFFFFFFFFFFFFFFFFull;
constexpr uint32_t MAX_ROUNDS = 1u << 16;   // round cap: E_NONCONVERGED beyond it

// --------------------------------------------------------------------- SV
// Hook phase as written: labels of both endpoints are read live; the larger
// one is writeMin'ed with the smaller when it was a root at round start.
__global__ void __launch_bounds__(256) k_sv_hook(const uint2* __restrict__ E, uint64_t m, uint32_t n, uint32_t* P,
                                                 const uint32_t* prev, uint32_t* changed, uint32_t* err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool ch = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint2 e = E[i];
        if (e.x >= n || e.y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
        uint32_t pu = __ldcg(P + e.x), pv = __ldcg(P + e.y);
        uint32_t lo = min(pu, pv), hi = max(pu, pv);
        if (lo != hi && prev[hi] == hi) {
            atomicMin(P + hi, lo);
            ch = true;
        }
    }
    if (__any_sync(0xFFFFFFFFu, ch) && (threadIdx.x & 31u) == 0) atomicOr(changed, 1u);
}

// Forest variant: endpoints' round-start roots (prev) are compared, and each
// round-start root h keeps the smallest (label, edge id) message, so the
// recorded edge joins h's tree to the tree it is hooked under.
__global__ void __launch_bounds__(256) k_sv_hook_sf(const uint2* __restrict__ E, const uint32_t* eids, uint64_t m,
                                                    uint32_t n, const uint32_t* prev, unsigned long long* msg,
                                                    uint32_t* err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint2 e = E[i];
        if (e.x >= n || e.y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
        uint32_t pu = prev[e.x], pv = prev[e.y];
        if (pu == pv) continue;
        uint32_t lo = min(pu, pv), hi = max(pu, pv);
        uint32_t id = eids ? eids[i] : (uint32_t)i;
        atomicMin(msg + hi, ((unsigned long long)lo << 32) | id);
    }
}

// Apply the winning messages to roots (P[h] == h at round start) and reset.
__global__ void k_apply_root_msgs(uint32_t n, uint32_t* P, unsigned long long* msg, uint32_t* sf,
                                  uint32_t* changed) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool ch = false;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        unsigned long long mv = msg[x];
        if (mv == NOMSG) continue;
        msg[x] = NOMSG;
        uint32_t val = (uint32_t)(mv >> 32);
        if (P[x] == (uint32_t)x && val < (uint32_t)x) {
            P[x] = val;
            if (sf) sf[x] = (uint32_t)mv;
            ch = true;
        }
    }
    if (__any_sync(0xFFFFFFFFu, ch) && (threadIdx.x & 31u) == 0) atomicOr(changed, 1u);
}

__global__ void k_copy_u32(uint32_t n, const uint32_t* src, uint32_t* dst) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) dst[x] = src[x];
}

__global__ void k_fill_u64(uint64_t n, unsigned long long* a, unsigned long long v) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) a[x] = v;
}

// --------------------------------------------------------------------- LT
// Connect phase; messages are computed from the round-start parents P and
// go to msg[] by atomicMin (packed with the edge id for forests).
//   C: u receives v, v receives u
//   P: P[u] receives P[v], P[v] receives P[u]
//   E: u, v, P[u], P[v] all receive min(P[u], P[v])
__global__ void __launch_bounds__(256) k_lt_connect(const uint2* __restrict__ E, const uint32_t* eids, uint64_t m,
                                                    uint32_t n, const uint32_t* P, int conn,
                                                    unsigned long long* msg, uint32_t* err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint2 e = E[i];
        if (e.x == GC_DINF) continue;   // dropped by Alter
        if (e.x >= n || e.y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
        if (e.x == e.y) continue;
        unsigned long long id = eids ? eids[i] : (uint32_t)i;
        if (conn == GCONN_LT_CONNECT) {
            atomicMin(msg + e.x, ((unsigned long long)e.y << 32) | id);
            atomicMin(msg + e.y, ((unsigned long long)e.x << 32) | id);
        } else {
            uint32_t pu = P[e.x], pv = P[e.y];
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
}

// Update (all vertices) or RootUpdate (roots at round start only).
__global__ void k_lt_update(uint32_t n, uint32_t* P, unsigned long long* msg, int root_only, uint32_t* sf,
                            uint32_t* changed) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool ch = false;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        unsigned long long mv = msg[x];
        if (mv == NOMSG) continue;
        msg[x] = NOMSG;
        uint32_t p = P[x], val = (uint32_t)(mv >> 32);
        if (root_only && p != (uint32_t)x) continue;
        if (val < p) {
            P[x] = val;
            if (sf) sf[x] = (uint32_t)mv;
            ch = true;
        }
    }
    if (__any_sync(0xFFFFFFFFu, ch) && (threadIdx.x & 31u) == 0) atomicOr(changed, 1u);
}

// Shortcut: one pointer jump per vertex (in place).
__global__ void k_lt_shortcut(uint32_t n, uint32_t* P, uint32_t* changed) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool ch = false;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        uint32_t p = __ldcg(P + x), g = __ldcg(P + p);
        if (g != p) {
            __stcg(P + x, g);
            ch = true;
        }
    }
    if (__any_sync(0xFFFFFFFFu, ch) && (threadIdx.x & 31u) == 0) atomicOr(changed, 1u);
}

// Alter: every edge becomes (P[u], P[v]); an edge whose ends meet is dropped.
__global__ void k_lt_alter(uint2* E, uint64_t m, const uint32_t* P, uint32_t* changed) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool ch = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint2 e = E[i];
        if (e.x == GC_DINF) continue;
        uint2 f = make_uint2(P[e.x], P[e.y]);
        if (f.x == f.y) f = make_uint2(GC_DINF, GC_DINF);
        if (f.x != e.x || f.y != e.y) {
            E[i] = f;
            ch = true;
        }
    }
    if (__any_sync(0xFFFFFFFFu, ch) && (threadIdx.x & 31u) == 0) atomicOr(changed, 1u);
}

// --------------------------------------------------------------------- LP
// Label Propagation round: the larger label of each edge takes the smaller.
__global__ void __launch_bounds__(256) k_lp(const uint2* __restrict__ E, uint64_t m, uint32_t n, uint32_t* P,
                                            uint32_t* changed, uint32_t* err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool ch = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint2 e = E[i];
        if (e.x >= n || e.y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
        uint32_t a = __ldcg(P + e.x), b = __ldcg(P + e.y);
        if (a == b) continue;
        uint32_t lo = min(a, b);
        if (a > lo) atomicMin(P + e.x, lo);
        if (b > lo) atomicMin(P + e.y, lo);
        ch = true;
    }
    if (__any_sync(0xFFFFFFFFu, ch) && (threadIdx.x & 31u) == 0) atomicOr(changed, 1u);
}

// ---------------------------------------------------------------- Stergiou
// One round over the previous labels: the entry of each endpoint's label
// receives the other endpoint's label (atomicMin into the current array).
__global__ void __launch_bounds__(256) k_stergiou(const uint2* __restrict__ E, uint64_t m, uint32_t n,
                                                  const uint32_t* prev, uint32_t* P, uint32_t* err) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        uint2 e = E[i];
        if (e.x >= n || e.y >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
        uint32_t a = prev[e.x], b = prev[e.y];
        if (a == b) continue;
        if (b < a) atomicMin(P + a, b);
        else atomicMin(P + b, a);
    }
}

// Compare the current labels with the previous ones (a change means another round).
__global__ void k_changed(uint32_t n, const uint32_t* prev, const uint32_t* P, uint32_t* changed) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool ch = false;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) ch |= prev[x] != P[x];
    if (__any_sync(0xFFFFFFFFu, ch) && (threadIdx.x & 31u) == 0) atomicOr(changed, 1u);
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

__global__ void k_gather_small(const uint64_t* off, const uint32_t* cols, uint32_t n, const uint32_t* active,
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

__global__ void k_gather_tasks(const uint64_t* off, const uint32_t* cols, uint32_t n, const uint32_t* active,
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

__global__ void k_gather_over(const uint64_t* off, const uint32_t* cols, uint32_t n, const uint32_t* active,
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
struct RoundFlag {
    DevBuf dev;
    uint32_t* host = nullptr;
    gconn_status init(cudaStream_t st) {
        GC_TRY(dev.alloc(sizeof(uint32_t), st));
        if (cudaMallocHost(&host, sizeof(uint32_t)) != cudaSuccess) return GCONN_E_NOMEM;
        return GCONN_OK;
    }
    ~RoundFlag() {
        if (host) cudaFreeHost(host);
    }
    uint32_t* d() { return dev.as<uint32_t>(); }
    gconn_status reset(cudaStream_t st) {
        GC_CUDA(cudaMemsetAsync(d(), 0, sizeof(uint32_t), st));
        return GCONN_OK;
    }
    gconn_status read(cudaStream_t st, bool* out) {
        GC_CUDA(cudaMemcpyAsync(host, d(), sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        GC_CUDA(cudaStreamSynchronize(st));
        *out = *host != 0;
        return GCONN_OK;
    }
};

static gconn_status run_sv(const Variant& v, const UFState& s, const uint2* E, const uint32_t* eids, uint64_t m,
                           cudaStream_t st, uint32_t& passes) {
    uint32_t n = s.n;
    DevBuf prevb, msgb;
    GC_TRY(prevb.alloc(sizeof(uint32_t) * (size_t)n, st));
    uint32_t* prev = prevb.as<uint32_t>();
    unsigned long long* msg = nullptr;
    bool sf = s.sf != nullptr;
    unsigned gn = grid_for(k_copy_u32, 256, n);
    if (sf) {
        GC_TRY(msgb.alloc(sizeof(unsigned long long) * (size_t)n, st));
        msg = msgb.as<unsigned long long>();
        GC_TRY(launch("fill_u64", k_fill_u64, grid_for(k_fill_u64, 256, n), 256, 0, st, (uint64_t)n, msg, NOMSG));
    }
    RoundFlag flag;
    GC_TRY(flag.init(st));
    Variant va = v;
    va.link = GCONN_LINK_ASYNC;
    GC_TRY(compress_all(va, s, st));
    GC_TRY(launch("sv_copy", k_copy_u32, gn, 256, 0, st, n, (const uint32_t*)s.P, prev));
    for (uint32_t round = 0;; ++round) {
        if (round >= MAX_ROUNDS) return GCONN_E_NONCONVERGED;
        GC_TRY(flag.reset(st));
        ++passes;
        if (sf) {
            GC_TRY(launch("sv_hook_sf", k_sv_hook_sf, grid_for(k_sv_hook_sf, 256, m), 256, 0, st, E, eids, m, n,
                          (const uint32_t*)prev, msg, s.err));
            GC_TRY(launch("sv_apply", k_apply_root_msgs, gn, 256, 0, st, n, s.P, msg, s.sf, flag.d()));
        } else {
            GC_TRY(launch("sv_hook", k_sv_hook, grid_for(k_sv_hook, 256, m), 256, 0, st, E, m, n, s.P,
                          (const uint32_t*)prev, flag.d(), s.err));
        }
        GC_TRY(compress_all(va, s, st));
        GC_TRY(launch("sv_copy", k_copy_u32, gn, 256, 0, st, n, (const uint32_t*)s.P, prev));
        bool changed = false;
        GC_TRY(flag.read(st, &changed));
        if (!changed) break;
    }
    return GCONN_OK;
}

static gconn_status run_lt(const Variant& v, const UFState& s, const uint2* E_in, const uint32_t* eids, uint64_t m,
                           cudaStream_t st, uint32_t& passes) {
    uint32_t n = s.n;
    int conn = v.lt_rules & 3;
    bool root_only = (v.lt_rules & GCONN_LT_ROOTUPDATE) != 0;
    bool full = (v.lt_rules & GCONN_LT_FULLSHORTCUT) != 0;
    bool alter = (v.lt_rules & GCONN_LT_ALTER) != 0;
    DevBuf msgb, eb;
    GC_TRY(msgb.alloc(sizeof(unsigned long long) * (size_t)n, st));
    unsigned long long* msg = msgb.as<unsigned long long>();
    GC_TRY(launch("fill_u64", k_fill_u64, grid_for(k_fill_u64, 256, n), 256, 0, st, (uint64_t)n, msg, NOMSG));
    const uint2* E = E_in;
    uint2* Ew = nullptr;
    if (alter && m) {
        GC_TRY(eb.alloc(sizeof(uint2) * m, st));
        Ew = eb.as<uint2>();
        GC_CUDA(cudaMemcpyAsync(Ew, E_in, sizeof(uint2) * m, cudaMemcpyDeviceToDevice, st));
        E = Ew;
    }
    RoundFlag flag;
    GC_TRY(flag.init(st));
    Variant va = v;
    va.link = GCONN_LINK_ASYNC;
    unsigned gn = grid_for(k_lt_update, 256, n);
    for (uint32_t round = 0;; ++round) {
        if (round >= MAX_ROUNDS) return GCONN_E_NONCONVERGED;
        GC_TRY(flag.reset(st));
        passes += (m ? 1u : 0u) + (alter && m ? 1u : 0u);   // connect (+ alter) read every edge
        if (m)
            GC_TRY(launch("lt_connect", k_lt_connect, grid_for(k_lt_connect, 256, m), 256, 0, st, E, eids, m, n,
                          (const uint32_t*)s.P, conn, msg, s.err));
        GC_TRY(launch("lt_update", k_lt_update, gn, 256, 0, st, n, s.P, msg, (int)root_only, s.sf, flag.d()));
        if (full) {
            GC_TRY(compress_all(va, s, st));
        } else {
            GC_TRY(launch("lt_shortcut", k_lt_shortcut, gn, 256, 0, st, n, s.P, flag.d()));
        }
        if (alter && m)
            GC_TRY(launch("lt_alter", k_lt_alter, grid_for(k_lt_alter, 256, m), 256, 0, st, Ew, m,
                          (const uint32_t*)s.P, flag.d()));
        bool changed = false;
        GC_TRY(flag.read(st, &changed));
        if (!changed) break;
    }
    return compress_all(va, s, st);
}

static gconn_status run_lp(const Variant& v, const UFState& s, const uint2* E, uint64_t m, cudaStream_t st,
                           uint32_t& passes) {
    RoundFlag flag;
    GC_TRY(flag.init(st));
    for (uint32_t round = 0; m; ++round) {
        if (round >= MAX_ROUNDS) return GCONN_E_NONCONVERGED;
        GC_TRY(flag.reset(st));
        ++passes;
        GC_TRY(launch("lp", k_lp, grid_for(k_lp, 256, m), 256, 0, st, E, m, s.n, s.P, flag.d(), s.err));
        bool changed = false;
        GC_TRY(flag.read(st, &changed));
        if (!changed) break;
    }
    Variant va = v;
    va.link = GCONN_LINK_ASYNC;
    return compress_all(va, s, st);
}

static gconn_status run_stergiou(const Variant& v, const UFState& s, const uint2* E, uint64_t m, cudaStream_t st,
                                 uint32_t& passes) {
    uint32_t n = s.n;
    DevBuf prevb;
    GC_TRY(prevb.alloc(sizeof(uint32_t) * (size_t)n, st));
    uint32_t* prev = prevb.as<uint32_t>();
    RoundFlag flag;
    GC_TRY(flag.init(st));
    unsigned gn = grid_for(k_copy_u32, 256, n);
    for (uint32_t round = 0; m; ++round) {
        if (round >= MAX_ROUNDS) return GCONN_E_NONCONVERGED;
        GC_TRY(flag.reset(st));
        GC_TRY(launch("stergiou_copy", k_copy_u32, gn, 256, 0, st, n, (const uint32_t*)s.P, prev));
        ++passes;
        GC_TRY(launch("stergiou", k_stergiou, grid_for(k_stergiou, 256, m), 256, 0, st, E, m, n,
                      (const uint32_t*)prev, s.P, s.err));
        GC_TRY(launch("lt_shortcut", k_lt_shortcut, gn, 256, 0, st, n, s.P, flag.d()));
        GC_TRY(launch("stergiou_changed", k_changed, gn, 256, 0, st, n, (const uint32_t*)prev,
                      (const uint32_t*)s.P, flag.d()));
        bool changed = false;
        GC_TRY(flag.read(st, &changed));
        if (!changed) break;
    }
    Variant va = v;
    va.link = GCONN_LINK_ASYNC;
    return compress_all(va, s, st);
}

gconn_status rounds_coo(const Variant& v, const UFState& s, const uint32_t* edges, const uint32_t* eids, uint64_t m,
                        cudaStream_t st, uint32_t* edge_passes) {
    uint32_t passes = 0;
    gconn_status r = GCONN_OK;
    if (s.n == 0) r = GCONN_OK;
    else if (v.link == GCONN_LINK_SV) r = run_sv(v, s, (const uint2*)edges, eids, m, st, passes);
    else if (v.link == GCONN_LINK_LP) r = run_lp(v, s, (const uint2*)edges, m, st, passes);
    else if (v.link == GCONN_LINK_STERGIOU) r = run_stergiou(v, s, (const uint2*)edges, m, st, passes);
    else r = run_lt(v, s, (const uint2*)edges, eids, m, st, passes);
    if (edge_passes) *edge_passes = passes;
    return r;
}

gconn_status rounds_csr(const Variant& v, const UFState& s, const uint64_t* off, const uint32_t* cols,
                        const uint32_t* active, const uint32_t* small, const uint32_t* nsmall,
                        const unsigned long long* tasks, const uint32_t* ntasks, uint32_t task_cap,
                        const uint32_t* over, const uint32_t* nover, cudaStream_t st) {
    uint32_t n = s.n;
    uint64_t narcs = 0;
    GC_CUDA(cudaMemcpyAsync(&narcs, off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    GC_CUDA(cudaStreamSynchronize(st));
    DevBuf eb, ib, cb;
    uint64_t cap = narcs ? narcs : 1;
    GC_TRY(eb.alloc(sizeof(uint2) * cap, st));
    GC_TRY(ib.alloc(sizeof(uint32_t) * cap, st));
    GC_TRY(cb.alloc(sizeof(unsigned long long), st));
    Gather g{eb.as<uint2>(), ib.as<uint32_t>(), cb.as<unsigned long long>(), cap};
    GC_CUDA(cudaMemsetAsync(g.cnt, 0, sizeof(unsigned long long), st));
    GC_TRY(launch("gather_small", k_gather_small, grid_for(k_gather_small, 256, n), 256, 0, st, off, cols, n, active,
                  small, nsmall, g, s.err));
    GC_TRY(launch("gather_tasks", k_gather_tasks, grid_for(k_gather_tasks, 256, (uint64_t)n * 32), 256, 0, st, off,
                  cols, n, active, tasks, ntasks, task_cap, g, s.err));
    GC_TRY(launch("gather_over", k_gather_over, grid_for(k_gather_over, 256, (uint64_t)n * 256), 256, 0, st, off,
                  cols, n, active, over, nover, g, s.err));
    unsigned long long m = 0;
    GC_CUDA(cudaMemcpyAsync(&m, g.cnt, sizeof(m), cudaMemcpyDeviceToHost, st));
    GC_CUDA(cudaStreamSynchronize(st));
    if (m > cap) m = cap;
    return rounds_coo(v, s, (const uint32_t*)g.E, g.ids, m, st);
}

}  // namespace gc
