// static_kernels.cuh -- kernels of the static two-phase method (Algorithm 1,
// Algorithm 2) shared by the COO and CSR paths: label initialisation, COO
// finish, k-out / HB sampling, full compression, L_max, vertex gathering,
// load-balanced CSR finish, finalisation and forest compaction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "uf_device.cuh"

namespace gc {

constexpr int SMALL_DEG = 32;     // CSR finish: thread per vertex up to this degree
constexpr int TASK_ARCS = 256;    // CSR finish: arcs per warp task above it
constexpr int LMAX_SAMPLES = 1024;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t hash_u32(uint64_t seed, uint64_t i) {
    unsigned long long z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (uint32_t)((z ^ (z >> 31)) >> 32);
}

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialisation attribute may be scheduled while the grid before it in
// the stream is still running; griddepcontrol.wait blocks until that grid has
// completed and its writes are visible, and launch_dependents then lets the
// next kernel's blocks be scheduled early in turn.  Both are no-ops for a
// kernel launched normally, so every kernel that starts with pdl_entry() may
// be launched either way.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ bool err_abort(const uint32_t* err) {
    return (__ldcg(err) & GC_DERR_NONCONV) != 0;
}

// InitLabel (Algorithm 1) and InitEdge (Algorithm 2): P[v] = v, hooks and
// forest slots to "none", JTB words to (rank 0, parent v).
// `zero` (nzero words, may be null) is cleared too: the pass's counters.
static __global__ void k_init(uint32_t n, uint32_t* P, uint32_t* H, u64w* W, uint32_t* sf, uint32_t* zero,
                              uint32_t nzero) {
    pdl_entry();
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (zero && blockIdx.x == 0)
        for (uint32_t i = threadIdx.x; i < nzero; i += blockDim.x) zero[i] = 0;
    if (P && !H && !W && !sf && ((uintptr_t)P & 15u) == 0) {   // P only: 16-byte stores
        uint64_t nv = n / 4;
        uint4* P4 = reinterpret_cast<uint4*>(P);
        for (uint64_t i = t0; i < nv; i += stride) {
            uint32_t b = (uint32_t)(4 * i);
            P4[i] = make_uint4(b, b + 1, b + 2, b + 3);
        }
        for (uint64_t v = nv * 4 + t0; v < n; v += stride) P[v] = (uint32_t)v;
        return;
    }
    for (uint64_t v = t0; v < n; v += stride) {
        if (P) P[v] = (uint32_t)v;
        if (H) H[v] = GC_DINF;
        if (W) W[v] = wmake(0, (uint32_t)v);
        if (sf) sf[v] = GC_DINF;
    }
}

// Finish phase over a COO edge list (Section 3.5 batches use it too): one
// union per edge, grid-stride, edges streamed once.  eid_base offsets the
// recorded forest ids (incremental batches).
template <int L, int F, int S, bool SF>
static __global__ void __launch_bounds__(256) k_union_coo(const uint2* __restrict__ E, uint64_t m, UFState s,
                                                   uint32_t eid_base) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t it = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        if ((++it & 63u) == 0 && err_abort(s.err)) return;
        uint2 e = __ldcs(E + i);
        if (e.x >= s.n || e.y >= s.n) {
            atomicOr(s.err, GC_DERR_RANGE);
            continue;
        }
        if (e.x == e.y) continue;
        Spin sp(s.cap);
        uf_union<L, F, S, SF>(s, e.x, e.y, eid_base + (uint32_t)i, sp);
    }
}

// k-out sampling (Algorithm 2, first k edges of every vertex).  A warp takes
// 32 consecutive vertices, reads their first k <= KOUT_WARP_K column entries
// (one sector per row), and packs one job per vertex with a sampled arc into
// a per-warp list in shared memory with a ballot prefix: isolated vertices
// (often ~40 % of an RMAT graph) leave the high lanes idle instead of
// scattering idle lanes through the warp.  A lane runs its vertex's unions one
// after the other (RMAT scale 22: 79 -> 73 us against one job per arc, where
// a vertex's two unions raced for its own entry on two lanes; refilling the
// idle lanes from the next word, 32 jobs per round, took 83-85 us: more
// unions at once only add contention).  Larger k falls back to one thread per
// vertex.
constexpr int KOUT_WARP_K = 2;
constexpr int KOUT_BLOCK = 256;

struct KoutJob {
    uint32_t u, v, eid;
};

// Deferred unions: a union that has not finished within KOUT_FAST_STEPS loop
// steps is abandoned (the forest it leaves is valid: only root links and
// compression happened) and re-run later from its endpoints by
// k_union_jobs, so a few long climbs do not hold 31 idle lanes.
constexpr uint32_t KOUT_FAST_STEPS = 8;

struct JobQueue {
    KoutJob* jobs;
    unsigned long long* count;
    uint32_t cap;
};

// One union under the soft budget when a queue is given: an abandoned union
// goes to the queue (or, if it is full, runs on with the full cap).
template <int L, int F, int S, bool SF>
__device__ __forceinline__ void union_or_defer(const UFState& s, const JobQueue& dq, uint32_t a, uint32_t b,
                                               uint32_t eid) {
    if (dq.jobs) {
        Spin fast(KOUT_FAST_STEPS, true);
        uf_union<L, F, S, SF>(s, a, b, eid, fast);
        if (!fast.dead) return;
        unsigned long long slot = atomicAdd(dq.count, 1ull);
        if (slot < dq.cap) {   // resume where the climb stopped (see Spin)
            dq.jobs[slot] = KoutJob{fast.at_u != GC_DINF ? fast.at_u : a, fast.at_v != GC_DINF ? fast.at_v : b, eid};
            return;
        }
    }
    Spin sp(s.cap);
    uf_union<L, F, S, SF>(s, a, b, eid, sp);
}

template <int L, int F, int S, bool SF, class OffT = uint64_t>
// plain: one thread per vertex over its first k arcs (the form without the
// per-warp packing; also taken for k > KOUT_WARP_K).
static __global__ void __launch_bounds__(KOUT_BLOCK) k_kout(const OffT* __restrict__ off,
                                                            const uint32_t* __restrict__ cols, int k, UFState s,
                                                            JobQueue dq, bool plain) {
    pdl_entry();
    __shared__ uint4 jobs[KOUT_BLOCK / 32][32];   // (v, first arc, second arc, arc index)
    if (k > KOUT_WARP_K || plain) {
        uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < s.n; v += stride) {
            uint64_t lo = off[v], hi = off[v + 1];
            uint64_t end = lo + (uint64_t)k < hi ? lo + (uint64_t)k : hi;
            for (uint64_t a = lo; a < end; ++a) {
                uint32_t w = cols[a];
                if (w >= s.n) { atomicOr(s.err, GC_DERR_RANGE); continue; }
                if (w == (uint32_t)v) continue;
                Spin sp(s.cap);
                uf_union<L, F, S, SF>(s, (uint32_t)v, w, (uint32_t)a, sp);
            }
        }
        return;
    }
    uint4* my = jobs[threadIdx.x / 32];
    unsigned lane = lane_id();
    unsigned lt = (1u << lane) - 1;
    uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    uint64_t nwords = ((uint64_t)s.n + 31) / 32;
    // Two-deep software pipeline over this warp's words: while word i's
    // unions drain, the column loads of word i+1 and the offset loads of
    // word i+2 are in flight.
    // Words are taken from the highest vertex ids down.  A high-id vertex's
    // smallest neighbour is almost always below it, so while it is still a
    // root its first union links it by a CAS on its own entry; a low-id
    // vertex's unions instead link its neighbours' roots under it, entries
    // that many warps reach at once.  Starting high keeps the early, most
    // concurrent part of the kernel on uncontended CASes (RMAT scale 22:
    // 87 -> 78 us for this kernel).
    uint64_t w = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    auto load_off = [&](uint64_t ww, uint64_t& lo, uint64_t& hi) {
        uint64_t x = (nwords - 1 - ww) * 32 + lane;
        lo = hi = 0;
        if (ww < nwords && x < s.n) {
            lo = off[x];
            hi = off[x + 1];
        }
    };
    auto load_cols = [&](uint64_t lo, uint64_t hi, uint32_t& c0, uint32_t& c1) {
        c0 = hi > lo ? cols[lo] : GC_DINF;
        c1 = (k > 1 && hi > lo + 1) ? cols[lo + 1] : GC_DINF;
    };
    uint64_t lo0, hi0, lo1, hi1;
    uint32_t c0, c1;
    load_off(w, lo0, hi0);
    load_off(w + nwarps, lo1, hi1);
    load_cols(lo0, hi0, c0, c1);
    for (; w < nwords; w += nwarps) {
        uint32_t n0, n1;
        uint64_t lo2, hi2;
        load_cols(lo1, hi1, n0, n1);             // word i+1
        load_off(w + 2 * nwarps, lo2, hi2);      // word i+2
        uint64_t v = (nwords - 1 - w) * 32 + lane;
        if ((c0 != GC_DINF && c0 >= s.n) || (c1 != GC_DINF && c1 >= s.n)) atomicOr(s.err, GC_DERR_RANGE);
        bool j0 = c0 < s.n && c0 != (uint32_t)v;
        bool j1 = c1 < s.n && c1 != (uint32_t)v;
        // one job per vertex with a sampled arc, packed to the low lanes: the
        // lane runs the vertex's unions one after the other, so the two
        // unions of a vertex never race for its own parent entry
        bool jv = j0 || j1;
        unsigned mv = __ballot_sync(0xFFFFFFFFu, jv);
        if (jv) my[__popc(mv & lt)] = make_uint4((uint32_t)v, j0 ? c0 : GC_DINF, j1 ? c1 : GC_DINF, (uint32_t)lo0);
        __syncwarp();
        if (lane < (unsigned)__popc(mv)) {
            uint4 jb = my[lane];
            if (jb.y != GC_DINF) union_or_defer<L, F, S, SF>(s, dq, jb.x, jb.y, jb.w);
            if (jb.z != GC_DINF) union_or_defer<L, F, S, SF>(s, dq, jb.x, jb.z, jb.w + 1);
        }
        __syncwarp();
        lo0 = lo1; hi0 = hi1; c0 = n0; c1 = n1;
        lo1 = lo2; hi1 = hi2;
    }
}

// GetMostFrequentLabel (Algorithm 1): mode of the root labels of
// LMAX_SAMPLES seeded random vertices, ties to the smaller label.  A block of
// any size (a multiple of 32) walks the samples to their roots (thread t takes
// samples t, t + blockDim, ...) and counts them in a shared-memory
// open-addressing table; the best (count, smallest label) wins.  L1 selects
// L1-allowed parent loads (only safe in a kernel that has not itself changed P).
constexpr uint32_t LMAX_SLOTS = 2 * LMAX_SAMPLES;

struct LmaxSmem {
    uint32_t key[LMAX_SLOTS];
    uint32_t cnt[LMAX_SLOTS];
    unsigned long long wbest[32];
};

template <int L, bool L1>
__device__ void block_lmax(const UFState& s, uint64_t seed, uint32_t* lmax_out, LmaxSmem& sm) {
    const unsigned t = threadIdx.x, nt = blockDim.x;
    for (unsigned i = t; i < LMAX_SLOTS; i += nt) {
        sm.key[i] = GC_DINF;
        sm.cnt[i] = 0;
    }
    __syncthreads();
    for (unsigned j = t; j < LMAX_SAMPLES; j += nt) {   // every lane of a warp runs the same iterations
        uint32_t x = (uint32_t)(((uint64_t)hash_u32(seed, j) * s.n) >> 32);
        uint32_t lab = uf_root<L, L1>(s, x);
        // lanes holding the same label add it once (the big component's label
        // would otherwise serialise hundreds of shared-memory atomics)
        unsigned peers = __match_any_sync(0xFFFFFFFFu, lab);
        if ((unsigned)(__ffs(peers) - 1) == lane_id()) {
            uint32_t slot = hash_u32(0x5A17ull, lab) & (LMAX_SLOTS - 1);
            for (uint32_t probe = 0; probe < LMAX_SLOTS; ++probe) {
                uint32_t prev = atomicCAS(&sm.key[slot], GC_DINF, lab);
                if (prev == GC_DINF || prev == lab) {
                    atomicAdd(&sm.cnt[slot], (uint32_t)__popc(peers));
                    break;
                }
                slot = (slot + 1) & (LMAX_SLOTS - 1);
            }
        }
    }
    __syncthreads();
    // larger count wins, on a tie the smaller label (larger ~label): a
    // shuffle max per warp, then over the warps
    unsigned long long mine = 0;
    for (unsigned i = t; i < LMAX_SLOTS; i += nt)
        if (sm.cnt[i]) {
            unsigned long long kv = ((unsigned long long)sm.cnt[i] << 32) | (uint32_t)(~sm.key[i]);
            mine = kv > mine ? kv : mine;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, mine, o);
        mine = other > mine ? other : mine;
    }
    if (lane_id() == 0) sm.wbest[t / 32] = mine;
    __syncthreads();
    if (t < 32) {
        mine = t < nt / 32 ? sm.wbest[t] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, mine, o);
            mine = other > mine ? other : mine;
        }
        if (t == 0) *lmax_out = ~(uint32_t)mine;
    }
}

template <int L>
static __global__ void __launch_bounds__(LMAX_SAMPLES) k_lmax(UFState s, uint64_t seed, uint32_t* lmax_out) {
    pdl_entry();
    __shared__ LmaxSmem sm;
    block_lmax<L, true>(s, seed, lmax_out, sm);
}

// Unions deferred by k_kout / k_hb2w, finished with the full cap from where
// each abandoned climb stopped (see Spin).
// Blocks of LMAX_SAMPLES threads.  L_max needs every union done, so it is
// resolved by the block that finishes last (a counter taken after a fence;
// `done` must start at zero): no block waits for another, the last one just
// does more work.  It reads parents through L2 only, since its own L1 may
// hold lines from before other blocks' links.
// With mode_tmp set (grids of at least two blocks), block 0 takes the most
// frequent root label of the samples right away, while the other blocks run
// the deferred unions, and the last block only walks that label to its root:
// a label's root only moves down its own set, so L_max = root(mode) picks the
// same set without serialising 1,024 walks behind the unions.  Otherwise the
// last block computes the mode of the samples' final roots itself.
template <int L, int F, int S, bool SF>
static __global__ void __launch_bounds__(LMAX_SAMPLES) k_union_jobs(UFState s, JobQueue dq, uint64_t seed,
                                                           uint32_t* lmax_out, uint32_t* done, uint32_t* mode_tmp) {
    pdl_entry();
    __shared__ LmaxSmem sm;
    __shared__ bool last;
    constexpr int LR = L == LK_JTB ? LK_JTB : LK_ASYNC;
    unsigned long long cnt = *dq.count;
    if (cnt > dq.cap) cnt = dq.cap;
    const bool split = mode_tmp && gridDim.x > 1;
    if (split && blockIdx.x == 0) {
        block_lmax<LR, false>(s, seed, mode_tmp, sm);
    } else {
        uint64_t b0 = split ? blockIdx.x - 1 : blockIdx.x, nb = split ? gridDim.x - 1 : gridDim.x;
        uint64_t stride = nb * blockDim.x;
        for (uint64_t i = b0 * blockDim.x + threadIdx.x; i < cnt; i += stride) {
            KoutJob jb = dq.jobs[i];
            Spin sp(s.cap);
            uf_union<L, F, S, SF>(s, jb.u, jb.v, jb.eid, sp);
        }
    }
    if (!lmax_out) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (split) {
        if (threadIdx.x == 0) *lmax_out = uf_root<LR, false>(s, __ldcg(mode_tmp));
        return;
    }
    block_lmax<LR, false>(s, seed, lmax_out, sm);
}

// HB sampling step 1 (Algorithm 3): P[v] = min(v, w) for the smallest
// neighbour w = cols[off[v]].  Each thread writes only its own P[v].
template <class OffT = uint64_t>
static __global__ void k_hb1(const OffT* __restrict__ off, const uint32_t* __restrict__ cols, uint32_t n,
                      uint32_t* P, uint32_t* sf, uint32_t* err) {
    pdl_entry();
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint64_t lo = off[v];
        if (off[v + 1] > lo) {
            uint32_t w = cols[lo];
            if (w >= n) { atomicOr(err, GC_DERR_RANGE); continue; }
            if (w < (uint32_t)v) {
                P[v] = w;
                if (sf) sf[v] = (uint32_t)lo;
            }
        }
    }
}

// InitLabel fused with HB step 1 (Algorithm 3): P[v] = the smallest
// neighbour w = cols[off[v]] when w < v, else v; a hooked vertex's forest slot
// records arc off[v]; hooks are cleared and so is `zero` (the pass's
// counters).  Every thread writes only its own entries and nothing reads P in
// this kernel, so step 1 needs no separate initialisation pass before it.
template <class OffT = uint64_t>
static __global__ void k_hb_init(const OffT* __restrict__ off, const uint32_t* __restrict__ cols, uint32_t n,
                                 uint32_t* P, uint32_t* H, uint32_t* sf, uint32_t* err, uint32_t* zero,
                                 uint32_t nzero) {
    pdl_entry();
    if (zero && blockIdx.x == 0)
        for (uint32_t i = threadIdx.x; i < nzero; i += blockDim.x) zero[i] = 0;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint64_t lo = off[v];
        uint32_t p = (uint32_t)v, e = GC_DINF;
        if (off[v + 1] > lo) {
            uint32_t w = cols[lo];
            if (w >= n) atomicOr(err, GC_DERR_RANGE);
            else if (w < (uint32_t)v) {
                p = w;
                e = (uint32_t)lo;
            }
        }
        P[v] = p;
        if (H) H[v] = GC_DINF;
        if (sf) sf[v] = e;
    }
}

// HB sampling step 2 with the k-out machinery: a warp takes 32 consecutive
// vertices, keeps those still roots after step 1 (no smaller first
// neighbour, read from the row), packs the unions of their first
// N <= HB_WARP_N arcs into a per-warp job list in shared memory (ballot
// prefix) and drains it with all lanes; a union still climbing after
// KOUT_FAST_STEPS steps is deferred to k_union_jobs.  A thread per vertex
// would leave most lanes idle while a few run four unions in sequence.
constexpr int HB_WARP_N = 4;

template <int L, int F, int S, bool SF, class OffT = uint64_t>
static __global__ void __launch_bounds__(256) k_hb2w(const OffT* __restrict__ off,
                                                     const uint32_t* __restrict__ cols, int N, UFState s,
                                                     JobQueue dq) {
    pdl_entry();
    __shared__ KoutJob jobs[256 / 32][32 * HB_WARP_N];
    KoutJob* my = jobs[threadIdx.x / 32];
    const unsigned lane = lane_id(), lt = (1u << lane) - 1;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const uint64_t nwords = ((uint64_t)s.n + 31) / 32;
    // as in k_kout: words from the highest ids down, offsets of word i+2 and
    // columns of word i+1 in flight while word i's unions drain
    auto load_off = [&](uint64_t ww, uint64_t& lo, uint64_t& hi) {
        uint64_t x = (nwords - 1 - ww) * 32 + lane;
        lo = hi = 0;
        if (ww < nwords && x < s.n) {
            lo = off[x];
            hi = off[x + 1];
        }
    };
    auto load_cols = [&](uint64_t lo, uint64_t hi, uint32_t* c) {
#pragma unroll
        for (int j = 0; j < HB_WARP_N; ++j) c[j] = (j < N && hi > lo + (uint64_t)j) ? cols[lo + j] : GC_DINF;
    };
    uint64_t w = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    uint64_t lo0, hi0, lo1, hi1;
    uint32_t c[HB_WARP_N];
    load_off(w, lo0, hi0);
    load_off(w + nwarps, lo1, hi1);
    load_cols(lo0, hi0, c);
    for (; w < nwords; w += nwarps) {
        uint32_t cn[HB_WARP_N];
        uint64_t lo2, hi2;
        load_cols(lo1, hi1, cn);
        load_off(w + 2 * nwarps, lo2, hi2);
        uint64_t v = (nwords - 1 - w) * 32 + lane;
        bool root = hi0 > lo0 && !(c[0] < (uint32_t)v);   // not hooked in step 1
        unsigned total = 0;
#pragma unroll
        for (int j = 0; j < HB_WARP_N; ++j) {
            if (c[j] != GC_DINF && c[j] >= s.n) atomicOr(s.err, GC_DERR_RANGE);
            bool want = root && c[j] < s.n && c[j] != (uint32_t)v;
            unsigned m = __ballot_sync(0xFFFFFFFFu, want);
            if (want) my[total + __popc(m & lt)] = KoutJob{(uint32_t)v, c[j], (uint32_t)(lo0 + j)};
            total += __popc(m);
        }
        __syncwarp();
        for (unsigned j = lane; j < total; j += 32) {
            KoutJob jb = my[j];
            union_or_defer<L, F, S, SF>(s, dq, jb.u, jb.v, jb.eid);
        }
        __syncwarp();
        lo0 = lo1; hi0 = hi1;
#pragma unroll
        for (int j = 0; j < HB_WARP_N; ++j) c[j] = cn[j];
        lo1 = lo2; hi1 = hi2;
    }
}

// HB sampling step 2: every vertex that is still a root after step 1 unions
// its first N edges.  "Still a root after step 1" is read from the row (no
// smaller neighbour), not from P, which step-2 unions change concurrently.
template <int L, int F, int S, bool SF, class OffT = uint64_t>
static __global__ void __launch_bounds__(256) k_hb2(const OffT* __restrict__ off, const uint32_t* __restrict__ cols,
                                             int N, UFState s) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < s.n; v += stride) {
        uint64_t lo = off[v], hi = off[v + 1];
        if (hi > lo && cols[lo] < (uint32_t)v) continue;   // hooked in step 1
        uint64_t end = lo + (uint64_t)N < hi ? lo + (uint64_t)N : hi;
        for (uint64_t a = lo; a < end; ++a) {
            uint32_t w = cols[a];
            if (w >= s.n) { atomicOr(s.err, GC_DERR_RANGE); continue; }
            if (w == (uint32_t)v) continue;
            Spin sp(s.cap);
            uf_union<L, F, S, SF>(s, (uint32_t)v, w, (uint32_t)a, sp);
        }
    }
}

// Full compression (the FullShortcut fixpoint): every vertex points straight
// at its root.  Roots do not move during this kernel, so one walk per vertex
// reaches the fixpoint of repeated pointer jumping.
template <int L>
static __global__ void k_compress(UFState s) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < s.n; v += stride) {
        uint32_t r = uf_root<L, true>(s, (uint32_t)v);
        if (L == LK_JTB) {
            u64w w = ldw(s.W, (uint32_t)v);
            if (wpar(w) != r) s.W[v] = wmake(wrank(w), r);
        } else {
            if (ldp(s.P, (uint32_t)v) != r) stp(s.P, (uint32_t)v, r);
        }
    }
}

// Union-JTB after a min-linking step (HB step 1, BFS): the trees are flat
// (parent = root), so roots get rank 1 and everything else rank 0, which keeps
// every parent's key above its children's.
static __global__ void k_w_from_p(uint32_t n, const uint32_t* P, u64w* W) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t p = P[v];
        W[v] = wmake(p == (uint32_t)v ? 1u : 0u, p);
    }
}


// Vertex v's nch warp tasks from slot `base` of the task array (reserved by
// the caller).  Slots at or above task_cap do not exist: a vertex whose tasks
// do not all fit goes to the overflow list instead, and the slots it reserved
// below the cap get empty tasks (a chunk index past every row's end), since
// the readers take every slot below min(count, cap) as a task.
__device__ __forceinline__ void put_tasks(uint64_t v, uint64_t nch, uint64_t base, unsigned long long* tasks,
                                          uint32_t task_cap, uint32_t* over, uint32_t* nover) {
    const bool fits = base + nch <= task_cap;
    const unsigned long long tag = (unsigned long long)v << 32;
    for (uint64_t j = 0; j < nch && base + j < task_cap; ++j)
        tasks[base + j] = tag | (fits ? j : 0xFFFFFFFFull);
    if (!fits) over[atomicAdd(nover, 1u)] = (uint32_t)v;
}

// Vertex gathering (the VG optimisation): vertices whose sampled label is not
// L_max and that have edges become active.  Low-degree ones go to a list
// (thread per vertex); higher-degree ones are cut into TASK_ARCS-arc warp
// tasks.  A vertex whose tasks do not fit the task array goes to the overflow
// list (one block per vertex).  With `active` non-null one bit per vertex
// records the active set for the arc filter of the finish kernels.
template <int L, bool COMPRESS = false, class OffT = uint64_t>
static __global__ void __launch_bounds__(256) k_vg(const OffT* __restrict__ off, UFState s, const uint32_t* lmax_p,
                                            uint32_t* active, uint32_t* small, uint32_t* nsmall,
                                            unsigned long long* tasks, uint32_t task_cap, uint32_t* ntasks,
                                            uint32_t* over, uint32_t* nover) {
    pdl_entry();
    uint32_t lmax = lmax_p ? *lmax_p : GC_DINF;
    uint64_t nwords = ((uint64_t)s.n + 31) / 32;
    uint64_t wstride = (uint64_t)gridDim.x * (blockDim.x / 32);
    unsigned lane = lane_id();
    for (uint64_t w = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < nwords; w += wstride) {
        uint64_t v = w * 32 + lane;
        bool act = false;
        uint64_t deg = 0;
        if (v < s.n) {
            deg = off[v + 1] - off[v];
            uint32_t lab;
            if (COMPRESS) {                 // full compression fused in: P[v] = root(v)
                lab = uf_root<L, true>(s, (uint32_t)v);
                if (L == LK_JTB) {
                    u64w w = ldw(s.W, (uint32_t)v);
                    if (wpar(w) != lab) s.W[v] = wmake(wrank(w), lab);
                } else if (ldp(s.P, (uint32_t)v) != lab) {
                    stp(s.P, (uint32_t)v, lab);
                }
            } else {
                lab = (L == LK_JTB) ? wpar(ldw(s.W, (uint32_t)v)) : ldp(s.P, (uint32_t)v);
            }
            act = deg > 0 && lab != lmax;
        }
        unsigned am = __ballot_sync(0xFFFFFFFFu, act);
        if (active && lane == 0) active[w] = am;
        bool is_small = act && deg <= (uint64_t)SMALL_DEG;
        unsigned sm = __ballot_sync(0xFFFFFFFFu, is_small);
        if (sm) {
            unsigned leader = __ffs(sm) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(nsmall, (uint32_t)__popc(sm));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (is_small) small[base + __popc(sm & ((1u << lane) - 1))] = (uint32_t)v;
        }
        if (act && !is_small) {
            uint64_t nch = (deg + TASK_ARCS - 1) / TASK_ARCS;
            uint32_t base = atomicAdd(ntasks, (uint32_t)nch);
            put_tasks(v, nch, base, tasks, task_cap, over, nover);
        }
    }
}

// Four consecutive CSR offsets from one 16-byte aligned address.
template <class OffT>
__device__ __forceinline__ void load_off4(const OffT* p, uint64_t o[4]) {
    if constexpr (sizeof(OffT) == 4) {
        uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
    } else {
        ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2*>(p));
        ulonglong2 b = __ldg(reinterpret_cast<const ulonglong2*>(p) + 1);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
}

// The body of k_vg4 over this grid's share of the 128-vertex groups (also
// a phase of the fused tail kernel).  Parent loads may use L1 (L1P): no
// union runs while it does, so a stale line holds an older ancestor and the
// walks still end at the current roots.
template <int L, class OffT, bool L1P>
__device__ __forceinline__ void vg4_pass(const OffT* __restrict__ off, const UFState& s, uint32_t lmax,
                                         uint32_t* active, uint32_t* small, uint32_t* nsmall,
                                         unsigned long long* tasks, uint32_t task_cap, uint32_t* ntasks,
                                         uint32_t* over, uint32_t* nover) {
    const uint64_t n = s.n;
    const uint64_t nwords = (n + 31) / 32;
    const uint64_t ngroups = (n + 127) / 128;
    const unsigned lane = lane_id();
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t gi = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; gi < ngroups; gi += nw) {
        const uint64_t v0 = gi * 128 + 4 * (uint64_t)lane;
        const bool full = v0 + 4 <= n;
        uint32_t p[4];
        uint64_t o[5];
        if (full) {
            uint4 pp = L1P ? __ldca(reinterpret_cast<const uint4*>(s.P + v0))
                           : __ldcg(reinterpret_cast<const uint4*>(s.P + v0));
            load_off4(off + v0, o);
            p[0] = pp.x; p[1] = pp.y; p[2] = pp.z; p[3] = pp.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                bool in = v0 + j < n;
                p[j] = in ? ldq<L1P>(s.P, (uint32_t)(v0 + j)) : 0u;   // vertex 0 is its own root
                o[j] = v0 + j <= n ? (uint64_t)off[v0 + j] : 0;       // off[n] ends the last row
            }
        }
        uint64_t nx = __shfl_down_sync(0xFFFFFFFFu, o[0], 1);   // next lane's off[v0 + 4]
        if (lane == 31 || v0 + 4 >= n) nx = v0 + 4 <= n ? (uint64_t)off[v0 + 4] : 0;
        o[4] = nx;
        uint32_t cur[4], nxt[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            cur[j] = p[j];
            nxt[j] = cur[j] < s.n ? ldq<L1P>(s.P, cur[j]) : cur[j];
        }
        for (uint32_t step = 0; step <= s.n; ++step) {
            bool any = false;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (nxt[j] != cur[j]) {
                    cur[j] = nxt[j];
                    any = true;
                }
            }
            if (!any) break;
#pragma unroll
            for (int j = 0; j < 4; ++j) nxt[j] = cur[j] < s.n ? ldq<L1P>(s.P, cur[j]) : cur[j];
            if (step == s.n) atomicOr(s.err, GC_DERR_NONCONV);
        }
        // P[v] = root(v)
        bool changed = cur[0] != p[0] || cur[1] != p[1] || cur[2] != p[2] || cur[3] != p[3];
        if (changed) {
            if (full) {
                __stcg(reinterpret_cast<uint4*>(s.P + v0), make_uint4(cur[0], cur[1], cur[2], cur[3]));
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (v0 + j < n && cur[j] != p[j]) stp(s.P, (uint32_t)(v0 + j), cur[j]);
            }
        }
        unsigned nib = 0, snib = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint64_t deg = o[j + 1] - o[j];
            bool act = v0 + j < n && deg > 0 && cur[j] != lmax;
            nib |= (unsigned)act << j;
            snib |= (unsigned)(act && deg <= (uint64_t)SMALL_DEG) << j;
        }
        if (active) {   // lane l holds bits 4(l % 8) .. 4(l % 8) + 3 of word 4 gi + l / 8
            unsigned x = nib << (4 * (lane & 7));
            x |= __shfl_xor_sync(0xFFFFFFFFu, x, 1);
            x |= __shfl_xor_sync(0xFFFFFFFFu, x, 2);
            x |= __shfl_xor_sync(0xFFFFFFFFu, x, 4);
            uint64_t word = gi * 4 + lane / 8;
            if ((lane & 7) == 0 && word < nwords) active[word] = x;
        }
        if (__any_sync(0xFFFFFFFFu, nib != 0)) {
            unsigned c = __popc(snib), inc = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                unsigned t = __shfl_up_sync(0xFFFFFFFFu, inc, d);
                if ((int)lane >= d) inc += t;
            }
            unsigned total = __shfl_sync(0xFFFFFFFFu, inc, 31);
            uint32_t base = 0;
            if (lane == 31 && total) base = atomicAdd(nsmall, total);
            base = __shfl_sync(0xFFFFFFFFu, base, 31) + (inc - c);
            // the warp's higher-degree vertices reserve their tasks together:
            // one atomic per warp, not one per vertex (without sampling most
            // of a graph's vertices are here)
            uint32_t tc = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (((nib & ~snib) >> j) & 1u) tc += (uint32_t)((o[j + 1] - o[j] + TASK_ARCS - 1) / TASK_ARCS);
            uint32_t tinc = tc;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                uint32_t t = __shfl_up_sync(0xFFFFFFFFu, tinc, d);
                if ((int)lane >= d) tinc += t;
            }
            const uint32_t ttotal = __shfl_sync(0xFFFFFFFFu, tinc, 31);
            uint32_t tbase = 0;
            if (lane == 31 && ttotal) tbase = atomicAdd(ntasks, ttotal);
            uint64_t tb = (uint64_t)__shfl_sync(0xFFFFFFFFu, tbase, 31) + (tinc - tc);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if ((snib >> j) & 1u) small[base++] = (uint32_t)(v0 + j);
                if (((nib & ~snib) >> j) & 1u) {
                    uint64_t nch = (o[j + 1] - o[j] + TASK_ARCS - 1) / TASK_ARCS;
                    put_tasks(v0 + j, nch, tb, tasks, task_cap, over, nover);
                    tb += nch;
                }
            }
        }
    }
}

// Vertex gathering with full compression for the min-linking rules, written
// for few instructions per vertex: a warp takes 128 consecutive vertices, each
// lane 4 of them, with one 16-byte parent load and 16 bytes (uint32 offsets)
// or 32 bytes (uint64) of offsets (the fifth offset is the next lane's first).
// The lane's 4 root walks run in lock step, changed parents go back in one
// 16-byte store, and the 4 active bits of each lane are merged into the
// bitmask words by three shuffles.  The list appends (rare after sampling)
// run only in warps that have active vertices.  Needs 16-byte aligned offsets
// and parents; others use k_vg.
template <int L, class OffT = uint64_t>
static __global__ void __launch_bounds__(256) k_vg4(const OffT* __restrict__ off, UFState s,
                                                    const uint32_t* lmax_p, uint32_t* active, uint32_t* small,
                                                    uint32_t* nsmall, unsigned long long* tasks, uint32_t task_cap,
                                                    uint32_t* ntasks, uint32_t* over, uint32_t* nover) {
    pdl_entry();
    const uint32_t lmax = lmax_p ? *lmax_p : GC_DINF;
    vg4_pass<L, OffT, true>(off, s, lmax, active, small, nsmall, tasks, task_cap, ntasks, over, nover);
}

// COH: the bitmask was written by other blocks of the same kernel, so it is
// read through L2 instead of the read-only path.
template <bool COH = false>
__device__ __forceinline__ bool arc_needed(const uint32_t* active, uint32_t u, uint32_t v) {
    // each undirected edge is processed once: from its larger endpoint when
    // both are active, from the active one when the other was skipped
    if (v < u) return true;
    if (!active) return false;
    uint32_t w = COH ? __ldcg(active + (v >> 5)) : __ldg(active + (v >> 5));
    return ((w >> (v & 31)) & 1u) == 0;
}

template <int L, int F, int S, bool SF, class OffT = uint64_t>
static __global__ void __launch_bounds__(256) k_finish_small(const OffT* __restrict__ off,
                                                      const uint32_t* __restrict__ cols, UFState s,
                                                      const uint32_t* active, const uint32_t* small,
                                                      const uint32_t* nsmall) {
    uint32_t cnt = *nsmall;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t it = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
        if ((++it & 63u) == 0 && err_abort(s.err)) return;
        uint32_t u = small[i];
        uint64_t lo = off[u], hi = off[u + 1];
        for (uint64_t a = lo; a < hi; ++a) {
            uint32_t v = cols[a];
            if (v >= s.n) { atomicOr(s.err, GC_DERR_RANGE); continue; }
            if (!arc_needed(active, u, v)) continue;
            Spin sp(s.cap);
            uf_union<L, F, S, SF>(s, u, v, (uint32_t)a, sp);
        }
    }
}

template <int L, int F, int S, bool SF, class OffT = uint64_t>
static __global__ void __launch_bounds__(256) k_finish_tasks(const OffT* __restrict__ off,
                                                      const uint32_t* __restrict__ cols, UFState s,
                                                      const uint32_t* active, const unsigned long long* tasks,
                                                      const uint32_t* ntasks, uint32_t task_cap) {
    uint32_t cnt = *ntasks;
    if (cnt > task_cap) cnt = task_cap;
    uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    unsigned lane = lane_id();
    for (uint64_t t = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; t < cnt; t += nw) {
        if (err_abort(s.err)) return;
        unsigned long long task = tasks[t];
        uint32_t u = (uint32_t)(task >> 32);
        uint64_t lo = off[u] + (task & 0xFFFFFFFFull) * TASK_ARCS, hi = off[u + 1];
        if (lo + TASK_ARCS < hi) hi = lo + TASK_ARCS;
        for (uint64_t a = lo + lane; a < hi; a += 32) {
            uint32_t v = cols[a];
            if (v >= s.n) { atomicOr(s.err, GC_DERR_RANGE); continue; }
            if (!arc_needed(active, u, v)) continue;
            Spin sp(s.cap);
            uf_union<L, F, S, SF>(s, u, v, (uint32_t)a, sp);
        }
    }
}

// The whole finish phase over this grid: 256-arc warp tasks first, then the
// low-degree list (thread per vertex), then overflow vertices (warp per
// vertex striding over all its arcs).  ct / cs / co are the task, low-degree
// and overflow counts; COH reads the lists and the bitmask through L2 (they
// were written earlier in the same kernel by other blocks).
template <int L, int F, int S, bool SF, class OffT, bool COH>
__device__ __forceinline__ void finish_pass(const OffT* __restrict__ off, const uint32_t* __restrict__ cols,
                                            const UFState& s, const uint32_t* active, const uint32_t* small,
                                            uint32_t cs, const unsigned long long* tasks, uint32_t ct,
                                            const uint32_t* over, uint32_t co) {
    uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    uint64_t gw = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    unsigned lane = lane_id();
    for (uint64_t t = gw; t < ct; t += nw) {
        if (err_abort(s.err)) return;
        unsigned long long task = COH ? __ldcg(tasks + t) : tasks[t];
        uint32_t u = (uint32_t)(task >> 32);
        uint64_t lo = (uint64_t)off[u] + (task & 0xFFFFFFFFull) * TASK_ARCS, hi = off[u + 1];
        if (lo + TASK_ARCS < hi) hi = lo + TASK_ARCS;
        for (uint64_t a = lo + lane; a < hi; a += 32) {
            uint32_t v = cols[a];
            if (v >= s.n) { atomicOr(s.err, GC_DERR_RANGE); continue; }
            if (!arc_needed<COH>(active, u, v)) continue;
            Spin sp(s.cap);
            uf_union<L, F, S, SF>(s, u, v, (uint32_t)a, sp);
        }
    }
    // low-degree vertices, flattened per warp: G listed vertices' arcs form one
    // range [0, total) that the lanes cover densely (owner lane found by a
    // shuffle binary search over the inclusive degree scan).  G is sized to the
    // list: a short list (the usual case after sampling) is spread one vertex
    // per warp, so no warp walks several rows' unions in sequence; a long one
    // packs up to 32 vertices per warp.
    uint64_t G = ((uint64_t)cs + nw - 1) / nw;
    G = G < 1 ? 1 : G > 32 ? 32 : G;
    for (uint64_t base = gw * G; base < cs; base += nw * G) {
        if (err_abort(s.err)) return;
        uint64_t i = base + lane;
        uint32_t u = 0, d = 0;
        uint64_t lo = 0;
        if (lane < G && i < cs) {
            u = COH ? __ldcg(small + i) : small[i];
            lo = off[u];
            d = (uint32_t)(off[u + 1] - lo);
        }
        uint32_t inc = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if ((int)lane >= o) inc += t;
        }
        uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
        uint32_t exc = inc - d;
        for (uint32_t jb = 0; jb < total; jb += 32) {
            uint32_t j = jb + lane;
            int l0 = 0, l1 = 31;                       // first lane whose inclusive sum exceeds j
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                int mid = (l0 + l1) >> 1;
                uint32_t vm = __shfl_sync(0xFFFFFFFFu, inc, mid);
                if (vm > j) l1 = mid; else l0 = mid + 1;
            }
            uint32_t ou = __shfl_sync(0xFFFFFFFFu, u, l0);
            uint64_t olo = __shfl_sync(0xFFFFFFFFu, lo, l0);
            uint32_t oex = __shfl_sync(0xFFFFFFFFu, exc, l0);
            if (j >= total) continue;
            uint64_t a = olo + (j - oex);
            uint32_t v = cols[a];
            if (v >= s.n) { atomicOr(s.err, GC_DERR_RANGE); continue; }
            if (!arc_needed<COH>(active, ou, v)) continue;
            Spin sp(s.cap);
            uf_union<L, F, S, SF>(s, ou, v, (uint32_t)a, sp);
        }
    }
    for (uint64_t i = gw; i < co; i += nw) {
        uint32_t u = COH ? __ldcg(over + i) : over[i];
        for (uint64_t a = (uint64_t)off[u] + lane; a < off[u + 1]; a += 32) {
            uint32_t v = cols[a];
            if (v >= s.n) { atomicOr(s.err, GC_DERR_RANGE); continue; }
            if (!arc_needed<COH>(active, u, v)) continue;
            Spin sp(s.cap);
            uf_union<L, F, S, SF>(s, u, v, (uint32_t)a, sp);
        }
    }
}

template <int L, int F, int S, bool SF, class OffT = uint64_t>
__global__ void __launch_bounds__(256) k_finish(const OffT* __restrict__ off, const uint32_t* __restrict__ cols,
                                               UFState s, const uint32_t* active, const uint32_t* small,
                                               const uint32_t* nsmall, const unsigned long long* tasks,
                                               const uint32_t* ntasks, uint32_t task_cap, const uint32_t* over,
                                               const uint32_t* nover) {
    pdl_entry();
    uint32_t ct = *ntasks;
    if (ct > task_cap) ct = task_cap;
    finish_pass<L, F, S, SF, OffT, false>(off, cols, s, active, small, *nsmall, tasks, ct, over, *nover);
}

// Finish without vertex gathering (measurement form, GCONN_ABL_NO_VG): one
// thread per vertex; a vertex whose parent is L_max (after the full
// compression) is skipped, any other unions its whole row in sequence.  Each
// undirected edge between two processed vertices is unioned from both sides.
// Skipping stays exact: a vertex seen with parent L_max is in L_max's tree,
// membership never ends, so an edge skipped from both ends joins two vertices
// already connected.
template <int L, int F, int S, bool SF, class OffT = uint64_t>
static __global__ void __launch_bounds__(256) k_finish_plain(const OffT* __restrict__ off,
                                                             const uint32_t* __restrict__ cols, UFState s,
                                                             const uint32_t* lmax_p) {
    pdl_entry();
    uint32_t lmax = lmax_p ? *lmax_p : GC_DINF;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < s.n; v += stride) {
        if (ldp(s.P, (uint32_t)v) == lmax) continue;
        for (uint64_t a = off[v]; a < off[v + 1]; ++a) {
            uint32_t u = cols[a];
            if (u >= s.n) { atomicOr(s.err, GC_DERR_RANGE); continue; }
            if (u == (uint32_t)v) continue;
            Spin sp(s.cap);
            uf_union<L, F, S, SF>(s, (uint32_t)v, u, (uint32_t)a, sp);
        }
    }
}

// Overflow vertices: one block strides over all arcs of one vertex.
template <int L, int F, int S, bool SF, class OffT = uint64_t>
static __global__ void __launch_bounds__(256) k_finish_over(const OffT* __restrict__ off,
                                                     const uint32_t* __restrict__ cols, UFState s,
                                                     const uint32_t* active, const uint32_t* over,
                                                     const uint32_t* nover) {
    uint64_t cnt = *nover;
    for (uint64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
        uint32_t u = over[i];
        for (uint64_t a = off[u] + threadIdx.x; a < off[u + 1]; a += blockDim.x) {
            uint32_t v = cols[a];
            if (v >= s.n) { atomicOr(s.err, GC_DERR_RANGE); continue; }
            if (!arc_needed(active, u, v)) continue;
            Spin sp(s.cap);
            uf_union<L, F, S, SF>(s, u, v, (uint32_t)a, sp);
        }
    }
}

// LabelFinalization (Algorithm 1): labels[v] = root(v).  With min-linking the
// root is the smallest id of its tree, i.e. already canonical.
// When labels is the parent array, each thread takes four consecutive vertices
// with one 16-byte load; the four walks advance in lock step (four parent loads in
// flight), and the four labels are written back only when one changed (after
// the vertex-gathering pass most vertices already point at their root).
template <bool L1 = true>
__device__ __forceinline__ void finalize_all(const UFState& s, uint32_t* labels) {
    constexpr int W = 4;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool vec = labels == s.P && ((uintptr_t)labels & 15u) == 0;
    uint64_t nv = vec ? s.n / 4 : 0;
    for (uint64_t q = t0; q < nv; q += stride) {
        uint4 p4 = __ldcg(reinterpret_cast<const uint4*>(s.P) + q);
        uint32_t cur[W] = {p4.x, p4.y, p4.z, p4.w}, nxt[W];
#pragma unroll
        for (int j = 0; j < W; ++j) nxt[j] = ldq<L1>(s.P, cur[j]);
        for (uint32_t step = 0; step <= s.n; ++step) {
            bool any = false;
#pragma unroll
            for (int j = 0; j < W; ++j) {
                if (nxt[j] != cur[j]) {
                    cur[j] = nxt[j];
                    any = true;
                }
            }
            if (!any) break;
#pragma unroll
            for (int j = 0; j < W; ++j) nxt[j] = ldq<L1>(s.P, cur[j]);
            if (step == s.n) atomicOr(s.err, GC_DERR_NONCONV);
        }
        if (cur[0] != p4.x || cur[1] != p4.y || cur[2] != p4.z || cur[3] != p4.w)
            reinterpret_cast<uint4*>(labels)[q] = make_uint4(cur[0], cur[1], cur[2], cur[3]);
    }
    for (uint64_t v = nv * 4 + t0; v < s.n; v += stride) labels[v] = uf_root<LK_ASYNC, L1>(s, (uint32_t)v);
}

static __global__ void k_finalize(UFState s, uint32_t* labels) {
    pdl_entry();
    finalize_all(s, labels);
}

// LabelFinalization in place after vertex gathering.  Gathering left every
// vertex pointing at its sampled root, and a root moves in the finish only
// when a union links it: the roots of active components (whose vertices all
// have edges and a label other than L_max, so all of them are in the gathered
// lists) or the L_max root itself.  So while P[L_max] is still L_max, walking
// the listed vertices to their roots finalises every label; otherwise (or
// without an L_max) every vertex is walked.  L1: parent loads may use L1
// (not when this grid's own earlier phase linked roots).
template <bool L1>
__device__ __forceinline__ void finalize_gathered_pass(const UFState& s, uint32_t lmax, const uint32_t* small,
                                                       uint64_t cs, const unsigned long long* tasks, uint64_t ct,
                                                       const uint32_t* over, uint64_t co) {
    if (lmax >= s.n || ldp(s.P, lmax) != lmax) {
        finalize_all<L1>(s, s.P);
        return;
    }
    uint64_t total = cs + ct + co;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        uint32_t u = i < cs ? __ldcg(small + i) : i < cs + ct ? (uint32_t)(__ldcg(tasks + (i - cs)) >> 32)
                                                              : __ldcg(over + (i - cs - ct));
        uint32_t r = uf_root<LK_ASYNC, L1>(s, u);
        if (ldp(s.P, u) != r) stp(s.P, u, r);
    }
}

static __global__ void k_finalize_gathered(UFState s, const uint32_t* lmax_p, const uint32_t* small,
                                           const uint32_t* nsmall, const unsigned long long* tasks,
                                           const uint32_t* ntasks, uint32_t task_cap, const uint32_t* over,
                                           const uint32_t* nover) {
    pdl_entry();
    uint32_t lmax = lmax_p ? *lmax_p : GC_DINF;
    uint64_t ct = *ntasks;
    if (ct > task_cap) ct = task_cap;
    finalize_gathered_pass<true>(s, lmax, small, *nsmall, tasks, ct, over, *nover);
}

// ------------------------------------------------------------ grid barrier
// A barrier over every block of a cooperative launch (all blocks resident).
// Arrivals are counted in two levels so they do not serialise on one word:
// block b arrives at group b % G (G <= GRID_GROUPS counters); the last
// arrival of a group arrives at the top counter, and the last of those
// publishes the generation that the other blocks' thread 0 poll for.  The
// counters only grow (64-bit, zeroed before the launch): a block's own
// arrival count tells it which barrier it is at, so no word is reset and no
// block reads the generation before arriving.  The arrivals are acquire-
// release atomics and the publication a release store, so the writes of
// every block before the barrier are visible to every block after it.  Every
// word has a 128-byte line of its own, so the polling does not slow the
// arrivals.  The wait is bounded: it ends when the device error word shows
// that a block gave up, or after GRID_WAIT_NS, when it raises that error
// itself -- then every block returns instead of waiting forever.
constexpr int GRID_GROUPS = 32;
struct GridBar {
    uint32_t gen, pad0[31];
    unsigned long long top, pad1[15];
    unsigned long long group[GRID_GROUPS][16];
};
constexpr unsigned long long GRID_WAIT_NS = 20ull * 1000000000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu(unsigned long long* p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

static __device__ __noinline__ bool grid_sync(GridBar* b, uint32_t* err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        const uint32_t nb = gridDim.x;
        const uint32_t G = nb < GRID_GROUPS ? nb : GRID_GROUPS;
        const uint32_t grp = blockIdx.x % G;
        const uint32_t gsize = nb / G + (grp < nb % G ? 1u : 0u);
        // releases this block's writes (ordered before by the block barrier)
        const unsigned long long old = atom_add_acq_rel_gpu(&b->group[grp][0], 1ull);
        const uint32_t target = (uint32_t)(old / gsize) + 1u;   // the generation this barrier publishes
        bool last = false;
        if (old % gsize == gsize - 1) {     // the group's last arrival: acquires the group, releases it on
            const unsigned long long top = atom_add_acq_rel_gpu(&b->top, 1ull);
            last = top % G == G - 1;
        }
        if (last) {
            st_release_gpu(&b->gen, target);
        } else {
            unsigned long long t0 = globaltimer_ns();
            unsigned ns = 32;
            while ((int32_t)(ld_acquire_gpu(&b->gen) - target) < 0) {
                if (__ldcg(err) & GC_DERR_NONCONV) { good = 0; break; }
                if (globaltimer_ns() - t0 > GRID_WAIT_NS) {
                    atomicOr(err, GC_DERR_NONCONV);
                    good = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 128) ns *= 2;
            }
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// Union-JTB roots are not minimal: canonicalise through the root.
static __global__ void k_fill(uint32_t n, uint32_t* a, uint32_t val) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) a[v] = val;
}

static __global__ void k_jtb_min(UFState s, uint32_t* labels) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < s.n; v += stride)
        atomicMin(labels + wpar(ldw(s.W, (uint32_t)v)), (uint32_t)v);
}

static __global__ void k_jtb_gather(UFState s, uint32_t* labels) {
    // W is flat here; a root's own slot already holds its component minimum
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < s.n; v += stride) {
        uint32_t r = wpar(ldw(s.W, (uint32_t)v));
        if (r != (uint32_t)v) labels[v] = __ldcg(labels + r);
    }
}

// Spanning forest output: compact the recorded slots into a dense id list.
static __global__ void __launch_bounds__(256) k_sf_compact(uint32_t n, const uint32_t* sf, unsigned long long* out,
                                                            unsigned long long* count) {
    // Each block owns a contiguous range of 32-vertex words and reserves its
    // output slots with ONE atomic: pass 1 counts (ballots), pass 2 re-reads
    // the same words in the same order and writes (one counter shared by
    // thousands of per-warp atomics would serialise at its L2 slice).
    __shared__ unsigned long long wsum[8];
    __shared__ unsigned long long base;
    const uint64_t nwords = ((uint64_t)n + 31) / 32;
    const uint64_t per = (nwords + gridDim.x - 1) / gridDim.x;
    const uint64_t w0 = (uint64_t)blockIdx.x * per;
    const uint64_t w1 = w0 + per < nwords ? w0 + per : nwords;
    const unsigned lane = lane_id(), warp = threadIdx.x / 32, nwarp = blockDim.x / 32;
    unsigned long long mine = 0;
    for (uint64_t w = w0 + warp; w < w1; w += nwarp) {
        uint64_t v = w * 32 + lane;
        bool has = v < n && sf[v] != GC_DINF;
        mine += __popc(__ballot_sync(0xFFFFFFFFu, has));
    }
    if (lane == 0) wsum[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (unsigned i = 0; i < nwarp; ++i) {
            unsigned long long c = wsum[i];
            wsum[i] = tot;                 // exclusive prefix over the warps
            tot += c;
        }
        base = tot ? atomicAdd(count, tot) : 0;
    }
    __syncthreads();
    unsigned long long pos = base + wsum[warp];
    for (uint64_t w = w0 + warp; w < w1; w += nwarp) {
        uint64_t v = w * 32 + lane;
        uint32_t id = v < n ? sf[v] : GC_DINF;
        bool has = id != GC_DINF;
        unsigned m = __ballot_sync(0xFFFFFFFFu, has);
        if (has) out[pos + __popc(m & ((1u << lane) - 1))] = id;
        pos += __popc(m);
    }
}

// offsets[n] must fit a 32-bit forest id.
template <class OffT = uint64_t>
static __global__ void k_check_arcs(const OffT* off, uint32_t n, uint32_t* err) {
    if ((uint64_t)off[n] >= 0xFFFFFFFFull) atomicOr(err, GC_DERR_OVERFLOW);
}

}  // namespace gc
