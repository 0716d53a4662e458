// gconn_batched.cu -- many independent graphs in one persistent launch.
//
// Each graph of the batch is one task for one CTA: its whole union-find lives
// in shared memory, as 32-bit parents where the class's largest graph fits a
// CTA's 227 KiB that way (n <= 58,112), else as 16-bit parents (a graph of up
// to 65,536 vertices needs at most 128 KiB); its edges stream once from HBM,
// and its labels are written once.  Graphs are grouped into size classes; every class runs one
// persistent kernel (CTAs pull graphs from an atomic queue, largest first) on
// its own forked stream, so the classes share the GPU, and the whole sequence
// is captured into one CUDA graph at plan creation.  Block size and union rule
// per class come from a tune table (gconn_batch_autotune measures it).
// Graphs above the last class use the global-memory COO path, one launch
// each.  The per-graph method is the paper's finish phase without sampling
// (Algorithm 1 on COO input), so labels are min-id per graph.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "gc_internal.h"
#include "gc_static.h"
#include "uf_device.cuh"

namespace gc {

constexpr int NCLS = GCONN_BATCH_CLASSES;
constexpr uint32_t SMEM_MAX_N = 65536;
constexpr uint32_t SMEM_CAP = 1u << 20;   // loop cap per shared-memory union

enum { BR_ASYNC_NAIVE = 0, BR_ASYNC_HALVE = 1, BR_REM_SPLIT = 2 };
constexpr int BATCH_ILP = 8;   // edge loads in flight per thread

template <class T>
__device__ __forceinline__ uint32_t sm_ld(const volatile T* P, uint32_t i) { return P[i]; }
__device__ __forceinline__ uint32_t sm_cas(volatile uint16_t* P, uint32_t i, uint32_t cmp, uint32_t val) {
    return atomicCAS((unsigned short*)(P + i), (unsigned short)cmp, (unsigned short)val);
}
__device__ __forceinline__ uint32_t sm_cas(volatile uint32_t* P, uint32_t i, uint32_t cmp, uint32_t val) {
    return atomicCAS((unsigned int*)(P + i), cmp, val);
}

template <int R, class T>
__device__ __forceinline__ uint32_t sm_find(volatile T* P, uint32_t u, uint32_t& left) {
    if constexpr (R == BR_ASYNC_HALVE) {
        while (left) {
            uint32_t v = sm_ld(P, u), w = sm_ld(P, v);
            if (v == w) return v;
            uint32_t old = sm_cas(P, u, v, w);
            u = old == v ? w : old;
            --left;
        }
        return u;
    } else {
        while (left) {
            uint32_t p = sm_ld(P, u);
            if (p == u) return u;
            u = p;
            --left;
        }
        return u;
    }
}

// One union in shared memory: Union-Async (naive or halving find) or
// Union-Rem-CAS with SplitAtomicOne (Algorithms 7, 11).
template <int R, class T>
__device__ __forceinline__ void sm_union(volatile T* P, uint32_t u, uint32_t v, uint32_t* err) {
    uint32_t left = SMEM_CAP;
    if (R == BR_REM_SPLIT) {
        uint32_t ru = u, rv = v;
        while (left--) {
            uint32_t pu = sm_ld(P, ru), pv = sm_ld(P, rv);
            if (pu == pv) return;
            if (pu < pv) {
                uint32_t t = ru; ru = rv; rv = t;
                t = pu; pu = pv; pv = t;
            }
            if (ru == pu && sm_cas(P, ru, ru, pv) == ru) return;
            uint32_t a = sm_ld(P, ru), b = sm_ld(P, a);
            if (a != b) sm_cas(P, ru, a, b);
            ru = a;
        }
        atomicOr(err, GC_DERR_NONCONV);
        return;
    }
    uint32_t pu = sm_find<R, T>(P, u, left), pv = sm_find<R, T>(P, v, left);
    while (pu != pv && left) {
        if (pu < pv) { uint32_t t = pu; pu = pv; pv = t; }
        if (sm_ld(P, pu) == pu && sm_cas(P, pu, pu, pv) == pu) return;
        --left;
        pu = sm_find<R, T>(P, pu, left);
        pv = sm_find<R, T>(P, pv, left);
    }
    if (!left) atomicOr(err, GC_DERR_NONCONV);
}

// Persistent class kernel: CTAs pull graph indices (largest first) from an
// atomic queue; each graph: init parents in shared memory, stream its edges,
// union, then write every vertex's root (its min-id label) to global memory.
template <int R, class T>
__global__ void k_batch_smem(const uint64_t* __restrict__ vo, const uint64_t* __restrict__ eo,
                             const uint2* __restrict__ E, uint32_t* __restrict__ labels,
                             const uint32_t* __restrict__ order, uint32_t count, uint32_t* queue, uint32_t* err) {
    extern __shared__ uint32_t Psm_raw[];
    volatile T* P = reinterpret_cast<volatile T*>(Psm_raw);
    __shared__ uint32_t s_idx;
    while (true) {
        if (threadIdx.x == 0) s_idx = atomicAdd(queue, 1u);
        __syncthreads();
        uint32_t idx = s_idx;
        if (idx >= count) break;
        uint32_t g = order[idx];
        uint64_t vb = vo[g];
        uint32_t n = (uint32_t)(vo[g + 1] - vb);
        uint64_t eb = eo[g], m = eo[g + 1] - eb;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) P[i] = (T)i;
        __syncthreads();
        // BATCH_ILP coalesced edge loads in flight per thread before their
        // unions: the edge stream, not the shared-memory unions, is the
        // latency that bounds a large graph's CTA
        auto one = [&](uint2 e) {
            if (e.x >= n || e.y >= n) atomicOr(err, GC_DERR_RANGE);
            else if (e.x != e.y) sm_union<R, T>(P, e.x, e.y, err);
        };
        const uint64_t B = blockDim.x;
        uint64_t j = threadIdx.x;
        for (; j + (BATCH_ILP - 1) * B < m; j += BATCH_ILP * B) {
            uint2 e[BATCH_ILP];
#pragma unroll
            for (int q = 0; q < BATCH_ILP; ++q) e[q] = __ldcs(E + eb + j + q * B);
#pragma unroll
            for (int q = 0; q < BATCH_ILP; ++q) one(e[q]);
        }
        for (; j < m; j += B) one(__ldcs(E + eb + j));
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            uint32_t r = i, left = SMEM_CAP;
            while (left--) {
                uint32_t p = sm_ld(P, r);
                if (p == r) break;
                r = p;
            }
            labels[vb + i] = r;
        }
        __syncthreads();
    }
}

}  // namespace gc

using namespace gc;

struct gconn_batch {
    int device;
    uint32_t G;
    gconn_batch_tune tune;
    // device copies of the offsets owned by the plan when the caller passed host arrays
    uint64_t* own_vo = nullptr;
    uint64_t* own_eo = nullptr;
    const uint64_t* vo = nullptr;
    const uint64_t* eo = nullptr;
    const uint32_t* edges = nullptr;
    uint32_t* labels = nullptr;
    uint32_t* order = nullptr;      // per class, concatenated
    uint32_t* queues = nullptr;     // one counter per class
    uint32_t cls_begin[NCLS + 1];
    uint32_t cls_maxn[NCLS];
    std::vector<uint32_t> large;    // graphs above the last class
    std::vector<uint64_t> hvo, heo;
    cudaStream_t side[NCLS] = {};
    cudaEvent_t fork = nullptr, join[NCLS] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ProfSink sink;                  // kernels and profiling events captured in the graph
};

namespace gc {

static int rule_of(int link, int find) {
    if (link == GCONN_LINK_REMCAS) return BR_REM_SPLIT;
    return find == GCONN_FIND_HALVE ? BR_ASYNC_HALVE : BR_ASYNC_NAIVE;
}

static void* smem_kernel(int rule, bool wide) {
    if (wide) {
        if (rule == BR_REM_SPLIT) return (void*)k_batch_smem<BR_REM_SPLIT, uint32_t>;
        if (rule == BR_ASYNC_HALVE) return (void*)k_batch_smem<BR_ASYNC_HALVE, uint32_t>;
        return (void*)k_batch_smem<BR_ASYNC_NAIVE, uint32_t>;
    }
    if (rule == BR_REM_SPLIT) return (void*)k_batch_smem<BR_REM_SPLIT, uint16_t>;
    if (rule == BR_ASYNC_HALVE) return (void*)k_batch_smem<BR_ASYNC_HALVE, uint16_t>;
    return (void*)k_batch_smem<BR_ASYNC_NAIVE, uint16_t>;
}

// Launch one class's persistent kernel on stream st.
static gconn_status launch_class(gconn_batch* b, int c, int block, int rule, cudaStream_t st) {
    uint32_t cnt = b->cls_begin[c + 1] - b->cls_begin[c];
    if (!cnt) return GCONN_OK;
    // 32-bit parents where a CTA's shared memory holds them (no 16-bit CAS)
    const bool wide = 4ull * b->cls_maxn[c] <= 227ull * 1024;
    size_t smem = wide ? sizeof(uint32_t) * (size_t)b->cls_maxn[c]
                       : sizeof(uint16_t) * (size_t)((b->cls_maxn[c] + 1) & ~1u);
    if (smem < 16) smem = 16;
    int per_sm = 0;
    void* kf = smem_kernel(rule, wide);
    GC_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, block, smem));
    if (per_sm < 1) return GCONN_E_UNSUPPORTED;
    uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)per_sm * num_sms(), cnt);
    const uint32_t* ord = b->order + b->cls_begin[c];
    uint32_t* q = b->queues + c;
    uint32_t* err = err_word();
    const uint2* E = (const uint2*)b->edges;
#define GC_BLAUNCH(RR, TT) \
    return launch("batch_smem", k_batch_smem<RR, TT>, grid, block, smem, st, b->vo, b->eo, E, b->labels, ord, cnt, q, err)
    if (wide) {
        if (rule == BR_REM_SPLIT) GC_BLAUNCH(BR_REM_SPLIT, uint32_t);
        if (rule == BR_ASYNC_HALVE) GC_BLAUNCH(BR_ASYNC_HALVE, uint32_t);
        GC_BLAUNCH(BR_ASYNC_NAIVE, uint32_t);
    }
    if (rule == BR_REM_SPLIT) GC_BLAUNCH(BR_REM_SPLIT, uint16_t);
    if (rule == BR_ASYNC_HALVE) GC_BLAUNCH(BR_ASYNC_HALVE, uint16_t);
    GC_BLAUNCH(BR_ASYNC_NAIVE, uint16_t);
#undef GC_BLAUNCH
}

// The whole batch on `st`: reset queues, fork one stream per class, join,
// then the graphs above the last class one by one.
static gconn_status enqueue_batch(gconn_batch* b, cudaStream_t st) {
    GC_CUDA(cudaMemsetAsync(b->queues, 0, sizeof(uint32_t) * NCLS, st));
    GC_CUDA(cudaEventRecord(b->fork, st));
    for (int c = 0; c < NCLS; ++c) {
        if (b->cls_begin[c + 1] == b->cls_begin[c]) continue;
        GC_CUDA(cudaStreamWaitEvent(b->side[c], b->fork, 0));
        GC_TRY(launch_class(b, c, b->tune.block[c], rule_of(b->tune.link[c], b->tune.find[c]), b->side[c]));
        GC_CUDA(cudaEventRecord(b->join[c], b->side[c]));
        GC_CUDA(cudaStreamWaitEvent(st, b->join[c], 0));
    }
    if (!b->large.empty()) {
        Variant v;
        gconn_variant d;
        gconn_variant_default(&d);
        d.sample = GCONN_SAMPLE_NONE;
        d.link = GCONN_LINK_REMCAS;
        d.splice = GCONN_SPLICE_SPLIT_ONE;
        GC_TRY(resolve_variant(&d, 0, 0, &v));
        for (uint32_t g : b->large) {
            uint32_t n = (uint32_t)(b->hvo[g + 1] - b->hvo[g]);
            uint64_t m = b->heo[g + 1] - b->heo[g];
            UFState s = make_state(n, b->labels + b->hvo[g], nullptr, nullptr, nullptr, v);
            GC_TRY(init_state(s, st));
            GC_TRY(union_coo(v, s, b->edges + 2 * b->heo[g], m, 0, st));
            GC_TRY(finalize_labels(v, s, s.P, st));
        }
    }
    return GCONN_OK;
}

static void batch_free(gconn_batch* b) {
    if (!b) return;
    prof_release(b->sink);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (int c = 0; c < NCLS; ++c) {
        if (b->side[c]) cudaStreamDestroy(b->side[c]);
        if (b->join[c]) cudaEventDestroy(b->join[c]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->own_vo) cudaFree(b->own_vo);
    if (b->own_eo) cudaFree(b->own_eo);
    if (b->order) cudaFree(b->order);
    if (b->queues) cudaFree(b->queues);
    delete b;
}

static gconn_status check_tune(const gconn_batch_tune* t) {
    uint32_t prev = 0;
    for (int c = 0; c < NCLS; ++c) {
        if (t->class_max_n[c] < prev || t->class_max_n[c] > SMEM_MAX_N) return GCONN_E_INVAL;
        prev = t->class_max_n[c];
        if (t->block[c] < 32 || t->block[c] > 1024 || t->block[c] % 32) return GCONN_E_INVAL;
        if (t->link[c] != GCONN_LINK_ASYNC && t->link[c] != GCONN_LINK_REMCAS) return GCONN_E_UNSUPPORTED;
        if (t->find[c] != GCONN_FIND_NAIVE && t->find[c] != GCONN_FIND_HALVE) return GCONN_E_UNSUPPORTED;
    }
    return GCONN_OK;
}

// Build the schedule (classes, largest-first order) without capturing.
static gconn_status batch_build(uint32_t G, const uint64_t* vtx_off, const uint64_t* edge_off, const uint32_t* edges,
                                uint32_t* labels, const gconn_batch_tune* tune, cudaStream_t st, gconn_batch** out) {
    if (!out) return GCONN_E_INVAL;
    *out = nullptr;
    if (!vtx_off || !edge_off) return GCONN_E_INVAL;
    gconn_batch_tune t;
    if (tune) t = *tune;
    else gconn_batch_tune_default(&t);
    GC_TRY(check_tune(&t));
    if (!err_word()) return GCONN_E_CUDA;   // resolved outside any stream capture
    gconn_batch* b = new gconn_batch();
    b->G = G;
    b->tune = t;
    cudaGetDevice(&b->device);
    b->hvo.resize((size_t)G + 1);
    b->heo.resize((size_t)G + 1);
    bool vdev = is_device_ptr(vtx_off), edev = is_device_ptr(edge_off);
    size_t ob = sizeof(uint64_t) * ((size_t)G + 1);
    auto fail = [&](gconn_status s) { batch_free(b); return s; };
    if (vdev) {
        if (cudaMemcpy(b->hvo.data(), vtx_off, ob, cudaMemcpyDeviceToHost) != cudaSuccess) return fail(GCONN_E_CUDA);
    } else {
        memcpy(b->hvo.data(), vtx_off, ob);
    }
    if (edev) {
        if (cudaMemcpy(b->heo.data(), edge_off, ob, cudaMemcpyDeviceToHost) != cudaSuccess) return fail(GCONN_E_CUDA);
    } else {
        memcpy(b->heo.data(), edge_off, ob);
    }
    for (uint32_t g = 0; g < G; ++g) {
        if (b->hvo[g + 1] < b->hvo[g] || b->heo[g + 1] < b->heo[g]) return fail(GCONN_E_INVAL);
        if (b->hvo[g + 1] - b->hvo[g] > 0xFFFFFFFEull) return fail(GCONN_E_INVAL);   // local ids are uint32
    }
    uint64_t total_n = b->hvo[G], total_m = b->heo[G];
    if (total_m - b->heo[0] > GC_MAX_COUNT) return fail(GCONN_E_INVAL);
    if ((total_m && !edges) || (total_n && !labels)) return fail(GCONN_E_INVAL);
    if (total_m && (!is_device_ptr(edges) || ((uintptr_t)edges & 7u))) return fail(GCONN_E_INVAL);
    if (total_n && !is_device_ptr(labels)) return fail(GCONN_E_INVAL);
    b->edges = edges;
    b->labels = labels;
    if (vdev) b->vo = vtx_off;
    else {
        if (cudaMalloc(&b->own_vo, ob) != cudaSuccess) return fail(GCONN_E_NOMEM);
        cudaMemcpy(b->own_vo, b->hvo.data(), ob, cudaMemcpyHostToDevice);
        b->vo = b->own_vo;
    }
    if (edev) b->eo = edge_off;
    else {
        if (cudaMalloc(&b->own_eo, ob) != cudaSuccess) return fail(GCONN_E_NOMEM);
        cudaMemcpy(b->own_eo, b->heo.data(), ob, cudaMemcpyHostToDevice);
        b->eo = b->own_eo;
    }
    // size classes, largest first inside each class
    std::vector<std::vector<uint32_t>> cls(NCLS);
    for (uint32_t g = 0; g < G; ++g) {
        uint64_t n = b->hvo[g + 1] - b->hvo[g];
        if (n == 0) continue;
        int c = 0;
        while (c < NCLS && n > t.class_max_n[c]) ++c;
        if (c == NCLS) b->large.push_back(g);
        else cls[c].push_back(g);
    }
    std::vector<uint32_t> order;
    for (int c = 0; c < NCLS; ++c) {
        std::sort(cls[c].begin(), cls[c].end(), [&](uint32_t a, uint32_t x) {
            uint64_t wa = b->heo[a + 1] - b->heo[a], wx = b->heo[x + 1] - b->heo[x];
            return wa != wx ? wa > wx : a < x;
        });
        b->cls_begin[c] = (uint32_t)order.size();
        uint32_t mx = 0;
        for (uint32_t g : cls[c]) mx = std::max<uint32_t>(mx, (uint32_t)(b->hvo[g + 1] - b->hvo[g]));
        b->cls_maxn[c] = mx;
        order.insert(order.end(), cls[c].begin(), cls[c].end());
    }
    b->cls_begin[NCLS] = (uint32_t)order.size();
    if (cudaMalloc(&b->order, sizeof(uint32_t) * std::max<size_t>(order.size(), 1)) != cudaSuccess ||
        cudaMalloc(&b->queues, sizeof(uint32_t) * NCLS) != cudaSuccess)
        return fail(GCONN_E_NOMEM);
    if (!order.empty())
        cudaMemcpy(b->order, order.data(), sizeof(uint32_t) * order.size(), cudaMemcpyHostToDevice);
    for (int c = 0; c < NCLS; ++c) {
        if (cudaStreamCreateWithFlags(&b->side[c], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming) != cudaSuccess)
            return fail(GCONN_E_CUDA);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return fail(GCONN_E_CUDA);
    (void)st;
    *out = b;
    return GCONN_OK;
}

}  // namespace gc

extern "C" gconn_status gconn_batch_tune_default(gconn_batch_tune* t) {
    if (!t) return GCONN_E_INVAL;
    const uint32_t bounds[NCLS] = {1024, 4096, 16384, 65536};
    const int32_t blocks[NCLS] = {256, 256, 512, 1024};
    for (int c = 0; c < NCLS; ++c) {
        t->class_max_n[c] = bounds[c];
        t->block[c] = blocks[c];
        t->link[c] = GCONN_LINK_REMCAS;
        t->find[c] = GCONN_FIND_NAIVE;
    }
    return GCONN_OK;
}

extern "C" gconn_status gconn_batch_create(uint32_t G, const uint64_t* vtx_off, const uint64_t* edge_off,
                                           const uint32_t* edges, uint32_t* labels, const gconn_batch_tune* tune,
                                           void* stream, gconn_batch** out) {
    cudaStream_t st = (cudaStream_t)stream;
    gconn_batch* b = nullptr;
    GC_TRY(batch_build(G, vtx_off, edge_off, edges, labels, tune, st, &b));
    // capture the launch sequence into one CUDA graph
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        batch_free(b);
        return GCONN_E_CUDA;
    }
    gconn_status s = GCONN_OK;
    prof_set_sink(&b->sink);
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) s = GCONN_E_CUDA;
    if (s == GCONN_OK) {
        gconn_status e = enqueue_batch(b, cap);
        cudaGraph_t gr = nullptr;
        cudaError_t ce = cudaStreamEndCapture(cap, &gr);
        if (e != GCONN_OK) s = e;
        else if (ce != cudaSuccess) s = GCONN_E_CUDA;
        b->graph = gr;
    }
    prof_set_sink(nullptr);
    if (s == GCONN_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) s = GCONN_E_CUDA;
    cudaStreamDestroy(cap);
    if (s != GCONN_OK) {
        cudaGetLastError();
        batch_free(b);
        return s;
    }
    *out = b;
    return GCONN_OK;
}

extern "C" gconn_status gconn_batch_run(gconn_batch* b, void* stream) {
    if (!b) return GCONN_E_INVAL;
    g_launches.fetch_add(b->sink.launches, std::memory_order_relaxed);
    GC_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    if (!b->sink.recs.empty()) prof_requeue(b->sink);
    return GCONN_OK;
}

extern "C" gconn_status gconn_batch_destroy(gconn_batch* b) {
    if (!b) return GCONN_E_INVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    batch_free(b);
    cudaSetDevice(prev);
    return GCONN_OK;
}

extern "C" gconn_status gconn_cc_batched(uint32_t G, const uint64_t* vtx_off, const uint64_t* edge_off,
                                         const uint32_t* edges, uint32_t* labels, const gconn_batch_tune* tune,
                                         void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    gconn_batch* b = nullptr;
    GC_TRY(batch_build(G, vtx_off, edge_off, edges, labels, tune, st, &b));
    gconn_status s = enqueue_batch(b, st);
    cudaStreamSynchronize(st);
    batch_free(b);
    return s;
}

// Measured tuning: for every class with graphs, time each (block, rule)
// candidate on that class alone (median of 3, CUDA events) and keep the best.
extern "C" gconn_status gconn_batch_autotune(uint32_t G, const uint64_t* vtx_off, const uint64_t* edge_off,
                                             const uint32_t* edges, uint32_t* labels, gconn_batch_tune* out,
                                             void* stream) {
    if (!out) return GCONN_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    gconn_batch_tune t;
    gconn_batch_tune_default(&t);
    gconn_batch* b = nullptr;
    GC_TRY(batch_build(G, vtx_off, edge_off, edges, labels, &t, st, &b));
    static const int blocks[] = {128, 256, 512, 1024};
    static const int rules[][2] = {{GCONN_LINK_ASYNC, GCONN_FIND_NAIVE},
                                   {GCONN_LINK_ASYNC, GCONN_FIND_HALVE},
                                   {GCONN_LINK_REMCAS, GCONN_FIND_NAIVE}};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    gconn_status s = GCONN_OK;
    for (int c = 0; c < NCLS && s == GCONN_OK; ++c) {
        if (b->cls_begin[c + 1] == b->cls_begin[c]) continue;
        float best = 1e30f;
        for (int bi = 0; bi < 4 && s == GCONN_OK; ++bi) {
            for (int ri = 0; ri < 3 && s == GCONN_OK; ++ri) {
                int rule = rule_of(rules[ri][0], rules[ri][1]);
                float ts[3];
                for (int rep = 0; rep < 3 && s == GCONN_OK; ++rep) {
                    cudaMemsetAsync(b->queues, 0, sizeof(uint32_t) * NCLS, st);
                    cudaEventRecord(e0, st);
                    s = launch_class(b, c, blocks[bi], rule, st);
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&ts[rep], e0, e1);
                }
                if (s == GCONN_E_UNSUPPORTED) {   // block does not fit this class's shared memory
                    s = GCONN_OK;
                    continue;
                }
                std::sort(ts, ts + 3);
                if (s == GCONN_OK && ts[1] < best) {
                    best = ts[1];
                    t.block[c] = blocks[bi];
                    t.link[c] = rules[ri][0];
                    t.find[c] = rules[ri][1];
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    gconn_status s2 = read_and_clear_err(st);
    batch_free(b);
    if (s != GCONN_OK) return s;
    if (s2 != GCONN_OK) return s2;
    *out = t;
    return GCONN_OK;
}
