// gconn_inc.cu -- incremental connectivity (Section 3.5, Algorithm 3): a
// device-resident union-find that absorbs batches of edge insertions and
// answers batches of connectivity queries.  Old batches are never re-read:
// every finish algorithm allowed here is root-based, so the forest alone
// carries the connectivity of everything inserted so far.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gc_internal.h"
#include "gc_static.h"
#include "static_kernels.cuh"

using namespace gc;

struct gconn_inc {
    uint32_t n;
    int device;
    Variant v;
    uint32_t* P;
    uint32_t* H;
    u64w* W;
    uint32_t* Lk;
    cudaStream_t last;
    uint64_t inspected_last, inspected_total;   // edge inspections of the inserts (Section 4.4)
};

namespace gc {

// Query batch: find both endpoints (with the handle's find rule, which may
// compress) and compare the roots.
template <int L, int F>
__global__ void __launch_bounds__(256) k_query(const uint2* __restrict__ Q, uint64_t q, UFState s, uint8_t* out) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < q; i += stride) {
        uint2 e = __ldcs(Q + i);
        if (e.x >= s.n || e.y >= s.n) {
            atomicOr(s.err, GC_DERR_RANGE);
            out[i] = 0;
            continue;
        }
        Spin sp(s.cap);
        uint32_t a, b;
        if (L == LK_JTB) {
            a = jtb_find<F>(s, e.x, sp);
            b = jtb_find<F>(s, e.y, sp);
        } else if (F == FD_NAIVE) {
            out[i] = same_root_lockstep(s, e.x, e.y, sp) ? 1 : 0;
            continue;
        } else {
            a = uf_find<F, true>(s, e.x, sp);   // no link happens during a query batch
            b = uf_find<F, true>(s, e.y, sp);
        }
        out[i] = (a == b) ? 1 : 0;
    }
}

// Mixed batch (Algorithm 3): op i is an insert or a query; a warp covers 32
// consecutive ops and writes one 32-bit word of the answer bitvector.
// PHASE: 0 = inserts and queries together, 1 = inserts only, 2 = queries only.
template <int L, int F, int S, int PHASE>
__global__ void __launch_bounds__(256) k_mixed(const uint2* __restrict__ E, const uint8_t* __restrict__ isq,
                                               uint64_t b, UFState s, uint32_t* bits) {
    uint64_t nwords = (b + 31) / 32;
    uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    unsigned lane = threadIdx.x & 31u;
    for (uint64_t w = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w < nwords; w += nw) {
        uint64_t i = w * 32 + lane;
        bool ans = false;
        if (i < b) {
            uint2 e = __ldcs(E + i);
            bool q = isq[i] != 0;
            if (e.x >= s.n || e.y >= s.n) {
                atomicOr(s.err, GC_DERR_RANGE);
            } else if (!q && PHASE != 2) {
                if (e.x != e.y) {
                    Spin sp(s.cap);
                    uf_union<L, F, S, false>(s, e.x, e.y, 0, sp);
                }
            } else if (q && PHASE != 1) {
                Spin sp(s.cap);
                ans = same_set<L, F>(s, e.x, e.y, sp);
            }
        }
        unsigned word = __ballot_sync(0xFFFFFFFFu, ans);
        if (PHASE != 1 && lane == 0) bits[w] = word;
    }
}

template <int L, int F>
static gconn_status launch_query(const UFState& s, const uint2* Q, uint64_t q, uint8_t* out, int block,
                                 cudaStream_t st) {
    auto k = k_query<L, F>;
    return launch("query", k, grid_for(k, block, q), block, 0, st, Q, q, s, out);
}

static gconn_status query_dispatch(const Variant& v, const UFState& s, const uint2* Q, uint64_t q, uint8_t* out,
                                   cudaStream_t st) {
    int L, F, S;
    if (v.link == GCONN_LINK_SV || v.link == GCONN_LINK_LT) {
        L = LK_ASYNC;
        F = FD_NAIVE;
    } else {
        uf_triple(v, &L, &F, &S);
    }
    int B = v.block > 0 ? v.block : 256;
    if (L == LK_JTB) return F == FD_TWOTRY ? launch_query<LK_JTB, FD_TWOTRY>(s, Q, q, out, B, st)
                                           : launch_query<LK_JTB, FD_NAIVE>(s, Q, q, out, B, st);
    switch (F) {
        case FD_COMPRESS: return launch_query<LK_ASYNC, FD_COMPRESS>(s, Q, q, out, B, st);
        case FD_SPLIT: return launch_query<LK_ASYNC, FD_SPLIT>(s, Q, q, out, B, st);
        case FD_HALVE: return launch_query<LK_ASYNC, FD_HALVE>(s, Q, q, out, B, st);
        default: return launch_query<LK_ASYNC, FD_NAIVE>(s, Q, q, out, B, st);
    }
}

template <class Fn>
static gconn_status dispatch_inc(int L, int F, int S, Fn&& fn) {
#define GC_IN_CASE(l, f, s) \
    if (L == l && F == f && S == s) return fn.template operator()<l, f, s>();
    GC_IN_CASE(LK_ASYNC, FD_NAIVE, SP_NONE)
    GC_IN_CASE(LK_ASYNC, FD_COMPRESS, SP_NONE)
    GC_IN_CASE(LK_ASYNC, FD_SPLIT, SP_NONE)
    GC_IN_CASE(LK_ASYNC, FD_HALVE, SP_NONE)
    GC_IN_CASE(LK_HOOKS, FD_NAIVE, SP_NONE)
    GC_IN_CASE(LK_HOOKS, FD_COMPRESS, SP_NONE)
    GC_IN_CASE(LK_HOOKS, FD_SPLIT, SP_NONE)
    GC_IN_CASE(LK_HOOKS, FD_HALVE, SP_NONE)
    GC_IN_CASE(LK_EARLY, FD_NAIVE, SP_NONE)
    GC_IN_CASE(LK_EARLY, FD_COMPRESS, SP_NONE)
    GC_IN_CASE(LK_EARLY, FD_SPLIT, SP_NONE)
    GC_IN_CASE(LK_EARLY, FD_HALVE, SP_NONE)
    GC_IN_CASE(LK_REMCAS, FD_NAIVE, SP_SPLIT_ONE)
    GC_IN_CASE(LK_REMCAS, FD_NAIVE, SP_HALVE_ONE)
    GC_IN_CASE(LK_REMCAS, FD_NAIVE, SP_SPLICE)
    GC_IN_CASE(LK_REMCAS, FD_SPLIT, SP_SPLIT_ONE)
    GC_IN_CASE(LK_REMCAS, FD_SPLIT, SP_HALVE_ONE)
    GC_IN_CASE(LK_REMCAS, FD_SPLIT, SP_SPLICE)
    GC_IN_CASE(LK_REMCAS, FD_HALVE, SP_SPLIT_ONE)
    GC_IN_CASE(LK_REMCAS, FD_HALVE, SP_HALVE_ONE)
    GC_IN_CASE(LK_REMCAS, FD_HALVE, SP_SPLICE)
    GC_IN_CASE(LK_REMLOCK, FD_NAIVE, SP_SPLIT_ONE)
    GC_IN_CASE(LK_REMLOCK, FD_NAIVE, SP_HALVE_ONE)
    GC_IN_CASE(LK_REMLOCK, FD_NAIVE, SP_SPLICE)
    GC_IN_CASE(LK_REMLOCK, FD_SPLIT, SP_SPLIT_ONE)
    GC_IN_CASE(LK_REMLOCK, FD_SPLIT, SP_HALVE_ONE)
    GC_IN_CASE(LK_REMLOCK, FD_SPLIT, SP_SPLICE)
    GC_IN_CASE(LK_REMLOCK, FD_HALVE, SP_SPLIT_ONE)
    GC_IN_CASE(LK_REMLOCK, FD_HALVE, SP_HALVE_ONE)
    GC_IN_CASE(LK_REMLOCK, FD_HALVE, SP_SPLICE)
    GC_IN_CASE(LK_AFFOREST, FD_NAIVE, SP_NONE)
    GC_IN_CASE(LK_JTB, FD_NAIVE, SP_NONE)
    GC_IN_CASE(LK_JTB, FD_TWOTRY, SP_NONE)
#undef GC_IN_CASE
    return GCONN_E_UNSUPPORTED;
}

static UFState handle_state(gconn_inc* h) {
    UFState s = make_state(h->n, h->P, h->H, h->W, nullptr, h->v);
    s.Lk = h->Lk;
    return s;
}

bool inc_view(const gconn_inc* h, IncView* out) {
    if (!h || !out) return false;
    out->n = h->n;
    out->P = h->P;
    out->H = h->H;
    out->W = h->W;
    out->v = h->v;
    return true;
}

}  // namespace gc

extern "C" gconn_status gconn_inc_create(uint32_t n, const gconn_variant* vin, void* stream, gconn_inc** out) {
    if (!out || n == 0xFFFFFFFFu) return GCONN_E_INVAL;
    *out = nullptr;
    gconn_variant d;
    gconn_variant_default(&d);
    if (vin) d = *vin;
    else d.sample = GCONN_SAMPLE_NONE;
    if (d.sample != GCONN_SAMPLE_NONE) return GCONN_E_UNSUPPORTED;   // batches are COO
    Variant v;
    GC_TRY(resolve_variant(&d, 0, 2, &v));
    cudaStream_t st = (cudaStream_t)stream;
    gconn_inc* h = new gconn_inc();
    h->n = n;
    h->v = v;
    h->last = st;
    cudaGetDevice(&h->device);
    size_t cnt = n ? n : 1;
    cudaError_t e = cudaMalloc(&h->P, sizeof(uint32_t) * cnt);
    if (e == cudaSuccess && v.link == GCONN_LINK_HOOKS) e = cudaMalloc(&h->H, sizeof(uint32_t) * cnt);
    if (e == cudaSuccess && v.link == GCONN_LINK_JTB) e = cudaMalloc(&h->W, sizeof(u64w) * cnt);
    if (e == cudaSuccess && v.link == GCONN_LINK_REMLOCK) {
        e = cudaMalloc(&h->Lk, sizeof(uint32_t) * cnt);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->Lk, 0, sizeof(uint32_t) * cnt, st);
    }
    if (e != cudaSuccess) {
        gconn_inc_destroy(h);
        return cuda_status(e);
    }
    gconn_status s = init_state(handle_state(h), st);
    if (s != GCONN_OK) {
        gconn_inc_destroy(h);
        return s;
    }
    *out = h;
    return GCONN_OK;
}

extern "C" gconn_status gconn_inc_insert_batch(gconn_inc* h, uint64_t b, const uint32_t* edges, void* stream) {
    if (!h || (b && !edges) || b > GC_MAX_COUNT || ((uintptr_t)edges & 7u)) return GCONN_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    if (b == 0) return GCONN_OK;
    if (h->n == 0) return GCONN_E_RANGE;
    DevBuf eb;
    const uint32_t* de = nullptr;
    bool host = !is_device_ptr(edges);
    // a union-find finish reads the batch once (in place from host memory
    // where the device can); the round finishes re-read it
    if (is_rounds_link(h->v.link))
        GC_TRY(stage_in(edges, sizeof(uint32_t) * 2 * b, st, eb, (const void**)&de));
    else
        GC_TRY(stage_in_once(edges, sizeof(uint32_t) * 2 * b, st, eb, (const void**)&de));
    UFState s = handle_state(h);
    uint64_t inspected = b;   // a union-find finish reads each edge of the batch once
    if (is_rounds_link(h->v.link)) {
        uint32_t passes = 0;   // rounds re-read the whole batch until the labels converge
        GC_TRY(rounds_coo(h->v, s, de, nullptr, b, st, &passes));
        inspected = (uint64_t)passes * b;
    } else {
        GC_TRY(union_coo(h->v, s, de, b, 0, st));
    }
    h->inspected_last = inspected;
    h->inspected_total += inspected;
    if (host) return read_and_clear_err(st);
    return GCONN_OK;
}

extern "C" gconn_status gconn_inc_query(gconn_inc* h, uint64_t q, const uint32_t* pairs, uint8_t* connected,
                                        void* stream) {
    if (!h || (q && (!pairs || !connected)) || q > GC_MAX_COUNT || ((uintptr_t)pairs & 7u)) return GCONN_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    if (q == 0) return GCONN_OK;
    if (h->n == 0) return GCONN_E_RANGE;
    DevBuf pb, ob;
    const uint32_t* dp = nullptr;
    bool host_in = !is_device_ptr(pairs), host_out = !is_device_ptr(connected);
    GC_TRY(stage_in_once(pairs, sizeof(uint32_t) * 2 * q, st, pb, (const void**)&dp));   // read once
    uint8_t* dout = connected;
    if (host_out) {
        GC_TRY(ob.alloc(q, st));
        dout = ob.as<uint8_t>();
    }
    GC_TRY(query_dispatch(h->v, handle_state(h), (const uint2*)dp, q, dout, st));
    if (host_out) GC_CUDA(cudaMemcpyAsync(connected, dout, q, cudaMemcpyDeviceToHost, st));
    if (host_in || host_out) return read_and_clear_err(st);
    return GCONN_OK;
}

extern "C" gconn_status gconn_inc_process_batch(gconn_inc* h, uint64_t b, const uint32_t* pairs,
                                                const uint8_t* is_query, uint32_t* result_bits, void* stream) {
    if (!h || (b && (!pairs || !is_query || !result_bits)) || b > GC_MAX_COUNT || ((uintptr_t)pairs & 7u) ||
        ((uintptr_t)result_bits & 3u))
        return GCONN_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    if (b == 0) return GCONN_OK;
    if (h->n == 0) return GCONN_E_RANGE;
    if (is_rounds_link(h->v.link)) return GCONN_E_UNSUPPORTED;   // rounds finish a whole insert batch first
    DevBuf pb, qb, ob;
    const uint32_t* dp = nullptr;
    const uint8_t* dq = nullptr;
    bool host_in = !is_device_ptr(pairs) || !is_device_ptr(is_query), host_out = !is_device_ptr(result_bits);
    GC_TRY(stage_in(pairs, sizeof(uint32_t) * 2 * b, st, pb, (const void**)&dp));
    GC_TRY(stage_in(is_query, b, st, qb, (const void**)&dq));
    uint64_t words = (b + 31) / 32;
    uint32_t* dout = result_bits;
    if (host_out) {
        GC_TRY(ob.alloc(sizeof(uint32_t) * words, st));
        dout = ob.as<uint32_t>();
    }
    int L, F, S;
    uf_triple(h->v, &L, &F, &S);
    // Rem's algorithms are correct only phase-concurrently (Section 3.5):
    // their inserts run first, then the queries
    bool split = L == LK_REMCAS || L == LK_REMLOCK;
    UFState s = handle_state(h);
    int B = h->v.block > 0 ? h->v.block : 256;
    GC_TRY(dispatch_inc(L, F, S, [&]<int l, int f, int sp>() -> gconn_status {
        if (split) {
            auto k1 = k_mixed<l, f, sp, 1>;
            GC_TRY(launch("mixed_insert", k1, grid_for(k1, B, b), B, 0, st, (const uint2*)dp, dq, b, s, dout));
            auto k2 = k_mixed<l, f, sp, 2>;
            return launch("mixed_query", k2, grid_for(k2, B, b), B, 0, st, (const uint2*)dp, dq, b, s, dout);
        }
        auto k = k_mixed<l, f, sp, 0>;
        return launch("mixed", k, grid_for(k, B, b), B, 0, st, (const uint2*)dp, dq, b, s, dout);
    }));
    h->inspected_last = b;   // every op of a mixed batch is read once
    h->inspected_total += b;
    if (host_out) GC_CUDA(cudaMemcpyAsync(result_bits, dout, sizeof(uint32_t) * words, cudaMemcpyDeviceToHost, st));
    if (host_in || host_out) return read_and_clear_err(st);
    return GCONN_OK;
}

extern "C" gconn_status gconn_inc_edges_inspected(const gconn_inc* h, uint64_t* last_batch, uint64_t* total) {
    if (!h || !last_batch || !total) return GCONN_E_INVAL;
    *last_batch = h->inspected_last;
    *total = h->inspected_total;
    return GCONN_OK;
}

extern "C" gconn_status gconn_inc_labels(gconn_inc* h, uint32_t* labels, void* stream) {
    if (!h || (h->n && !labels)) return GCONN_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    h->last = st;
    if (h->n == 0) return GCONN_OK;
    bool host = !is_device_ptr(labels);
    DevBuf lb;
    uint32_t* dl = labels;
    if (host) {
        GC_TRY(lb.alloc(sizeof(uint32_t) * (size_t)h->n, st));
        dl = lb.as<uint32_t>();
    }
    Variant fv = h->v;
    if (fv.link == GCONN_LINK_SV || fv.link == GCONN_LINK_LT) fv.link = GCONN_LINK_ASYNC;
    GC_TRY(finalize_labels(fv, handle_state(h), dl, st));
    if (host) {
        GC_CUDA(cudaMemcpyAsync(labels, dl, sizeof(uint32_t) * (size_t)h->n, cudaMemcpyDeviceToHost, st));
        return read_and_clear_err(st);
    }
    return GCONN_OK;
}

extern "C" gconn_status gconn_inc_destroy(gconn_inc* h) {
    if (!h) return GCONN_E_INVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->last);
    if (h->P) cudaFree(h->P);
    if (h->H) cudaFree(h->H);
    if (h->W) cudaFree(h->W);
    if (h->Lk) cudaFree(h->Lk);
    cudaSetDevice(prev);
    delete h;
    return GCONN_OK;
}
