// gconn_plan.cu -- static connected components captured once into a CUDA
// graph and replayed: the whole pass of Algorithm 1 (init, sampling, L_max,
// vertex gathering, finish, finalisation) becomes one graph launch, so the
// device runs its kernels back to back without a host launch per kernel.
// Every variant can be captured: BFS sampling and the round-based finishes
// loop over their levels / rounds on the device.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gc_internal.h"
#include "gc_static.h"

using namespace gc;

struct gconn_plan {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ProfSink sink;
};

namespace {

template <class Body>
gconn_status capture_plan(Body&& body, gconn_plan** out) {
    if (!err_word()) return GCONN_E_CUDA;   // resolved before any capture
    gconn_plan* p = new gconn_plan();
    cudaGetDevice(&p->device);
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        delete p;
        return GCONN_E_CUDA;
    }
    gconn_status s = GCONN_OK;
    prof_set_sink(&p->sink);
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        s = GCONN_E_CUDA;
    } else {
        gconn_status b = body(cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap, &g);
        p->graph = g;
        if (b != GCONN_OK) s = b;
        else if (e != cudaSuccess) s = GCONN_E_CUDA;
    }
    prof_set_sink(nullptr);
    if (s == GCONN_OK && cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) s = GCONN_E_CUDA;
    cudaStreamDestroy(cap);
    if (s != GCONN_OK) {
        cudaGetLastError();
        gconn_plan_destroy(p);
        return s;
    }
    *out = p;
    return GCONN_OK;
}

gconn_status plan_variant_ok(const gconn_variant* vin, int input_kind, int want_forest = 0) {
    Variant v;
    return resolve_variant(vin, input_kind, want_forest, &v);
}

// offsets[n] of a device CSR, read before the capture starts.
template <class OffT>
gconn_status csr_arcs(uint32_t n, const OffT* offsets, uint64_t* out) {
    OffT last = 0;
    GC_CUDA(cudaMemcpy(&last, offsets + n, sizeof(OffT), cudaMemcpyDeviceToHost));
    *out = last;
    return GCONN_OK;
}

}  // namespace

extern "C" gconn_status gconn_plan_create_cc(uint32_t n, uint64_t m, const uint32_t* edges, uint32_t* labels,
                                             const gconn_variant* v, gconn_plan** out) {
    if (!out) return GCONN_E_INVAL;
    *out = nullptr;
    if (!labels || !is_device_ptr(labels) || (m && (!edges || !is_device_ptr(edges)))) return GCONN_E_INVAL;
    GC_TRY(plan_variant_ok(v, 0));
    return capture_plan([&](cudaStream_t st) { return gconn_cc(n, m, edges, labels, v, st); }, out);
}

extern "C" gconn_status gconn_plan_create_cc_csr(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                                                 uint32_t* labels, const gconn_variant* v, gconn_plan** out) {
    if (!out) return GCONN_E_INVAL;
    *out = nullptr;
    if (!offsets || !cols || !labels || !is_device_ptr(offsets) || !is_device_ptr(cols) || !is_device_ptr(labels))
        return GCONN_E_INVAL;
    GC_TRY(plan_variant_ok(v, 1));
    uint64_t arcs = 0;
    GC_TRY(csr_arcs<uint64_t>(n, offsets, &arcs));
    CsrArcsHint hint(arcs);
    return capture_plan([&](cudaStream_t st) { return gconn_cc_csr(n, offsets, cols, labels, v, st); }, out);
}

extern "C" gconn_status gconn_plan_create_forest_csr(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                                                     uint64_t* forest, uint64_t* forest_count, uint32_t* labels,
                                                     const gconn_variant* v, gconn_plan** out) {
    if (!out) return GCONN_E_INVAL;
    *out = nullptr;
    if (!offsets || !cols || !forest || !forest_count || !is_device_ptr(offsets) || !is_device_ptr(cols) ||
        !is_device_ptr(forest) || !is_device_ptr(forest_count) || (labels && !is_device_ptr(labels)))
        return GCONN_E_INVAL;
    GC_TRY(plan_variant_ok(v, 1, 1));
    uint64_t arcs = 0;
    GC_TRY(csr_arcs<uint64_t>(n, offsets, &arcs));
    CsrArcsHint hint(arcs);
    return capture_plan([&](cudaStream_t st) {
        return gconn_spanning_forest_csr(n, offsets, cols, forest, forest_count, labels, v, st);
    }, out);
}

extern "C" gconn_status gconn_plan_create_cc_csr32(uint32_t n, const uint32_t* offsets, const uint32_t* cols,
                                                   uint32_t* labels, const gconn_variant* v, gconn_plan** out) {
    if (!out) return GCONN_E_INVAL;
    *out = nullptr;
    if (!offsets || !cols || !labels || !is_device_ptr(offsets) || !is_device_ptr(cols) || !is_device_ptr(labels))
        return GCONN_E_INVAL;
    GC_TRY(plan_variant_ok(v, 1));
    uint64_t arcs = 0;
    GC_TRY(csr_arcs<uint32_t>(n, offsets, &arcs));
    CsrArcsHint hint(arcs);
    return capture_plan([&](cudaStream_t st) { return gconn_cc_csr32(n, offsets, cols, labels, v, st); }, out);
}

extern "C" gconn_status gconn_plan_create_forest_csr32(uint32_t n, const uint32_t* offsets, const uint32_t* cols,
                                                       uint64_t* forest, uint64_t* forest_count, uint32_t* labels,
                                                       const gconn_variant* v, gconn_plan** out) {
    if (!out) return GCONN_E_INVAL;
    *out = nullptr;
    if (!offsets || !cols || !forest || !forest_count || !is_device_ptr(offsets) || !is_device_ptr(cols) ||
        !is_device_ptr(forest) || !is_device_ptr(forest_count) || (labels && !is_device_ptr(labels)))
        return GCONN_E_INVAL;
    GC_TRY(plan_variant_ok(v, 1, 1));
    uint64_t arcs = 0;
    GC_TRY(csr_arcs<uint32_t>(n, offsets, &arcs));
    CsrArcsHint hint(arcs);
    return capture_plan([&](cudaStream_t st) {
        return gconn_spanning_forest_csr32(n, offsets, cols, forest, forest_count, labels, v, st);
    }, out);
}

extern "C" gconn_status gconn_plan_run(gconn_plan* p, void* stream) {
    if (!p || !p->exec) return GCONN_E_INVAL;
    g_launches.fetch_add(p->sink.launches, std::memory_order_relaxed);
    GC_CUDA(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
    if (!p->sink.recs.empty()) prof_requeue(p->sink);
    return GCONN_OK;
}

extern "C" gconn_status gconn_plan_destroy(gconn_plan* p) {
    if (!p) return GCONN_E_INVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    prof_release(p->sink);
    cudaSetDevice(prev);
    delete p;
    return GCONN_OK;
}
