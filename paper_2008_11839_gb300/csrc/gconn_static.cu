// gconn_static.cu -- host orchestration of static connectivity and spanning
// forest (Algorithms 1 and 2) over COO and CSR input.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string.h>

#include "csr_impl.cuh"
#include "gc_internal.h"
#include "gc_static.h"
#include "static_kernels.cuh"

namespace gc {

// Map the public variant onto the instantiated triple.
void uf_triple(const Variant& v, int* L, int* F, int* S) {
    *L = v.link;
    int f = v.find;
    if (v.link == GCONN_LINK_ECLCC) {   // ECL-CC's finish: Union-Async with path splitting
        *L = LK_ASYNC;
        f = GCONN_FIND_SPLIT;
    }
    if (f == GCONN_FIND_FULLSHORTCUT) f = GCONN_FIND_NAIVE;
    *F = f == GCONN_FIND_COMPRESS ? FD_COMPRESS
       : f == GCONN_FIND_SPLIT ? FD_SPLIT
       : f == GCONN_FIND_HALVE ? FD_HALVE
       : f == GCONN_FIND_TWOTRYSPLIT ? FD_TWOTRY : FD_NAIVE;
    *S = SP_NONE;
    if (v.link == GCONN_LINK_REMCAS || v.link == GCONN_LINK_REMLOCK)
        *S = v.splice == GCONN_SPLICE_SPLIT_ONE ? SP_SPLIT_ONE
           : v.splice == GCONN_SPLICE_HALVE_ONE ? SP_HALVE_ONE : SP_SPLICE;
}

UFState make_state(uint32_t n, uint32_t* P, uint32_t* H, u64w* W, uint32_t* sf, const Variant& v) {
    UFState s;
    s.P = P; s.H = H; s.W = W; s.sf = sf;
    s.Lk = nullptr;
    s.err = err_word_lookup();
    s.n = n;
    s.cap = v.cap;
    s.seed = (uint32_t)(v.seed ^ (v.seed >> 32));
    return s;
}

gconn_status init_state(const UFState& s, cudaStream_t st, uint32_t* zero, uint32_t nzero) {
    if (s.n == 0) return GCONN_OK;
    return launch_pdl("init", k_init, grid_for(k_init, 256, s.n), 256, 0, st, s.n, s.P, s.H, s.W, s.sf, zero, nzero);
}

gconn_status union_coo(const Variant& v, const UFState& s, const uint32_t* edges, uint64_t m,
                       uint32_t eid_base, cudaStream_t st) {
    if (m == 0) return GCONN_OK;
    int L, F, S;
    uf_triple(v, &L, &F, &S);
    int B = block_of(v);
    return dispatch_uf(L, F, S, s.sf != nullptr, [&]<int l, int f, int sp, bool sf>() {
        auto k = k_union_coo<l, f, sp, sf>;
        // at most about one thread per vertex: beyond that, concurrent unions
        // on a small vertex set mostly contend for the same few roots (ER
        // n = 65,536, m = 2^20, Rem-CAS + splice: 0.140 ms with the full
        // grid, 0.097 ms with a quarter of it, 0.116 ms with an eighth)
        uint64_t gr = grid_for(k, B, m);
        const uint64_t cap = std::max<uint64_t>((uint64_t)num_sms(), ((uint64_t)s.n + B - 1) / B);
        return launch("union_coo", k, (unsigned)std::min(gr, cap), B, 0, st, (const uint2*)edges, m, s, eid_base);
    });
}

gconn_status compress_all(const Variant& v, const UFState& s, cudaStream_t st) {
    if (s.n == 0) return GCONN_OK;
    if (v.link == GCONN_LINK_JTB)
        return launch("compress", k_compress<LK_JTB>, grid_for(k_compress<LK_JTB>, 256, s.n), 256, 0, st, s);
    return launch("compress", k_compress<LK_ASYNC>, grid_for(k_compress<LK_ASYNC>, 256, s.n), 256, 0, st, s);
}

gconn_status finalize_labels(const Variant& v, const UFState& s, uint32_t* labels, cudaStream_t st) {
    if (s.n == 0) return GCONN_OK;
    unsigned g = grid_for(k_finalize, 256, s.n);
    if (v.link != GCONN_LINK_JTB) {
        // labels may alias P: the walk then compresses in place
        return launch_pdl("finalize", k_finalize, g, 256, 0, st, s, labels);
    }
    GC_TRY(compress_all(v, s, st));
    GC_TRY(launch("jtb_fill", k_fill, g, 256, 0, st, s.n, labels, INF));
    GC_TRY(launch("jtb_min", k_jtb_min, g, 256, 0, st, s, labels));
    return launch("jtb_gather", k_jtb_gather, g, 256, 0, st, s, labels);
}

gconn_status sf_output(uint32_t n, const uint32_t* sf, uint64_t* forest, uint64_t* count, cudaStream_t st) {
    bool forest_dev = is_device_ptr(forest), count_dev = is_device_ptr(count);
    DevBuf fbuf, cbuf;
    unsigned long long* f = (unsigned long long*)forest;
    unsigned long long* c = (unsigned long long*)count;
    if (!forest_dev) { GC_TRY(fbuf.alloc(sizeof(uint64_t) * (size_t)(n ? n : 1), st)); f = fbuf.as<unsigned long long>(); }
    if (!count_dev) { GC_TRY(cbuf.alloc(sizeof(uint64_t), st)); c = cbuf.as<unsigned long long>(); }
    GC_CUDA(cudaMemsetAsync(c, 0, sizeof(uint64_t), st));
    if (n) GC_TRY(launch("sf_compact", k_sf_compact, grid_for(k_sf_compact, 256, n), 256, 0, st, n, sf, f, c));
    if (!forest_dev || !count_dev) {
        uint64_t hc = 0;
        GC_CUDA(cudaMemcpyAsync(&hc, c, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        GC_CUDA(cudaStreamSynchronize(st));
        if (!count_dev) *count = hc;
        if (!forest_dev && hc)
            GC_CUDA(cudaMemcpyAsync(forest, f, sizeof(uint64_t) * hc, cudaMemcpyDeviceToHost, st));
    }
    return GCONN_OK;
}

}  // namespace gc

using namespace gc;

extern "C" gconn_status gconn_cc(uint32_t n, uint64_t m, const uint32_t* edges, uint32_t* labels,
                                 const gconn_variant* v, void* stream) {
    return static_run<uint64_t>(n, m, edges, nullptr, nullptr, labels, nullptr, nullptr, v, 0, stream);
}

extern "C" gconn_status gconn_cc_csr(uint32_t n, const uint64_t* offsets, const uint32_t* cols, uint32_t* labels,
                                     const gconn_variant* v, void* stream) {
    if (!offsets) return GCONN_E_INVAL;
    return static_run<uint64_t>(n, 0, nullptr, offsets, cols, labels, nullptr, nullptr, v, 0, stream);
}

extern "C" gconn_status gconn_cc_csr_stats(uint32_t n, const uint64_t* offsets, const uint32_t* cols, uint32_t* labels,
                                           const gconn_variant* vin, gconn_sample_stats* out, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!out || !offsets || !labels || n == 0 || n == 0xFFFFFFFFu) return GCONN_E_INVAL;
    if (!is_device_ptr(offsets) || !is_device_ptr(labels) || (cols && !is_device_ptr(cols))) return GCONN_E_INVAL;
    Variant v;
    GC_TRY(resolve_variant(vin, 1, 0, &v));
    if (v.link == GCONN_LINK_JTB || is_rounds_link(v.link)) return GCONN_E_UNSUPPORTED;
    memset(out, 0, sizeof(*out));
    DevBuf cb, hbuf, lkbuf;
    GC_TRY(cb.alloc(9 * sizeof(unsigned long long), st));
    GC_CUDA(cudaMemsetAsync(cb.p, 0, 9 * sizeof(unsigned long long), st));
    uint32_t* H = nullptr;
    if (v.link == GCONN_LINK_HOOKS) { GC_TRY(hbuf.alloc(sizeof(uint32_t) * (size_t)n, st)); H = hbuf.as<uint32_t>(); }
    UFState s = make_state(n, labels, H, nullptr, nullptr, v);
    if (v.link == GCONN_LINK_REMLOCK) {
        GC_TRY(lkbuf.alloc(sizeof(uint32_t) * (size_t)n, st));
        s.Lk = lkbuf.as<uint32_t>();
        GC_CUDA(cudaMemsetAsync(s.Lk, 0, sizeof(uint32_t) * (size_t)n, st));
    }
    cudaEvent_t e0, e1, e1b, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e1b);
    cudaEventCreate(&e2);
    CsrStats cs{cb.as<unsigned long long>(), e1, e1b, (uint32_t*)(cb.as<unsigned long long>() + 8)};
    GC_CUDA(cudaEventRecord(e0, st));
    bool finalized = false;
    gconn_status r = csr_connect<uint64_t>(v, s, offsets, cols, st, &cs, &finalized);
    if (r == GCONN_OK && !finalized) r = finalize_labels(v, s, labels, st);
    if (r == GCONN_OK) r = cuda_status(cudaEventRecord(e2, st));
    unsigned long long h[8] = {0};
    if (r == GCONN_OK) r = cuda_status(cudaMemcpyAsync(h, cb.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    if (r == GCONN_OK) r = read_and_clear_err(st);
    float ms_total = 0, ms_sample = 0, ms_rest = 0;
    if (r == GCONN_OK) {
        cudaEventElapsedTime(&ms_sample, e0, e1);
        cudaEventElapsedTime(&ms_rest, e1b, e2);
        ms_total = ms_sample + ms_rest;
        uint64_t narcs = 0;
        cudaMemcpy(&narcs, offsets + n, sizeof(uint64_t), cudaMemcpyDeviceToHost);
        out->n = n;
        out->arcs = narcs;
        out->lmax_vertices = h[0];
        out->sampled_components = h[1];
        out->active_vertices = h[2];
        out->active_arcs = h[3];
        out->inter_component_arcs = h[4];
        out->sample_arcs_inspected = h[5];
        uint32_t lm = GC_DINF;
        if (v.sample != GCONN_SAMPLE_NONE) cudaMemcpy(&lm, cs.lmax, sizeof(uint32_t), cudaMemcpyDeviceToHost);
        out->lmax = lm;
        out->sample_ms = ms_sample;
        out->total_ms = ms_total;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e1b);
    cudaEventDestroy(e2);
    return r;
}

extern "C" gconn_status gconn_spanning_forest(uint32_t n, uint64_t m, const uint32_t* edges, uint64_t* forest,
                                              uint64_t* forest_count, uint32_t* labels, const gconn_variant* v,
                                              void* stream) {
    return static_run<uint64_t>(n, m, edges, nullptr, nullptr, labels, forest, forest_count, v, 1, stream);
}

extern "C" gconn_status gconn_spanning_forest_csr(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                                                  uint64_t* forest, uint64_t* forest_count, uint32_t* labels,
                                                  const gconn_variant* v, void* stream) {
    if (!offsets) return GCONN_E_INVAL;
    return static_run<uint64_t>(n, 0, nullptr, offsets, cols, labels, forest, forest_count, v, 1, stream);
}
