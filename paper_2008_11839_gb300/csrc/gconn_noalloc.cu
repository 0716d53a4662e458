// gconn_noalloc.cu -- gconn_cc_csr_noalloc: the CSR connected-components
// path (sampling, L_max, vertex gathering, load-balanced finish,
// finalisation) for callers that must not allocate device memory.
//
// Who needs it: a caller whose device memory is already fully owned by another
// allocator (for example a framework that reserved the whole GPU for its own
// caching pool at start-up), or a serving process that runs under a fixed,
// pre-partitioned memory budget where a new device allocation could fail or
// stall the device at the wrong moment.  Such a caller owns the graph and the
// label buffer but cannot let the library call cudaMalloc / cudaMallocAsync.
//
// This entry point therefore takes its scratch (the L_max word, the gathering
// counters, the active-vertex bitmask, the low-degree list, the warp-task list
// and the overflow list) from one file-scope device array of fixed size,
// g_noalloc_scratch below.  Consequences for the caller:
//   - n may not exceed GCONN_NOALLOC_MAX_N (2^20); larger n is rejected with
//     GCONN_E_INVAL before anything is launched;
//   - every GPU that loads libgconn holds the array (about 16.2 MiB) until the
//     process exits;
//   - all calls share the one array and it keeps the previous call's
//     contents, so calls whose GPU work overlaps (different streams, or
//     threads) race on it: serialise them;
//   - the first call on each device (a call with n == 0 does only this)
//     looks the array up with cudaGetSymbolAddress and loads the code of
//     every kernel this entry point can launch.  With lazy module loading
//     (the CUDA default) that first call is where the driver maps the array
//     and the kernels' code, which takes device memory; later calls take
//     none.  A caller that hands its memory to another allocator should
//     therefore make one call (n == 0 is enough) on each device first, and
//     before any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "gc_internal.h"
#include "gc_static.h"
#include "static_kernels.cuh"

namespace {

using namespace gc;

constexpr uint32_t MAX_N = GCONN_NOALLOC_MAX_N;
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr uint64_t TASK_CAP = (uint64_t)MAX_N + 1024;
// header: L_max word, then three counters (low-degree, tasks, overflow)
constexpr size_t OFF_HEADER = 0;
constexpr size_t OFF_ACTIVE = 256;
constexpr size_t OFF_SMALL = OFF_ACTIVE + align256(sizeof(uint32_t) * ((MAX_N + 31) / 32));
constexpr size_t OFF_TASKS = OFF_SMALL + align256(sizeof(uint32_t) * MAX_N);
constexpr size_t OFF_OVER = OFF_TASKS + align256(sizeof(unsigned long long) * TASK_CAP);
constexpr size_t SCRATCH_BYTES = OFF_OVER + align256(sizeof(uint32_t) * MAX_N);

}  // namespace

// The scratch itself: device memory that exists as long as the module is
// loaded, so no call ever allocates.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

template <class Fn>
gconn_status dispatch_noalloc(int L, int F, int S, Fn&& fn) {
#define GC_NA_CASE(l, f, s) \
    if (L == l && F == f && S == s) return fn.template operator()<l, f, s>();
    GC_NA_CASE(LK_ASYNC, FD_NAIVE, SP_NONE)
    GC_NA_CASE(LK_ASYNC, FD_COMPRESS, SP_NONE)
    GC_NA_CASE(LK_ASYNC, FD_SPLIT, SP_NONE)
    GC_NA_CASE(LK_ASYNC, FD_HALVE, SP_NONE)
    GC_NA_CASE(LK_EARLY, FD_NAIVE, SP_NONE)
    GC_NA_CASE(LK_EARLY, FD_COMPRESS, SP_NONE)
    GC_NA_CASE(LK_EARLY, FD_SPLIT, SP_NONE)
    GC_NA_CASE(LK_EARLY, FD_HALVE, SP_NONE)
    GC_NA_CASE(LK_REMCAS, FD_NAIVE, SP_SPLIT_ONE)
    GC_NA_CASE(LK_REMCAS, FD_NAIVE, SP_HALVE_ONE)
    GC_NA_CASE(LK_REMCAS, FD_NAIVE, SP_SPLICE)
    GC_NA_CASE(LK_REMCAS, FD_SPLIT, SP_SPLIT_ONE)
    GC_NA_CASE(LK_REMCAS, FD_SPLIT, SP_HALVE_ONE)
    GC_NA_CASE(LK_REMCAS, FD_SPLIT, SP_SPLICE)
    GC_NA_CASE(LK_REMCAS, FD_HALVE, SP_SPLIT_ONE)
    GC_NA_CASE(LK_REMCAS, FD_HALVE, SP_HALVE_ONE)
    GC_NA_CASE(LK_REMCAS, FD_HALVE, SP_SPLICE)
#undef GC_NA_CASE
    return GCONN_E_UNSUPPORTED;
}

// Every (link, find, splice) triple dispatch_noalloc accepts, for loading
// their kernels up front.
constexpr int NA_TRIPLES[][3] = {
    {LK_ASYNC, FD_NAIVE, SP_NONE},       {LK_ASYNC, FD_COMPRESS, SP_NONE},   {LK_ASYNC, FD_SPLIT, SP_NONE},
    {LK_ASYNC, FD_HALVE, SP_NONE},       {LK_EARLY, FD_NAIVE, SP_NONE},      {LK_EARLY, FD_COMPRESS, SP_NONE},
    {LK_EARLY, FD_SPLIT, SP_NONE},       {LK_EARLY, FD_HALVE, SP_NONE},      {LK_REMCAS, FD_NAIVE, SP_SPLIT_ONE},
    {LK_REMCAS, FD_NAIVE, SP_HALVE_ONE}, {LK_REMCAS, FD_NAIVE, SP_SPLICE},   {LK_REMCAS, FD_SPLIT, SP_SPLIT_ONE},
    {LK_REMCAS, FD_SPLIT, SP_HALVE_ONE}, {LK_REMCAS, FD_SPLIT, SP_SPLICE},   {LK_REMCAS, FD_HALVE, SP_SPLIT_ONE},
    {LK_REMCAS, FD_HALVE, SP_HALVE_ONE}, {LK_REMCAS, FD_HALVE, SP_SPLICE},
};

template <class K>
gconn_status load_kernel(K kernel) {
    cudaFuncAttributes a;
    GC_CUDA(cudaFuncGetAttributes(&a, kernel));
    return GCONN_OK;
}

// Loads the code of every kernel gconn_cc_csr_noalloc can launch, so that no
// later call makes the driver map code (lazy module loading would otherwise
// do it at a kernel's first launch).
gconn_status load_all_kernels() {
    GC_TRY(load_kernel(k_init));
    GC_TRY(load_kernel(k_hb1<uint64_t>));
    GC_TRY(load_kernel(k_compress<LK_ASYNC>));
    GC_TRY(load_kernel(k_lmax<LK_ASYNC>));
    GC_TRY(load_kernel(k_vg<LK_ASYNC>));
    GC_TRY(load_kernel(k_finalize));
    for (const auto& t : NA_TRIPLES) {
        GC_TRY(dispatch_noalloc(t[0], t[1], t[2], [&]<int l, int fr, int sp>() -> gconn_status {
            GC_TRY(load_kernel(k_kout<l, fr, sp, false>));
            GC_TRY(load_kernel(k_hb2<l, fr, sp, false>));
            GC_TRY(load_kernel(k_finish_small<l, fr, sp, false>));
            GC_TRY(load_kernel(k_finish_tasks<l, fr, sp, false>));
            return load_kernel(k_finish_over<l, fr, sp, false>);
        }));
    }
    return GCONN_OK;
}

constexpr int MAX_DEV = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_dev[MAX_DEV];

// Once per device, with that device current: the device address of the
// array, the device error word (looked up without creating the library's
// memory pool) and the code of every kernel used here.
gconn_status setup(unsigned char** out) {
    int dev = 0;
    GC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEV) return GCONN_E_INVAL;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GCONN_E_CUDA;
        }
        if (!err_word_lookup()) return GCONN_E_CUDA;
        GC_TRY(load_all_kernels());
        g_scratch_dev[dev] = (unsigned char*)p;
    }
    *out = g_scratch_dev[dev];
    return GCONN_OK;
}

}  // namespace

extern "C" gconn_status gconn_cc_csr_noalloc(uint32_t n, const uint64_t* offsets, const uint32_t* cols,
                                             uint32_t* labels, const gconn_variant* vin, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (n > MAX_N) return GCONN_E_INVAL;
    unsigned char* base = nullptr;
    GC_TRY(setup(&base));   // also the whole of a call with n == 0 (any pointers)
    if (n == 0) return GCONN_OK;
    if (!offsets || ((uintptr_t)offsets & 7u) || ((uintptr_t)cols & 3u)) return GCONN_E_INVAL;
    if (!labels || !cols) return GCONN_E_INVAL;
    // no staging copies here (they would allocate): device memory only
    if (!is_device_ptr(offsets) || !is_device_ptr(cols) || !is_device_ptr(labels)) return GCONN_E_INVAL;
    Variant v;
    GC_TRY(resolve_variant(vin, 1, 0, &v));
    if (v.sample == GCONN_SAMPLE_BFS) return GCONN_E_UNSUPPORTED;
    if (v.link != GCONN_LINK_ASYNC && v.link != GCONN_LINK_EARLY && v.link != GCONN_LINK_REMCAS)
        return GCONN_E_UNSUPPORTED;

    uint32_t* hdr = (uint32_t*)(base + OFF_HEADER);
    uint32_t* lmax = hdr;
    uint32_t* cnt = hdr + 1;
    uint32_t* active = (uint32_t*)(base + OFF_ACTIVE);
    uint32_t* small = (uint32_t*)(base + OFF_SMALL);
    unsigned long long* tasks = (unsigned long long*)(base + OFF_TASKS);
    uint32_t* over = (uint32_t*)(base + OFF_OVER);
    bool sampled = v.sample != GCONN_SAMPLE_NONE;

    // the same (link, find, splice) mapping and union-find state as gconn_cc_csr
    int L, F, S;
    uf_triple(v, &L, &F, &S);
    int B = v.block > 0 ? v.block : 256;
    UFState s = make_state(n, labels, nullptr, nullptr, nullptr, v);
    if (!s.err) return GCONN_E_CUDA;

    // the counters must start at zero; everything else is written before read
    GC_CUDA(cudaMemsetAsync(hdr, 0, 4 * sizeof(uint32_t), st));
    GC_TRY(launch("init", k_init, grid_for(k_init, 256, n), 256, 0, st, n, s.P, s.H, s.W, s.sf, nullptr, 0u));
    return dispatch_noalloc(L, F, S, [&]<int l, int fr, int sp>() -> gconn_status {
        if (v.sample == GCONN_SAMPLE_KOUT) {
            auto k = k_kout<l, fr, sp, false>;
            GC_TRY(launch("kout", k, grid_for(k, KOUT_BLOCK, n), KOUT_BLOCK, 0, st, offsets, cols, v.k, s,
                          JobQueue{nullptr, nullptr, 0}, false));
        } else if (v.sample == GCONN_SAMPLE_HB) {
            GC_TRY(launch("hb1", k_hb1<uint64_t>, grid_for(k_hb1<uint64_t>, 256, n), 256, 0, st, offsets, cols, n, s.P, s.sf, s.err));
            auto k = k_hb2<l, fr, sp, false>;
            GC_TRY(launch("hb2", k, grid_for(k, B, n), B, 0, st, offsets, cols, v.hb_n, s));
        }
        if (sampled) {
            GC_TRY(launch("compress", k_compress<LK_ASYNC>, grid_for(k_compress<LK_ASYNC>, 256, n), 256, 0, st, s));
            GC_TRY(launch("lmax", k_lmax<LK_ASYNC>, 1, LMAX_SAMPLES, 0, st, s, v.seed, lmax));
        }
        auto kv = k_vg<LK_ASYNC>;
        GC_TRY(launch("vg", kv, grid_for(kv, 256, (uint64_t)n), 256, 0, st, offsets, s,
                      sampled ? (const uint32_t*)lmax : nullptr, sampled ? active : nullptr, small, cnt + 0, tasks,
                      (uint32_t)TASK_CAP, cnt + 1, over, cnt + 2));
        const uint32_t* act = sampled ? active : nullptr;
        auto k1 = k_finish_small<l, fr, sp, false>;
        GC_TRY(launch("finish_small", k1, grid_for(k1, B, n), B, 0, st, offsets, cols, s, act,
                      (const uint32_t*)small, (const uint32_t*)(cnt + 0)));
        auto k2 = k_finish_tasks<l, fr, sp, false>;
        GC_TRY(launch("finish_tasks", k2, grid_for(k2, B, (uint64_t)n * 32), B, 0, st, offsets, cols, s, act,
                      (const unsigned long long*)tasks, (const uint32_t*)(cnt + 1), (uint32_t)TASK_CAP));
        auto k3 = k_finish_over<l, fr, sp, false>;
        GC_TRY(launch("finish_over", k3, grid_for(k3, B, (uint64_t)n * B), B, 0, st, offsets, cols, s, act,
                      (const uint32_t*)over, (const uint32_t*)(cnt + 2)));
        return launch("finalize", k_finalize, grid_for(k_finalize, 256, n), 256, 0, st, s, labels);
    });
}
