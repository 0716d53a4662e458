// gc_internal.h -- host-side helpers shared by the libgconn translation units:
// status plumbing, pointer classification, stream-ordered scratch buffers,
// occupancy-sized grids, and the launch wrapper that counts and (optionally)
// times every kernel launch with CUDA events on the launching stream.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>
#include <vector>

#include "../../include/gconn.h"

namespace gc {

constexpr uint32_t INF = 0xFFFFFFFFu;
constexpr uint32_t ERR_RANGE = 1u;
constexpr uint32_t ERR_NONCONV = 2u;
constexpr uint32_t ERR_OVERFLOW = 4u;
constexpr uint32_t DEFAULT_CAP = 1u << 24;
constexpr uint64_t DEFAULT_SEED = 0x6C0A0001ull;

// ------------------------------------------------------------------ status
#define GC_CUDA(call)                                                             \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) return ::gc::cuda_status(e_);                      \
    } while (0)
#define GC_TRY(call)                                                              \
    do {                                                                          \
        gconn_status s_ = (call);                                                 \
        if (s_ != GCONN_OK) return s_;                                            \
    } while (0)

gconn_status cuda_status(cudaError_t e);          // maps OOM -> E_NOMEM, else E_CUDA
uint32_t* err_word();                             // device error word of the current device (+ its pool)
uint32_t* err_word_lookup();                      // the same word, without creating the scratch pool
cudaMemPool_t scratch_pool();                     // caching scratch pool of the current device
gconn_status read_and_clear_err(cudaStream_t st); // sync st, then read/clear the word

// ----------------------------------------------------------------- devices
int num_sms();                                    // SM count of the current device
bool is_device_ptr(const void* p);                // device or managed memory

// ------------------------------------------------------- scratch buffers
// Stream-ordered device allocation: allocated and released on one stream.
struct DevBuf {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    gconn_status alloc(size_t bytes, cudaStream_t stream);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ------------------------------------------------------------ launching
extern std::atomic<uint64_t> g_launches;
extern std::atomic<bool> g_profiling;
void prof_begin(const char* name, cudaStream_t st, void** token);
void prof_end(void* token, cudaStream_t st);

// Per-kernel event pairs captured into a CUDA graph: while a capture sink is
// set on this thread, prof_end hands its record to the sink instead of the
// global pending list; a replay re-queues the captured records (their events
// re-record on every replay, so each replay must be collected before the next).
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
struct ProfSink {
    std::vector<ProfRec> recs;
    uint64_t launches = 0;
};
void prof_set_sink(ProfSink* sink);
void count_capture_launch();
void prof_requeue(const ProfSink& sink);
void prof_release(ProfSink& sink);

// Largest edge / pair / query count an entry point accepts: 8-byte items, so
// every byte count stays below 2^63.
constexpr uint64_t GC_MAX_COUNT = 1ull << 60;

// Persistent-style grid: min(ceil(work / block), resident blocks on all SMs).
template <class K>
unsigned grid_for(K kernel, int block, uint64_t work, size_t smem = 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    uint64_t cap = (uint64_t)per_sm * (uint64_t)num_sms();
    uint64_t need = (work + (uint64_t)block - 1) / (uint64_t)block;
    if (need < 1) need = 1;
    return (unsigned)(need < cap ? need : cap);
}

template <class... KArgs, class... Args>
gconn_status launch(const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                    cudaStream_t st, Args&&... args) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    count_capture_launch();
    cudaGetLastError();   // report this launch's error only
    void* tok = nullptr;
    if (g_profiling.load(std::memory_order_relaxed)) prof_begin(name, st, &tok);
    kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
    cudaError_t e = cudaGetLastError();
    if (tok) prof_end(tok, st);
    return e == cudaSuccess ? GCONN_OK : cuda_status(e);
}

// As launch(), with programmatic stream serialisation: the kernel may be
// scheduled while the previous kernel in the stream is still running (also as
// a programmatic edge inside a captured graph).  Only for kernels that begin
// with pdl_entry(), whose griddepcontrol.wait restores the ordering.
template <class... KArgs, class... Args>
gconn_status launch_pdl(const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                        cudaStream_t st, Args&&... args) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    count_capture_launch();
    cudaGetLastError();
    void* tok = nullptr;
    if (g_profiling.load(std::memory_order_relaxed)) prof_begin(name, st, &tok);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (tok) prof_end(tok, st);
    return e == cudaSuccess ? GCONN_OK : cuda_status(e);
}

// As launch(), as a cooperative launch: every block of the grid is resident
// at once (the grid must not exceed what the occupancy API allows), so the
// kernel may use grid-wide barriers.
template <class... KArgs, class... Args>
gconn_status launch_coop(const char* name, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                         cudaStream_t st, Args&&... args) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    count_capture_launch();
    cudaGetLastError();
    void* tok = nullptr;
    if (g_profiling.load(std::memory_order_relaxed)) prof_begin(name, st, &tok);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (tok) prof_end(tok, st);
    return e == cudaSuccess ? GCONN_OK : cuda_status(e);
}

// --------------------------------------------------------------- variant
struct Variant {
    int sample, k, hb_n, link, find, splice, lt_rules, block;
    uint64_t seed;
    uint32_t cap;
    int ablation;   // GCONN_ABL_* bits
};
gconn_status resolve_variant(const gconn_variant* in, int input_kind, int want_forest, Variant* out);

// Optional L2 persistence window over the parent array for the launches on
// one stream (GCONN_L2_WINDOW=1): sets the stream's access-policy window and
// restores the previous one on destruction.  The persisting-L2 carve-out is a
// limit of this process's context only.
struct L2Window {
    cudaStream_t st = nullptr;
    cudaStreamAttrValue old{};
    bool set = false;
    void apply(cudaStream_t s, void* base, size_t bytes);
    ~L2Window();
};

// Device view of an incremental handle (for the serving loop's merged launches).
struct IncView {
    uint32_t n;
    uint32_t* P;
    uint32_t* H;
    unsigned long long* W;
    Variant v;
};
bool inc_view(const gconn_inc* h, IncView* out);

// The arc count of the CSR input a plan is being captured for (UINT64_MAX =
// unknown): the plan-creation calls read offsets[n] before capturing and set
// it for the capture, so that the parts of a pass that size a buffer from the
// arc count need no device read (illegal while capturing).
uint64_t csr_arcs_hint();
struct CsrArcsHint {
    explicit CsrArcsHint(uint64_t arcs);
    ~CsrArcsHint();
};

// Staging of possibly-host arrays onto the device.
gconn_status stage_in(const void* src, size_t bytes, cudaStream_t st, DevBuf& buf, const void** dev);

// A device-usable address for host memory that kernels can read in place:
// page-locked memory (its device mapping), or pageable memory on a device
// that accesses pageable memory coherently (cudaDevAttrPageableMemoryAccess:
// through the host's page tables on NVLink-C2C systems); nullptr otherwise,
// or when the environment sets GCONN_HOST_STAGE=1 (always copy).
const void* host_direct(const void* p);
// For an array a pass reads once, or only in part: device memory as is, host
// memory in place when host_direct allows it, else a staged copy.
gconn_status stage_in_once(const void* src, size_t bytes, cudaStream_t st, DevBuf& buf, const void** dev);

}  // namespace gc
