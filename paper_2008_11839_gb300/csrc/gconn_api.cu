// gconn_api.cu -- status codes, the per-device error word, pointer checks,
// stream-ordered scratch, kernel-launch accounting and timing, and variant
// validation for libgconn.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "gc_internal.h"

// Device error word: bit 0 = endpoint out of range, bit 1 = iteration cap
// reached, bit 2 = a size limit was exceeded.  One per device.
__device__ uint32_t g_gconn_err;

namespace gc {

std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_profiling{false};

gconn_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return GCONN_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return GCONN_E_NOMEM;
    }
    return GCONN_E_CUDA;
}

static std::mutex g_mu;
static constexpr int MAX_DEV = 64;
static uint32_t* g_err_ptr[MAX_DEV];
static int g_sms[MAX_DEV];

static cudaMemPool_t g_pool[MAX_DEV];

// Scratch and staging buffers come from one stream-ordered pool per device
// whose release threshold is unlimited: memory a call frees stays reserved in
// the pool for the next call instead of being unmapped at the next
// synchronisation, so repeated calls (and host-input calls that stage whole
// CSR arrays) do not map and unmap device memory every time.
// gconn_release_cached returns the idle part to the device.
cudaMemPool_t scratch_pool() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= MAX_DEV) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps pr{};
        pr.allocType = cudaMemAllocationTypePinned;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &pr) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

static thread_local uint64_t t_csr_arcs_hint = UINT64_MAX;
uint64_t csr_arcs_hint() { return t_csr_arcs_hint; }
CsrArcsHint::CsrArcsHint(uint64_t arcs) { t_csr_arcs_hint = arcs; }
CsrArcsHint::~CsrArcsHint() { t_csr_arcs_hint = UINT64_MAX; }

uint32_t* err_word_lookup() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= MAX_DEV) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_err_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_gconn_err) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_err_ptr[dev] = (uint32_t*)p;
    }
    return g_err_ptr[dev];
}

uint32_t* err_word() {
    uint32_t* w = err_word_lookup();
    if (!w) return nullptr;
    scratch_pool();   // created here too, so that it exists before any stream capture
    return w;
}

int num_sms() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= MAX_DEV) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sms[dev]) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = sms > 0 ? sms : 1;
    }
    return g_sms[dev];
}

gconn_status read_and_clear_err(cudaStream_t st) {
    GC_CUDA(cudaStreamSynchronize(st));
    uint32_t* p = err_word();
    if (!p) return GCONN_E_CUDA;
    uint32_t h = 0;
    GC_CUDA(cudaMemcpy(&h, p, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (h) {
        uint32_t z = 0;
        GC_CUDA(cudaMemcpy(p, &z, sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    if (h & ERR_RANGE) return GCONN_E_RANGE;
    if (h & ERR_NONCONV) return GCONN_E_NONCONVERGED;
    if (h & ERR_OVERFLOW) return GCONN_E_INVAL;
    return GCONN_OK;
}

// A host thread that has not used CUDA yet has no current context, and the
// pointer queries below then cannot see the device's mappings (a page-locked
// buffer would be staged instead of read in place): bind the current
// device's primary context to the thread first, once per thread.
static void bind_context() {
    static thread_local bool bound = false;
    if (bound) return;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaSetDevice(dev) != cudaSuccess) cudaGetLastError();
    bound = true;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    bind_context();
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int pageable_access() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return 0;
    static std::atomic<int> cached[MAX_DEV];   // 0 unknown, 1 no, 2 yes
    int c = cached[dev].load();
    if (c == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
            cudaGetLastError();
            v = 0;
        }
        c = v ? 2 : 1;
        cached[dev].store(c);
    }
    return c == 2;
}

const void* host_direct(const void* p) {
    static const bool staged = [] {
        const char* e = getenv("GCONN_HOST_STAGE");
        return e && e[0] == '1';
    }();
    if (!p || staged) return nullptr;
    bind_context();
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;           // page-locked: its device mapping
    if (a.type == cudaMemoryTypeUnregistered && pageable_access()) return p;
    return nullptr;
}

gconn_status stage_in_once(const void* src, size_t bytes, cudaStream_t st, DevBuf& buf, const void** dev) {
    if (is_device_ptr(src)) {
        *dev = src;
        return GCONN_OK;
    }
    if (const void* d = host_direct(src)) {
        *dev = d;
        return GCONN_OK;
    }
    return stage_in(src, bytes, st, buf, dev);
}

gconn_status DevBuf::alloc(size_t bytes, cudaStream_t stream) {
    release();
    st = stream;
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool = scratch_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, stream) : cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        p = nullptr;
        return cuda_status(e);
    }
    return GCONN_OK;
}

void DevBuf::release() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
}

gconn_status stage_in(const void* src, size_t bytes, cudaStream_t st, DevBuf& buf, const void** dev) {
    if (is_device_ptr(src)) {
        *dev = src;
        return GCONN_OK;
    }
    GC_TRY(buf.alloc(bytes, st));
    GC_CUDA(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, st));
    *dev = buf.p;
    return GCONN_OK;
}

// -------------------------------------------------------- L2 window
void L2Window::apply(cudaStream_t s, void* base, size_t bytes) {
    static int enabled = -1;
    if (enabled < 0) {
        const char* e = getenv("GCONN_L2_WINDOW");
        enabled = (e && e[0] == '1') ? 1 : 0;
    }
    if (!enabled || !s || !base || !bytes) return;
    int dev = 0, max_persist = 0, max_window = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
    cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    if (max_persist <= 0 || max_window <= 0) return;
    size_t carve = bytes < (size_t)max_persist ? bytes : (size_t)max_persist;
    size_t cur = 0;
    cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    if (cur < carve && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, carve) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cudaStreamGetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &old) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaStreamAttrValue v{};
    size_t win = bytes < (size_t)max_window ? bytes : (size_t)max_window;
    v.accessPolicyWindow.base_ptr = base;
    v.accessPolicyWindow.num_bytes = win;
    v.accessPolicyWindow.hitRatio = (float)((double)carve / (double)win > 1.0 ? 1.0 : (double)carve / (double)win);
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    if (cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &v) == cudaSuccess) {
        st = s;
        set = true;
    } else {
        cudaGetLastError();
    }
}

L2Window::~L2Window() {
    if (set) cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &old);
}

// ------------------------------------------------------------- profiling
struct PendingRec {
    std::string name;
    cudaEvent_t a, b;
    bool pooled;      // events return to the pool after collection (not graph-owned)
};
static thread_local ProfSink* t_sink = nullptr;

void prof_set_sink(ProfSink* sink) { t_sink = sink; }

void count_capture_launch() {
    if (t_sink) t_sink->launches++;
}
struct Total {
    uint64_t launches = 0;
    double ms = 0;
};
static std::mutex g_pmu;
static std::vector<PendingRec> g_pending;
static std::vector<cudaEvent_t> g_event_pool;
static std::vector<std::string> g_order;
static std::map<std::string, Total> g_totals;
static std::deque<std::string> g_sink_names;   // stable storage for captured kernel names

static cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Kernel names selected for timing (empty: all).
static std::vector<std::string> g_prof_select;

void prof_begin(const char* name, cudaStream_t st, void** token) {
    std::lock_guard<std::mutex> lk(g_pmu);
    *token = nullptr;
    if (!g_prof_select.empty()) {
        bool hit = false;
        for (const std::string& s : g_prof_select) hit |= s == name;
        if (!hit) return;
    }
    PendingRec* r;
    if (t_sink) {   // graph-owned events: created fresh, kept by the plan
        cudaEvent_t a = nullptr, b = nullptr;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        r = new PendingRec{name, a, b, false};
    } else {
        r = new PendingRec{name, take_event(), take_event(), true};
    }
    // inside a capture an event becomes a graph node only as an external record
    if (t_sink) cudaEventRecordWithFlags(r->a, st, cudaEventRecordExternal);
    else cudaEventRecord(r->a, st);
    *token = r;
}

void prof_end(void* token, cudaStream_t st) {
    PendingRec* r = (PendingRec*)token;
    if (t_sink) cudaEventRecordWithFlags(r->b, st, cudaEventRecordExternal);
    else cudaEventRecord(r->b, st);
    std::lock_guard<std::mutex> lk(g_pmu);
    if (t_sink) {
        // the name is a string literal of the launching code: safe to keep
        t_sink->recs.push_back(ProfRec{nullptr, r->a, r->b});
        t_sink->recs.back().name = nullptr;
        g_sink_names.push_back(r->name);
        t_sink->recs.back().name = g_sink_names.back().c_str();
    } else {
        g_pending.push_back(*r);
    }
    delete r;
}

void prof_requeue(const ProfSink& sink) {
    std::lock_guard<std::mutex> lk(g_pmu);
    for (const ProfRec& r : sink.recs) g_pending.push_back(PendingRec{r.name, r.a, r.b, false});
}

void prof_release(ProfSink& sink) {
    for (ProfRec& r : sink.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    sink.recs.clear();
}

static void prof_collect() {
    std::lock_guard<std::mutex> lk(g_pmu);
    for (auto& r : g_pending) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();   // an unreadable pair is skipped, never left as a pending error
            ms = 0;
        }
        if (!g_totals.count(r.name)) g_order.push_back(r.name);
        Total& t = g_totals[r.name];
        t.launches++;
        t.ms += ms;
        if (r.pooled) {
            g_event_pool.push_back(r.a);
            g_event_pool.push_back(r.b);
        }
    }
    g_pending.clear();
}

// ---------------------------------------------------------------- variants
gconn_status resolve_variant(const gconn_variant* in, int input_kind, int want_forest, Variant* out) {
    gconn_variant d;
    gconn_variant_default(&d);
    if (in) d = *in;
    if (input_kind == 0 && !in) d.sample = GCONN_SAMPLE_NONE;
    gconn_status s = gconn_variant_check(&d, input_kind, want_forest);
    if (s != GCONN_OK) return s;
    out->sample = d.sample;
    out->k = d.k > 0 ? d.k : 2;
    out->hb_n = d.hb_n > 0 ? d.hb_n : 4;
    out->link = d.link;
    out->find = d.find;
    out->splice = d.splice;
    out->lt_rules = d.lt_rules;
    out->block = d.block;
    out->seed = d.seed;
    out->ablation = (int)d.ablation;
    out->cap = d.iter_cap ? d.iter_cap : DEFAULT_CAP;
    return GCONN_OK;
}

}  // namespace gc

using namespace gc;

static bool lt_valid(int r) {
    // the 16 rule sets of the appendix list
    static const int ok[] = {
        GCONN_LT_CONNECT | GCONN_LT_ALTER,                                                    // CUSA
        GCONN_LT_CONNECT | GCONN_LT_ROOTUPDATE | GCONN_LT_ALTER,                              // CRSA
        GCONN_LT_PARENT | GCONN_LT_ALTER,                                                     // PUSA
        GCONN_LT_PARENT | GCONN_LT_ROOTUPDATE | GCONN_LT_ALTER,                               // PRSA
        GCONN_LT_PARENT,                                                                      // PUS
        GCONN_LT_PARENT | GCONN_LT_ROOTUPDATE,                                                // PRS
        GCONN_LT_EXTENDED | GCONN_LT_ALTER,                                                   // EUSA
        GCONN_LT_EXTENDED,                                                                    // EUS
        GCONN_LT_CONNECT | GCONN_LT_FULLSHORTCUT | GCONN_LT_ALTER,                            // CUFA
        GCONN_LT_CONNECT | GCONN_LT_ROOTUPDATE | GCONN_LT_FULLSHORTCUT | GCONN_LT_ALTER,      // CRFA
        GCONN_LT_PARENT | GCONN_LT_FULLSHORTCUT | GCONN_LT_ALTER,                             // PUFA
        GCONN_LT_PARENT | GCONN_LT_ROOTUPDATE | GCONN_LT_FULLSHORTCUT | GCONN_LT_ALTER,       // PRFA
        GCONN_LT_PARENT | GCONN_LT_FULLSHORTCUT,                                              // PUF
        GCONN_LT_PARENT | GCONN_LT_ROOTUPDATE | GCONN_LT_FULLSHORTCUT,                        // PRF
        GCONN_LT_EXTENDED | GCONN_LT_FULLSHORTCUT | GCONN_LT_ALTER,                           // EUFA
        GCONN_LT_EXTENDED | GCONN_LT_FULLSHORTCUT,                                            // EUF
    };
    for (int x : ok)
        if (x == r) return true;
    return false;
}

extern "C" gconn_status gconn_variant_default(gconn_variant* v) {
    if (!v) return GCONN_E_INVAL;
    memset(v, 0, sizeof(*v));
    v->sample = GCONN_SAMPLE_KOUT;
    v->k = 2;
    v->hb_n = 4;
    v->link = GCONN_LINK_REMCAS;   // the fastest finish measured on GB300 (RMAT scale 22)
    v->find = GCONN_FIND_NAIVE;
    v->splice = GCONN_SPLICE_SPLIT_ONE;
    v->lt_rules = GCONN_LT_PARENT | GCONN_LT_ROOTUPDATE | GCONN_LT_FULLSHORTCUT;
    v->block = 0;
    v->seed = DEFAULT_SEED;
    return GCONN_OK;
}

extern "C" gconn_status gconn_variant_check(const gconn_variant* v, int input_kind, int want_forest) {
    if (!v) return GCONN_E_INVAL;
    if (input_kind != 0 && input_kind != 1) return GCONN_E_INVAL;
    if (want_forest < 0 || want_forest > 2) return GCONN_E_INVAL;
    if (v->ablation & ~(GCONN_ABL_PLAIN_SAMPLE | GCONN_ABL_NO_VG)) return GCONN_E_INVAL;
    if (v->sample < 0 || v->sample > GCONN_SAMPLE_BFS) return GCONN_E_INVAL;
    if (v->link < 0 || v->link > GCONN_LINK_STERGIOU) return GCONN_E_INVAL;
    if (v->find < 0 || v->find > GCONN_FIND_FULLSHORTCUT) return GCONN_E_INVAL;
    if (v->splice < 0 || v->splice > GCONN_SPLICE_SPLICE) return GCONN_E_INVAL;
    if (v->k < 0 || v->hb_n < 0 || v->k > 1024 || v->hb_n > 1024) return GCONN_E_INVAL;
    if (v->block != 0 && (v->block < 64 || v->block > 1024 || v->block % 32 != 0)) return GCONN_E_INVAL;
    if (v->sample != GCONN_SAMPLE_NONE && input_kind == 0) return GCONN_E_UNSUPPORTED;
    bool rem = v->link == GCONN_LINK_REMCAS || v->link == GCONN_LINK_REMLOCK, jtb = v->link == GCONN_LINK_JTB;
    bool fixed_find = v->link == GCONN_LINK_SV || v->link == GCONN_LINK_ECLCC || v->link == GCONN_LINK_AFFOREST ||
                      v->link == GCONN_LINK_LP || v->link == GCONN_LINK_STERGIOU;
    if (fixed_find && v->find != GCONN_FIND_NAIVE && v->find != GCONN_FIND_FULLSHORTCUT)
        return GCONN_E_UNSUPPORTED;
    // LP and Stergiou move non-roots between trees: components only
    if ((v->link == GCONN_LINK_LP || v->link == GCONN_LINK_STERGIOU) && want_forest) return GCONN_E_UNSUPPORTED;
    if (v->splice != GCONN_SPLICE_NONE && !rem) return GCONN_E_UNSUPPORTED;
    if (v->find == GCONN_FIND_TWOTRYSPLIT && !jtb) return GCONN_E_UNSUPPORTED;
    if (rem && v->find == GCONN_FIND_COMPRESS) return GCONN_E_UNSUPPORTED;
    // SpliceAtomic re-points non-roots into another tree: not root-based
    // (Section 2), so it cannot record a forest; fine for incremental batches
    if (want_forest == 1 && rem && (v->splice == GCONN_SPLICE_SPLICE || v->splice == GCONN_SPLICE_NONE))
        return GCONN_E_UNSUPPORTED;
    if (jtb && v->find != GCONN_FIND_NAIVE && v->find != GCONN_FIND_TWOTRYSPLIT &&
        v->find != GCONN_FIND_FULLSHORTCUT)
        return GCONN_E_UNSUPPORTED;
    if (v->link == GCONN_LINK_LT) {
        if (!lt_valid(v->lt_rules)) return GCONN_E_UNSUPPORTED;
        if (v->find != GCONN_FIND_NAIVE && v->find != GCONN_FIND_FULLSHORTCUT) return GCONN_E_UNSUPPORTED;
        if (want_forest && !(v->lt_rules & GCONN_LT_ROOTUPDATE)) return GCONN_E_UNSUPPORTED;
    }
    return GCONN_OK;
}

extern "C" gconn_status gconn_sync(void* stream) { return read_and_clear_err((cudaStream_t)stream); }

extern "C" const char* gconn_status_str(gconn_status s) {
    switch (s) {
        case GCONN_OK: return "ok";
        case GCONN_E_INVAL: return "invalid argument";
        case GCONN_E_RANGE: return "vertex id out of range";
        case GCONN_E_NOMEM: return "device out of memory";
        case GCONN_E_UNSUPPORTED: return "unsupported variant combination";
        case GCONN_E_NONCONVERGED: return "iteration cap reached";
        case GCONN_E_CUDA: return "CUDA runtime error";
    }
    return "unknown status";
}

extern "C" uint64_t gconn_launch_count(void) { return g_launches.load(); }

extern "C" gconn_status gconn_release_cached(void) {
    if (!err_word()) return GCONN_E_CUDA;
    cudaMemPool_t pool = scratch_pool();
    if (!pool) return GCONN_E_CUDA;
    GC_CUDA(cudaMemPoolTrimTo(pool, 0));
    return GCONN_OK;
}

extern "C" gconn_status gconn_profile_enable(int on) {
    g_profiling.store(on != 0);
    return GCONN_OK;
}

extern "C" gconn_status gconn_profile_select(const char* names) {
    std::vector<std::string> sel;
    if (names) {
        std::string cur;
        for (const char* c = names;; ++c) {
            if (*c == ',' || *c == 0) {
                if (!cur.empty()) sel.push_back(cur);
                cur.clear();
                if (*c == 0) break;
            } else if (*c != ' ') {
                cur.push_back(*c);
            }
        }
    }
    std::lock_guard<std::mutex> lk(g_pmu);
    g_prof_select.swap(sel);
    return GCONN_OK;
}

extern "C" gconn_status gconn_profile_reset(void) {
    prof_collect();
    std::lock_guard<std::mutex> lk(g_pmu);
    g_totals.clear();
    g_order.clear();
    return GCONN_OK;
}

extern "C" gconn_status gconn_profile_sync(void) {
    prof_collect();
    return GCONN_OK;
}

extern "C" gconn_status gconn_profile_get(int i, const char** name, uint64_t* launches, double* total_ms) {
    prof_collect();
    std::lock_guard<std::mutex> lk(g_pmu);
    if (i < 0 || i >= (int)g_order.size()) return GCONN_E_INVAL;
    const std::string& k = g_order[i];
    const Total& t = g_totals[k];
    if (name) *name = k.c_str();
    if (launches) *launches = t.launches;
    if (total_ms) *total_ms = t.ms;
    return GCONN_OK;
}
