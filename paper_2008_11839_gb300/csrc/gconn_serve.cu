// gconn_serve.cu -- a serving loop over device-resident incremental
// connectivity (Section 3.5): clients submit insert and query batches for
// sessions (one union-find forest each); a worker thread runs scheduler
// steps.  Each step takes, from every session that may proceed, the run of
// pending requests at the head of its queue that share one kind (insert or
// query), packs all of them -- across sessions -- into one pinned staging
// buffer, and processes them with one host-to-device copy, one multi-forest
// kernel per union rule present (every thread finds its request's segment and
// works in that session's forest), and one device-to-host copy of the
// answers.  Steps alternate between streams, so one step's copies and kernels
// overlap the next one's staging.  Admission is bounded by a device-memory
// budget and by the number of steps in flight.
//
// Where the kernels can use a request's buffers in place (device memory, or
// host memory the device reads directly: page-locked, or pageable on a device
// with coherent access), the step reads its pairs and writes its answers
// there: no staging copy and no copies to and from the device (only the
// segment table is copied); such a request above a step's size runs as a
// step of its own instead of through its handle's calls.
//
// Exactness per session: requests form phases of consecutive inserts or
// consecutive queries; a session joins a step only with requests of the phase
// it already has in flight (or any phase when it has nothing in flight), so a
// query sees exactly the inserts submitted before it.  Inserts of one phase
// commute and queries of one phase only compress paths, so packing and
// concurrency change no answer.  Requests larger than a step's staging and
// sessions with round-based finishes (SV, Liu-Tarjan) run through their
// handle's own calls as a step of their own.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "gc_internal.h"
#include "gc_static.h"
#include "uf_device.cuh"

namespace {

using Clock = std::chrono::steady_clock;
using namespace gc;

constexpr uint32_t MAX_SEGS = 4096;   // requests per merged step

struct Request {
    uint64_t ticket;
    uint32_t session;
    int op;                       // GCONN_OP_INSERT / GCONN_OP_QUERY
    uint64_t count;
    const uint32_t* pairs;        // host
    uint8_t* result;              // host, queries only
    Clock::time_point submitted;
    // device-usable addresses of pairs / result when kernels can use the
    // client's host buffers in place (host_direct), else null
    const uint32_t* d_pairs;
    uint8_t* d_result;
    bool direct() const { return d_pairs && (op != GCONN_OP_QUERY || d_result); }
};

struct Session {
    uint32_t id;
    gconn_inc* h = nullptr;
    IncView view;
    bool mergeable = false;       // union-find finish: can join merged steps
    std::deque<Request> pending;
    int inflight_phase = -1;      // kind of the work in flight, -1 = none
    int inflight = 0;             // steps holding this session's requests
    bool closing = false;
};

// One segment of a merged step: a request's pairs inside the step.
struct Seg {
    unsigned long long start;     // first pair of the segment in its launch range
    unsigned long long out;       // first answer slot (queries)
    uint32_t* P;
    uint32_t* H;
    unsigned long long* W;
    uint32_t n, op, cap, seed;
    const uint2* src;             // in-place steps: the request's pairs
    uint8_t* dst;                 //                 and answers (client memory)
};

struct StepBuf {
    cudaStream_t st = nullptr;
    uint32_t* h_pairs = nullptr;  // pinned
    uint8_t* h_out = nullptr;     // pinned
    Seg* h_segs = nullptr;        // pinned
    uint32_t* h_err = nullptr;    // pinned
    bool busy = false;
};

struct Step {
    int buf = -1;
    bool solo = false;            // one request through its handle's own calls
    bool direct = false;          // every request read / answered in place
    std::vector<Request> reqs;
    std::vector<uint32_t> seg_of; // request -> its answer offset (queries)
    uint64_t total = 0, answers = 0, bytes = 0;
    cudaEvent_t done = nullptr;
    gconn_status status = GCONN_OK;
};

// Multi-forest union / query over one launch range of a merged step.  An
// in-place step (DIRECT) reads each request's pairs and writes its answers in
// the client's own buffers through the segment's addresses; a staged step
// uses the step's packed device copy.
template <int L, int F, int S, bool DIRECT>
__global__ void __launch_bounds__(256) k_serve(const uint2* __restrict__ pairs, unsigned long long total,
                                               const Seg* __restrict__ segs, uint32_t nseg, uint8_t* out,
                                               uint32_t* err) {
    __shared__ unsigned long long sstart[MAX_SEGS];
    bool cached = nseg <= MAX_SEGS;
    if (cached)
        for (uint32_t i = threadIdx.x; i < nseg; i += blockDim.x) sstart[i] = segs[i].start;
    __syncthreads();
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        uint32_t lo = 0, hi = nseg;   // last segment with start <= i
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            unsigned long long sm = cached ? sstart[mid] : segs[mid].start;
            if (sm <= i) lo = mid; else hi = mid;
        }
        const Seg& g = segs[lo];
        UFState s;
        s.P = g.P; s.H = g.H; s.W = g.W; s.sf = nullptr; s.err = err; s.Lk = nullptr;
        s.n = g.n; s.cap = g.cap; s.seed = g.seed;
        uint2 e = DIRECT ? __ldcs(g.src + (i - g.start)) : __ldcs(pairs + i);
        bool inrange = e.x < g.n && e.y < g.n;
        if (!inrange) atomicOr(err, GC_DERR_RANGE);
        Spin sp(g.cap);
        if (g.op == GCONN_OP_INSERT) {
            if (inrange && e.x != e.y) uf_union<L, F, S, false>(s, e.x, e.y, 0, sp);
        } else {
            uint8_t a = 0;
            if (inrange) {
                if (L == LK_JTB) a = jtb_find<F>(s, e.x, sp) == jtb_find<F>(s, e.y, sp);
                else if (F == FD_NAIVE) a = same_root_lockstep(s, e.x, e.y, sp);
                else a = uf_find<F, true>(s, e.x, sp) == uf_find<F, true>(s, e.y, sp);
            }
            if (DIRECT) g.dst[i - g.start] = a;
            else out[g.out + (i - g.start)] = a;
        }
    }
}

int rule_key(const Variant& v) {
    int L, F, S;
    uf_triple(v, &L, &F, &S);
    return (L << 8) | (F << 4) | S;
}

template <class Fn>
gconn_status dispatch_rule(int key, Fn&& fn) {
    int L = key >> 8, F = (key >> 4) & 15, S = key & 15;
#define GC_SV_CASE(l, f, s) \
    if (L == l && F == f && S == s) return fn.template operator()<l, f, s>();
    GC_SV_CASE(LK_ASYNC, FD_NAIVE, SP_NONE)
    GC_SV_CASE(LK_ASYNC, FD_COMPRESS, SP_NONE)
    GC_SV_CASE(LK_ASYNC, FD_SPLIT, SP_NONE)
    GC_SV_CASE(LK_ASYNC, FD_HALVE, SP_NONE)
    GC_SV_CASE(LK_HOOKS, FD_NAIVE, SP_NONE)
    GC_SV_CASE(LK_HOOKS, FD_COMPRESS, SP_NONE)
    GC_SV_CASE(LK_HOOKS, FD_SPLIT, SP_NONE)
    GC_SV_CASE(LK_HOOKS, FD_HALVE, SP_NONE)
    GC_SV_CASE(LK_EARLY, FD_NAIVE, SP_NONE)
    GC_SV_CASE(LK_EARLY, FD_COMPRESS, SP_NONE)
    GC_SV_CASE(LK_EARLY, FD_SPLIT, SP_NONE)
    GC_SV_CASE(LK_EARLY, FD_HALVE, SP_NONE)
    GC_SV_CASE(LK_REMCAS, FD_NAIVE, SP_SPLIT_ONE)
    GC_SV_CASE(LK_REMCAS, FD_NAIVE, SP_HALVE_ONE)
    GC_SV_CASE(LK_REMCAS, FD_NAIVE, SP_SPLICE)
    GC_SV_CASE(LK_REMCAS, FD_SPLIT, SP_SPLIT_ONE)
    GC_SV_CASE(LK_REMCAS, FD_SPLIT, SP_HALVE_ONE)
    GC_SV_CASE(LK_REMCAS, FD_SPLIT, SP_SPLICE)
    GC_SV_CASE(LK_REMCAS, FD_HALVE, SP_SPLIT_ONE)
    GC_SV_CASE(LK_REMCAS, FD_HALVE, SP_HALVE_ONE)
    GC_SV_CASE(LK_REMCAS, FD_HALVE, SP_SPLICE)
    GC_SV_CASE(LK_JTB, FD_NAIVE, SP_NONE)
    GC_SV_CASE(LK_JTB, FD_TWOTRY, SP_NONE)
#undef GC_SV_CASE
    return GCONN_E_UNSUPPORTED;
}

}  // namespace

struct gconn_server {
    int device = 0;
    gconn_server_config cfg;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    uint32_t next_session = 1;
    uint32_t rr = 0;              // round-robin start among sessions
    std::map<uint32_t, Session> sessions;
    std::vector<StepBuf> bufs;
    std::deque<std::unique_ptr<Step>> inflight;
    uint64_t bytes_inflight = 0;
    struct Done {
        gconn_status status;
        double latency_ms;
    };
    std::map<uint64_t, Done> done;
    std::set<uint64_t> unclaimed;   // issued tickets no gconn_server_wait has taken yet
    uint64_t launches = 0, steps = 0, requests_done = 0;
};

namespace {

gconn_status status_of_err(uint32_t e) {
    if (e & GC_DERR_RANGE) return GCONN_E_RANGE;
    if (e & GC_DERR_NONCONV) return GCONN_E_NONCONVERGED;
    return GCONN_OK;
}

// A merged step: stage every request's pairs (grouped by union rule), copy
// once, launch per rule, copy the answers back, all on the buffer's stream.
// An in-place step copies only its segment table: the kernels read the
// pairs and write the answers in the clients' buffers.
gconn_status launch_merged(gconn_server* S, Step& sp, std::vector<Session*>& owners) {
    StepBuf& b = S->bufs[sp.buf];
    cudaStream_t st = b.st;
    // group requests by rule so each rule's pairs are contiguous
    std::vector<size_t> idx(sp.reqs.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::vector<int> key(sp.reqs.size());
    for (size_t i = 0; i < idx.size(); ++i) key[i] = rule_key(owners[i]->view.v);
    std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t c) { return key[a] < key[c]; });
    sp.seg_of.assign(sp.reqs.size(), 0);
    uint64_t pos = 0, ans = 0;
    for (size_t j = 0; j < idx.size(); ++j) {
        const Request& r = sp.reqs[idx[j]];
        if (!sp.direct) memcpy(b.h_pairs + 2 * pos, r.pairs, sizeof(uint32_t) * 2 * r.count);
        const IncView& v = owners[idx[j]]->view;
        Seg& g = b.h_segs[j];
        g.start = pos;
        g.out = ans;
        g.src = (const uint2*)r.d_pairs;
        g.dst = r.d_result;
        g.P = v.P; g.H = v.H; g.W = v.W;
        g.n = v.n;
        g.op = (uint32_t)r.op;
        g.cap = v.v.cap;
        g.seed = (uint32_t)(v.v.seed ^ (v.v.seed >> 32));
        sp.seg_of[idx[j]] = (uint32_t)ans;
        if (r.op == GCONN_OP_QUERY) ans += r.count;
        pos += r.count;
    }
    sp.total = pos;
    sp.answers = ans;
    size_t nseg = idx.size();
    // launch ranges: one per union rule; segment starts become relative to
    // their range before the table is copied (once)
    std::vector<std::pair<size_t, size_t>> ranges;
    std::vector<uint64_t> r0s;
    for (size_t a = 0; a < nseg;) {
        size_t c = a;
        while (c < nseg && key[idx[c]] == key[idx[a]]) ++c;
        ranges.push_back({a, c});
        r0s.push_back(b.h_segs[a].start);
        a = c;
    }
    for (size_t r = 0; r < ranges.size(); ++r)
        for (size_t j = ranges[r].first; j < ranges[r].second; ++j) b.h_segs[j].start -= r0s[r];
    size_t seg_bytes = sizeof(Seg) * nseg;
    // one device block: pairs | answers | segments | error word (an
    // in-place step keeps only the segments and the error word)
    size_t off_out = sp.direct ? 0 : sizeof(uint32_t) * 2 * pos;
    size_t off_seg = (off_out + (sp.direct ? 0 : ans) + 255) & ~(size_t)255;
    size_t off_err = off_seg + seg_bytes;
    // from the library's caching pool: the step's block is reused, not mapped
    // and unmapped per step
    char* d = nullptr;
    cudaMemPool_t pool = scratch_pool();
    GC_CUDA(pool ? cudaMallocFromPoolAsync((void**)&d, off_err + 16, pool, st)
                 : cudaMallocAsync((void**)&d, off_err + 16, st));
    GC_CUDA(cudaMemsetAsync(d + off_err, 0, sizeof(uint32_t), st));
    if (!sp.direct) GC_CUDA(cudaMemcpyAsync(d, b.h_pairs, off_out, cudaMemcpyHostToDevice, st));
    GC_CUDA(cudaMemcpyAsync(d + off_seg, b.h_segs, seg_bytes, cudaMemcpyHostToDevice, st));
    uint32_t* d_err = (uint32_t*)(d + off_err);
    const Seg* d_segs = (const Seg*)(d + off_seg);
    uint8_t* d_out = (uint8_t*)(d + off_out);
    for (size_t r = 0; r < ranges.size(); ++r) {
        size_t a = ranges[r].first, c = ranges[r].second;
        uint64_t r0 = r0s[r], r1 = r + 1 < ranges.size() ? r0s[r + 1] : pos;
        const uint2* rp = (const uint2*)d + r0;
        GC_TRY(dispatch_rule(key[idx[a]], [&]<int l, int f, int k2>() {
            auto k = sp.direct ? k_serve<l, f, k2, true> : k_serve<l, f, k2, false>;
            return launch("serve", k, grid_for(k, 256, r1 - r0), 256, 0, st, rp, (unsigned long long)(r1 - r0),
                          d_segs + a, (uint32_t)(c - a), d_out, d_err);
        }));
        S->launches++;
    }
    if (ans && !sp.direct) GC_CUDA(cudaMemcpyAsync(b.h_out, d + off_out, ans, cudaMemcpyDeviceToHost, st));
    GC_CUDA(cudaMemcpyAsync(b.h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GC_CUDA(cudaFreeAsync(d, st));
    GC_CUDA(cudaEventRecord(sp.done, st));
    return GCONN_OK;
}

// A solo step: one request through its handle's own calls (host buffers).
gconn_status launch_solo(gconn_server* S, Step& sp, Session& ses) {
    const Request& r = sp.reqs[0];
    cudaStream_t st = S->bufs[sp.buf].st;
    gconn_status s;
    if (r.op == GCONN_OP_INSERT) s = gconn_inc_insert_batch(ses.h, r.count, r.pairs, st);
    else s = gconn_inc_query(ses.h, r.count, r.pairs, r.result, st);
    S->launches++;
    cudaEventRecord(sp.done, st);
    return s;
}

void worker_loop(gconn_server* S) {
    cudaSetDevice(S->device);
    const uint64_t C = S->cfg.slot_pairs;
    auto last_progress = Clock::now();
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // 1. completions
        bool progressed = false;
        for (auto it = S->inflight.begin(); it != S->inflight.end();) {
            Step& sp = **it;
            cudaError_t q = cudaEventQuery(sp.done);
            if (q == cudaErrorNotReady) {
                ++it;
                continue;
            }
            StepBuf& b = S->bufs[sp.buf];
            if (q != cudaSuccess && sp.status == GCONN_OK) sp.status = cuda_status(q);
            if (!sp.solo && sp.status == GCONN_OK) {
                sp.status = status_of_err(*b.h_err);
                for (size_t i = 0; i < sp.reqs.size() && !sp.direct; ++i) {
                    const Request& r = sp.reqs[i];
                    if (r.op == GCONN_OP_QUERY) memcpy(r.result, b.h_out + sp.seg_of[i], r.count);
                }
            }
            auto now = Clock::now();
            for (const Request& r : sp.reqs) {
                double ms = std::chrono::duration<double, std::milli>(now - r.submitted).count();
                S->done[r.ticket] = {sp.status, ms};
                S->requests_done++;
                Session& ses = S->sessions[r.session];
                if (--ses.inflight == 0) ses.inflight_phase = -1;
            }
            b.busy = false;
            S->bytes_inflight -= sp.bytes;
            cudaEventDestroy(sp.done);
            it = S->inflight.erase(it);
            progressed = true;
        }
        if (progressed) S->cv_done.notify_all();
        // 2. new steps while staging buffers are free
        bool launched = false;
        auto free_buf = [&]() -> int {
            for (size_t i = 0; i < S->bufs.size(); ++i)
                if (!S->bufs[i].busy) return (int)i;
            return -1;
        };
        auto start_step = [&](std::unique_ptr<Step> sp, std::vector<Session*> owners) {
            S->bufs[sp->buf].busy = true;
            S->bytes_inflight += sp->bytes;
            S->steps++;
            cudaEventCreateWithFlags(&sp->done, cudaEventDisableTiming);
            Step* p = sp.get();
            S->inflight.push_back(std::move(sp));
            lk.unlock();
            gconn_status ls = p->solo ? launch_solo(S, *p, *owners[0]) : launch_merged(S, *p, owners);
            if (ls != GCONN_OK) {
                cudaGetLastError();
                p->status = ls;
                cudaEventRecord(p->done, S->bufs[p->buf].st);
            }
            lk.lock();
            launched = true;
        };
        size_t ns = S->sessions.size();
        // 2a. one request that cannot be merged (round-based finish, or larger
        //     than a step's staging) runs as a step of its own
        if (ns) {
            auto it = S->sessions.begin();
            std::advance(it, S->rr % ns);
            for (size_t visited = 0; visited < ns; ++visited, ++it) {
                if (it == S->sessions.end()) it = S->sessions.begin();
                Session& ses = it->second;
                if (ses.pending.empty()) continue;
                const Request& r = ses.pending.front();
                if (ses.inflight_phase != -1 && ses.inflight_phase != r.op) continue;
                if (ses.mergeable && (r.count <= C || r.direct())) continue;
                uint64_t need = (sizeof(uint32_t) * 2 + (r.op == GCONN_OP_QUERY ? 1 : 0)) * r.count;
                if (S->bytes_inflight && S->bytes_inflight + need > S->cfg.device_budget_bytes) break;
                int bi = free_buf();
                if (bi < 0) break;
                auto sp = std::make_unique<Step>();
                sp->buf = bi;
                sp->solo = true;
                sp->reqs.push_back(r);
                sp->bytes = need;
                ses.pending.pop_front();
                ses.inflight_phase = r.op;
                ses.inflight += 1;
                start_step(std::move(sp), std::vector<Session*>{&ses});
                break;
            }
        }
        // 2b. one merged step over every session that may proceed
        int bi = free_buf();
        ns = S->sessions.size();
        if (bi >= 0 && ns) {
            auto sp = std::make_unique<Step>();
            sp->buf = bi;
            std::vector<Session*> owners;
            auto it = S->sessions.begin();
            std::advance(it, S->rr % ns);
            int kind = -1;                  // in-place (1) or staged (0): fixed by the first request taken
            for (size_t visited = 0; visited < ns; ++visited, ++it) {
                if (it == S->sessions.end()) it = S->sessions.begin();
                Session& ses = it->second;
                if (ses.pending.empty() || !ses.mergeable) continue;
                int op = ses.pending.front().op;
                if (ses.inflight_phase != -1 && ses.inflight_phase != op) continue;
                while (!ses.pending.empty() && ses.pending.front().op == op && sp->reqs.size() < MAX_SEGS) {
                    const Request& r = ses.pending.front();
                    int rk = r.direct() ? 1 : 0;
                    if (kind != -1 && rk != kind) break;
                    // a step's requests all finish together, so a large request
                    // merges with nothing (a small one would wait for it): an
                    // in-place request above C pairs runs as a step of its own,
                    // other steps stop at C pairs (a staged request above C is a
                    // solo step, 2a)
                    if (rk && r.count > C && !sp->reqs.empty()) break;
                    if (!rk && r.count > C) break;
                    if (sp->total && sp->total + r.count > C) break;
                    uint64_t need = rk ? 0 : (sizeof(uint32_t) * 2 + (op == GCONN_OP_QUERY ? 1 : 0)) * r.count;
                    if (S->bytes_inflight + sp->bytes + need > S->cfg.device_budget_bytes &&
                        !(S->bytes_inflight == 0 && sp->reqs.empty()))
                        break;
                    kind = rk;
                    sp->direct = rk == 1;
                    sp->reqs.push_back(r);
                    owners.push_back(&ses);
                    sp->total += r.count;
                    sp->bytes += need;
                    ses.pending.pop_front();
                    ses.inflight_phase = op;
                    ses.inflight += 1;
                }
                if (sp->total >= C || sp->reqs.size() >= MAX_SEGS) break;
            }
            if (!sp->reqs.empty()) start_step(std::move(sp), owners);
        }
        S->rr++;
        if (S->stop && S->inflight.empty()) {
            bool any = false;
            for (auto& kv : S->sessions) any |= !kv.second.pending.empty();
            if (!any) break;
        }
        if (launched || progressed) last_progress = Clock::now();
        if (!launched && !progressed) {
            if (S->inflight.empty()) S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            else {
                // steps in flight: poll their events by yielding for the first
                // 200 us after the last progress (a timed sleep overshoots by
                // tens of microseconds, which a short step would wait for),
                // then by short sleeps
                lk.unlock();
                if (Clock::now() - last_progress < std::chrono::microseconds(200)) std::this_thread::yield();
                else std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            }
        }
    }
}

}  // namespace

extern "C" gconn_status gconn_server_config_default(gconn_server_config* c) {
    if (!c) return GCONN_E_INVAL;
    c->device_budget_bytes = 4ull << 30;
    c->slots = 3;
    c->coalesce_pairs = 1u << 22;
    c->slot_pairs = 1u << 22;
    c->reserved = 0;
    return GCONN_OK;
}

extern "C" gconn_status gconn_server_create(const gconn_server_config* cfg, gconn_server** out) {
    if (!out) return GCONN_E_INVAL;
    *out = nullptr;
    gconn_server_config c;
    gconn_server_config_default(&c);
    if (cfg) c = *cfg;
    if (c.slots < 1 || c.slots > 64 || c.slot_pairs < 1024 || c.device_budget_bytes < 1) return GCONN_E_INVAL;
    gconn_server* S = new gconn_server();
    S->cfg = c;
    cudaGetDevice(&S->device);
    if (!err_word()) {
        delete S;
        return GCONN_E_CUDA;
    }
    S->bufs.resize(c.slots);
    for (StepBuf& b : S->bufs) {
        if (cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&b.h_pairs, sizeof(uint32_t) * 2 * (size_t)c.slot_pairs) != cudaSuccess ||
            cudaMallocHost(&b.h_out, c.slot_pairs) != cudaSuccess ||
            cudaMallocHost(&b.h_segs, sizeof(Seg) * MAX_SEGS) != cudaSuccess ||
            cudaMallocHost(&b.h_err, sizeof(uint32_t)) != cudaSuccess) {
            gconn_server_destroy(S);
            return GCONN_E_NOMEM;
        }
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return GCONN_OK;
}

extern "C" gconn_status gconn_server_open_session(gconn_server* S, uint32_t n, const gconn_variant* v,
                                                  uint32_t* session) {
    if (!S || !session) return GCONN_E_INVAL;
    gconn_inc* h = nullptr;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    gconn_status s = gconn_inc_create(n, v, nullptr, &h);
    if (s == GCONN_OK) s = cuda_status(cudaStreamSynchronize(nullptr));
    cudaSetDevice(prev);
    if (s != GCONN_OK) {
        if (h) gconn_inc_destroy(h);
        return s;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    uint32_t id = S->next_session++;
    Session& ses = S->sessions[id];
    ses.id = id;
    ses.h = h;
    inc_view(h, &ses.view);
    {
        int l = ses.view.v.link;   // rules the merged kernel is instantiated for
        ses.mergeable = l == GCONN_LINK_ASYNC || l == GCONN_LINK_HOOKS || l == GCONN_LINK_EARLY ||
                        l == GCONN_LINK_REMCAS || l == GCONN_LINK_JTB || l == GCONN_LINK_ECLCC;
    }
    *session = id;
    return GCONN_OK;
}

extern "C" gconn_status gconn_server_submit(gconn_server* S, uint32_t session, int op, uint64_t count,
                                            const uint32_t* pairs, uint8_t* result, uint64_t* ticket) {
    if (!S || !ticket || (op != GCONN_OP_INSERT && op != GCONN_OP_QUERY)) return GCONN_E_INVAL;
    if ((count && !pairs) || count > GC_MAX_COUNT) return GCONN_E_INVAL;
    if (op == GCONN_OP_QUERY && count && !result) return GCONN_E_INVAL;
    // where the kernels can use the client's buffers in place (device memory,
    // or host memory the device reads directly), a step skips its staging
    auto usable = [](const void* p) -> const void* { return !p ? nullptr : is_device_ptr(p) ? p : host_direct(p); };
    // the pointer queries answer for the calling thread's current device: ask
    // as the server's device, then give the caller its device back
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
        cudaGetLastError();
        prev = -1;
    }
    if (prev != S->device) cudaSetDevice(S->device);
    const uint32_t* d_pairs = (const uint32_t*)usable(pairs);
    uint8_t* d_result = op == GCONN_OP_QUERY ? (uint8_t*)usable(result) : nullptr;
    if (prev >= 0 && prev != S->device) cudaSetDevice(prev);
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->sessions.find(session);
    if (it == S->sessions.end() || it->second.closing) return GCONN_E_INVAL;
    Request r{S->next_ticket++, session, op, count, pairs, result, Clock::now(), d_pairs, d_result};
    *ticket = r.ticket;
    S->unclaimed.insert(r.ticket);
    if (count == 0) {
        S->done[r.ticket] = {GCONN_OK, 0.0};
        return GCONN_OK;
    }
    it->second.pending.push_back(r);
    S->cv_work.notify_one();
    return GCONN_OK;
}

extern "C" gconn_status gconn_server_wait(gconn_server* S, uint64_t ticket, double* latency_ms) {
    if (!S) return GCONN_E_INVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    // each ticket is waited for once: a second wait (or one for a ticket never
    // issued) is an error instead of a wait that no completion would end
    if (S->unclaimed.erase(ticket) == 0) return GCONN_E_INVAL;
    S->cv_done.wait(lk, [&] { return S->done.count(ticket) > 0; });
    auto d = S->done[ticket];
    S->done.erase(ticket);
    if (latency_ms) *latency_ms = d.latency_ms;
    return d.status;
}

extern "C" gconn_status gconn_server_labels(gconn_server* S, uint32_t session, uint32_t* labels) {
    if (!S) return GCONN_E_INVAL;
    gconn_inc* h = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->sessions.find(session);
        if (it == S->sessions.end()) return GCONN_E_INVAL;
        // drain the session first: its labels reflect every request submitted so far
        S->cv_done.wait(lk, [&] {
            Session& ses = S->sessions[session];
            return ses.pending.empty() && ses.inflight == 0;
        });
        h = it->second.h;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    gconn_status s = gconn_inc_labels(h, labels, nullptr);
    if (s == GCONN_OK) s = read_and_clear_err(nullptr);
    cudaSetDevice(prev);
    return s;
}

extern "C" gconn_status gconn_server_close_session(gconn_server* S, uint32_t session) {
    if (!S) return GCONN_E_INVAL;
    gconn_inc* h = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->sessions.find(session);
        if (it == S->sessions.end()) return GCONN_E_INVAL;
        it->second.closing = true;
        S->cv_done.wait(lk, [&] {
            Session& ses = S->sessions[session];
            return ses.pending.empty() && ses.inflight == 0;
        });
        h = S->sessions[session].h;
        S->sessions.erase(session);
    }
    return gconn_inc_destroy(h);
}

extern "C" gconn_status gconn_server_stats(gconn_server* S, uint64_t* launches, uint64_t* groups,
                                           uint64_t* requests) {
    if (!S) return GCONN_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (launches) *launches = S->launches;
    if (groups) *groups = S->steps;
    if (requests) *requests = S->requests_done;
    return GCONN_OK;
}

extern "C" gconn_status gconn_server_destroy(gconn_server* S) {
    if (!S) return GCONN_E_INVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (auto& kv : S->sessions)
        if (kv.second.h) gconn_inc_destroy(kv.second.h);
    for (StepBuf& b : S->bufs) {
        if (b.st) {
            cudaStreamSynchronize(b.st);
            cudaStreamDestroy(b.st);
        }
        if (b.h_pairs) cudaFreeHost(b.h_pairs);
        if (b.h_out) cudaFreeHost(b.h_out);
        if (b.h_segs) cudaFreeHost(b.h_segs);
        if (b.h_err) cudaFreeHost(b.h_err);
    }
    cudaSetDevice(prev);
    delete S;
    return GCONN_OK;
}
