// gconn_serve.cu -- a serving loop over device-resident incremental
// connectivity (Section 3.5): clients submit insert and query batches for
// sessions (one union-find forest each); a worker thread admits them as
// device memory and stream slots free up, coalesces consecutive requests of
// the same session and kind into one launch, runs different sessions'
// launches concurrently on separate streams, and completes each request with
// its host-measured latency.
//
// Ordering per session keeps the incremental semantics exact: requests form
// phases of consecutive inserts or consecutive queries; a phase starts only
// after the previous phase of that session has finished on the device, so a
// query sees exactly the inserts submitted before it.  Inserts of one phase
// commute and queries of one phase only compress, so coalescing and running
// them together changes no answer.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "gc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    uint32_t session;
    int op;                       // GCONN_OP_INSERT / GCONN_OP_QUERY
    uint64_t count;
    const uint32_t* pairs;        // host
    uint8_t* result;              // host, queries only
    Clock::time_point submitted;
};

struct Group;

struct Session {
    uint32_t id;
    gconn_inc* h = nullptr;
    std::deque<Request> pending;
    int inflight_phase = -1;      // op of the groups in flight, -1 = none
    int inflight_groups = 0;
    bool closing = false;
};

struct Slot {
    cudaStream_t st = nullptr;
    uint32_t* h_in = nullptr;     // pinned staging (pairs)
    uint8_t* h_out = nullptr;     // pinned staging (query answers)
    bool busy = false;
};

struct Group {
    uint32_t session;
    int op;
    int slot;
    std::vector<Request> reqs;
    uint64_t total = 0;           // pairs in the group
    uint64_t bytes = 0;           // device bytes held
    void* d_in = nullptr;
    uint8_t* d_out = nullptr;
    cudaEvent_t done = nullptr;
    gconn_status status = GCONN_OK;
};

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
    std::map<uint32_t, Session> sessions;
    std::vector<Slot> slots;
    std::deque<std::unique_ptr<Group>> inflight;
    uint64_t bytes_inflight = 0;
    struct Done {
        gconn_status status;
        double latency_ms;
    };
    std::map<uint64_t, Done> done;
    uint64_t launches = 0, groups = 0, requests_done = 0;
};

namespace {

using namespace gc;

// Launch a formed group on its slot (called by the worker without the lock
// held for the CUDA calls; the group is owned by the worker until completion).
gconn_status launch_group(gconn_server* S, Session& ses, Group& g) {
    Slot& sl = S->slots[g.slot];
    cudaStream_t st = sl.st;
    const uint64_t cap = S->cfg.slot_pairs;
    GC_CUDA(cudaMallocAsync(&g.d_in, sizeof(uint32_t) * 2 * g.total, st));
    if (g.op == GCONN_OP_QUERY) GC_CUDA(cudaMallocAsync((void**)&g.d_out, g.total, st));
    // pack the requests' pairs into the slot's pinned buffer; one host-to-device
    // copy per full buffer (the buffer is reused only after its copy finished)
    uint64_t fill = 0, dev_pos = 0;
    auto flush = [&]() -> gconn_status {
        if (!fill) return GCONN_OK;
        GC_CUDA(cudaMemcpyAsync((uint32_t*)g.d_in + 2 * dev_pos, sl.h_in, sizeof(uint32_t) * 2 * fill,
                                cudaMemcpyHostToDevice, st));
        dev_pos += fill;
        fill = 0;
        return GCONN_OK;
    };
    for (const Request& r : g.reqs) {
        uint64_t done = 0;
        while (done < r.count) {
            if (fill == cap) {
                GC_TRY(flush());
                GC_CUDA(cudaStreamSynchronize(st));
            }
            uint64_t c = r.count - done < cap - fill ? r.count - done : cap - fill;
            memcpy(sl.h_in + 2 * fill, r.pairs + 2 * done, sizeof(uint32_t) * 2 * c);
            fill += c;
            done += c;
        }
    }
    GC_TRY(flush());
    if (g.op == GCONN_OP_INSERT) {
        GC_TRY(gconn_inc_insert_batch(ses.h, g.total, (const uint32_t*)g.d_in, st));
    } else {
        GC_TRY(gconn_inc_query(ses.h, g.total, (const uint32_t*)g.d_in, g.d_out, st));
    }
    S->launches++;
    GC_CUDA(cudaFreeAsync(g.d_in, st));
    GC_CUDA(cudaEventRecord(g.done, st));
    return GCONN_OK;
}

// Copy a finished query group's answers back to each request's buffer.
gconn_status finish_group(gconn_server* S, Group& g) {
    Slot& sl = S->slots[g.slot];
    if (g.op != GCONN_OP_QUERY || g.status != GCONN_OK) {
        if (g.d_out) cudaFreeAsync(g.d_out, sl.st);
        return g.status;
    }
    const uint64_t cap = S->cfg.slot_pairs;
    uint64_t pos = 0;
    for (const Request& r : g.reqs) {
        uint64_t done = 0;
        while (done < r.count) {
            uint64_t c = r.count - done < cap ? r.count - done : cap;
            GC_CUDA(cudaMemcpyAsync(sl.h_out, g.d_out + pos + done, c, cudaMemcpyDeviceToHost, sl.st));
            GC_CUDA(cudaStreamSynchronize(sl.st));
            memcpy(r.result + done, sl.h_out, c);
            done += c;
        }
        pos += r.count;
    }
    GC_CUDA(cudaFreeAsync(g.d_out, sl.st));
    return GCONN_OK;
}

void worker_loop(gconn_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // 1. completions
        bool progressed = false;
        for (auto it = S->inflight.begin(); it != S->inflight.end();) {
            Group& g = **it;
            cudaError_t q = cudaEventQuery(g.done);
            if (q == cudaErrorNotReady) {
                ++it;
                continue;
            }
            lk.unlock();
            if (q != cudaSuccess) g.status = cuda_status(q);
            gconn_status fs = finish_group(S, g);
            gconn_status es = read_and_clear_err(S->slots[g.slot].st);
            lk.lock();
            if (g.status == GCONN_OK) g.status = fs != GCONN_OK ? fs : es;
            auto now = Clock::now();
            for (const Request& r : g.reqs) {
                double ms = std::chrono::duration<double, std::milli>(now - r.submitted).count();
                S->done[r.ticket] = {g.status, ms};
                S->requests_done++;
            }
            S->slots[g.slot].busy = false;
            S->bytes_inflight -= g.bytes;
            Session& ses = S->sessions[g.session];
            if (--ses.inflight_groups == 0) ses.inflight_phase = -1;
            cudaEventDestroy(g.done);
            it = S->inflight.erase(it);
            progressed = true;
        }
        if (progressed) S->cv_done.notify_all();
        // 2. admissions: round-robin over sessions, one group per session per pass
        bool launched = false;
        for (auto& kv : S->sessions) {
            Session& ses = kv.second;
            if (ses.pending.empty()) continue;
            int op = ses.pending.front().op;
            if (ses.inflight_phase != -1 && ses.inflight_phase != op) continue;   // previous phase still running
            int slot = -1;
            for (size_t i = 0; i < S->slots.size(); ++i)
                if (!S->slots[i].busy) { slot = (int)i; break; }
            if (slot < 0) break;
            auto g = std::make_unique<Group>();
            g->session = ses.id;
            g->op = op;
            g->slot = slot;
            while (!ses.pending.empty() && ses.pending.front().op == op) {
                const Request& r = ses.pending.front();
                uint64_t need = (sizeof(uint32_t) * 2 + (op == GCONN_OP_QUERY ? 1 : 0)) * r.count;
                bool first = g->reqs.empty();
                if (!first && (g->total + r.count > S->cfg.coalesce_pairs ||
                               S->bytes_inflight + g->bytes + need > S->cfg.device_budget_bytes))
                    break;
                if (first && S->bytes_inflight > 0 && S->bytes_inflight + need > S->cfg.device_budget_bytes)
                    break;   // wait for memory (a lone request larger than the budget still runs alone)
                g->reqs.push_back(r);
                g->total += r.count;
                g->bytes += need;
                ses.pending.pop_front();
            }
            if (g->reqs.empty()) continue;
            S->slots[slot].busy = true;
            S->bytes_inflight += g->bytes;
            ses.inflight_phase = op;
            ses.inflight_groups++;
            S->groups++;
            cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming);
            Group* gp = g.get();
            S->inflight.push_back(std::move(g));
            lk.unlock();
            gp->status = launch_group(S, ses, *gp);
            if (gp->status != GCONN_OK) cudaEventRecord(gp->done, S->slots[slot].st);
            lk.lock();
            launched = true;
        }
        if (S->stop && S->inflight.empty()) {
            bool any = false;
            for (auto& kv : S->sessions) any |= !kv.second.pending.empty();
            if (!any) break;
        }
        if (!launched && !progressed) {
            if (S->inflight.empty()) S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            else S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" gconn_status gconn_server_config_default(gconn_server_config* c) {
    if (!c) return GCONN_E_INVAL;
    c->device_budget_bytes = 4ull << 30;
    c->slots = 8;
    c->coalesce_pairs = 1u << 22;
    c->slot_pairs = 1u << 22;
    return GCONN_OK;
}

extern "C" gconn_status gconn_server_create(const gconn_server_config* cfg, gconn_server** out) {
    if (!out) return GCONN_E_INVAL;
    *out = nullptr;
    gconn_server_config c;
    gconn_server_config_default(&c);
    if (cfg) c = *cfg;
    if (c.slots < 1 || c.slots > 64 || c.slot_pairs < 1024 || c.coalesce_pairs < 1 || c.device_budget_bytes < 1)
        return GCONN_E_INVAL;
    gconn_server* S = new gconn_server();
    S->cfg = c;
    cudaGetDevice(&S->device);
    if (!err_word()) {
        delete S;
        return GCONN_E_CUDA;
    }
    S->slots.resize(c.slots);
    for (Slot& sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&sl.h_in, sizeof(uint32_t) * 2 * c.slot_pairs) != cudaSuccess ||
            cudaMallocHost(&sl.h_out, c.slot_pairs) != cudaSuccess) {
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
    *session = id;
    return GCONN_OK;
}

extern "C" gconn_status gconn_server_submit(gconn_server* S, uint32_t session, int op, uint64_t count,
                                            const uint32_t* pairs, uint8_t* result, uint64_t* ticket) {
    if (!S || !ticket || (op != GCONN_OP_INSERT && op != GCONN_OP_QUERY)) return GCONN_E_INVAL;
    if (count && !pairs) return GCONN_E_INVAL;
    if (op == GCONN_OP_QUERY && count && !result) return GCONN_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->sessions.find(session);
    if (it == S->sessions.end() || it->second.closing) return GCONN_E_INVAL;
    Request r{S->next_ticket++, session, op, count, pairs, result, Clock::now()};
    *ticket = r.ticket;
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
    if (ticket == 0 || ticket >= S->next_ticket) return GCONN_E_INVAL;
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
            return ses.pending.empty() && ses.inflight_groups == 0;
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
            return ses.pending.empty() && ses.inflight_groups == 0;
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
    if (groups) *groups = S->groups;
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
    for (Slot& sl : S->slots) {
        if (sl.st) {
            cudaStreamSynchronize(sl.st);
            cudaStreamDestroy(sl.st);
        }
        if (sl.h_in) cudaFreeHost(sl.h_in);
        if (sl.h_out) cudaFreeHost(sl.h_out);
    }
    cudaSetDevice(prev);
    delete S;
    return GCONN_OK;
}
