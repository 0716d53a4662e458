// csr_impl.cuh -- the static CSR pass (Algorithm 1 with sampling, its
// spanning-forest form Algorithm 2) and the static driver, templated on the
// CSR offset type (uint64_t, or uint32_t for graphs with fewer than 2^32
// arcs).  Included by gconn_static.cu (uint64_t offsets and the COO path) and
// gconn_static32.cu (uint32_t offsets): each translation unit instantiates
// its kernels once.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "gc_internal.h"
#include "gc_static.h"
#include "static_kernels.cuh"

namespace gc {

// Every normalised (link, find, splice) triple the library instantiates.
// Calls fn.template operator()<L, F, S, SF>().
template <class Fn>
gconn_status dispatch_uf(int L, int F, int S, bool SF, Fn&& fn) {
#define GC_UF_CASE(l, f, s)                                                              \
    if (L == l && F == f && S == s)                                                      \
        return SF ? fn.template operator()<l, f, s, true>() : fn.template operator()<l, f, s, false>();
    GC_UF_CASE(LK_ASYNC, FD_NAIVE, SP_NONE)
    GC_UF_CASE(LK_ASYNC, FD_COMPRESS, SP_NONE)
    GC_UF_CASE(LK_ASYNC, FD_SPLIT, SP_NONE)
    GC_UF_CASE(LK_ASYNC, FD_HALVE, SP_NONE)
    GC_UF_CASE(LK_HOOKS, FD_NAIVE, SP_NONE)
    GC_UF_CASE(LK_HOOKS, FD_COMPRESS, SP_NONE)
    GC_UF_CASE(LK_HOOKS, FD_SPLIT, SP_NONE)
    GC_UF_CASE(LK_HOOKS, FD_HALVE, SP_NONE)
    GC_UF_CASE(LK_EARLY, FD_NAIVE, SP_NONE)
    GC_UF_CASE(LK_EARLY, FD_COMPRESS, SP_NONE)
    GC_UF_CASE(LK_EARLY, FD_SPLIT, SP_NONE)
    GC_UF_CASE(LK_EARLY, FD_HALVE, SP_NONE)
    GC_UF_CASE(LK_REMCAS, FD_NAIVE, SP_SPLIT_ONE)
    GC_UF_CASE(LK_REMCAS, FD_NAIVE, SP_HALVE_ONE)
    GC_UF_CASE(LK_REMCAS, FD_NAIVE, SP_SPLICE)
    GC_UF_CASE(LK_REMCAS, FD_SPLIT, SP_SPLIT_ONE)
    GC_UF_CASE(LK_REMCAS, FD_SPLIT, SP_HALVE_ONE)
    GC_UF_CASE(LK_REMCAS, FD_SPLIT, SP_SPLICE)
    GC_UF_CASE(LK_REMCAS, FD_HALVE, SP_SPLIT_ONE)
    GC_UF_CASE(LK_REMCAS, FD_HALVE, SP_HALVE_ONE)
    GC_UF_CASE(LK_REMCAS, FD_HALVE, SP_SPLICE)
    GC_UF_CASE(LK_JTB, FD_NAIVE, SP_NONE)
    GC_UF_CASE(LK_JTB, FD_TWOTRY, SP_NONE)
    GC_UF_CASE(LK_REMLOCK, FD_NAIVE, SP_SPLIT_ONE)
    GC_UF_CASE(LK_REMLOCK, FD_NAIVE, SP_HALVE_ONE)
    GC_UF_CASE(LK_REMLOCK, FD_NAIVE, SP_SPLICE)
    GC_UF_CASE(LK_REMLOCK, FD_SPLIT, SP_SPLIT_ONE)
    GC_UF_CASE(LK_REMLOCK, FD_SPLIT, SP_HALVE_ONE)
    GC_UF_CASE(LK_REMLOCK, FD_SPLIT, SP_SPLICE)
    GC_UF_CASE(LK_REMLOCK, FD_HALVE, SP_SPLIT_ONE)
    GC_UF_CASE(LK_REMLOCK, FD_HALVE, SP_HALVE_ONE)
    GC_UF_CASE(LK_REMLOCK, FD_HALVE, SP_SPLICE)
    GC_UF_CASE(LK_AFFOREST, FD_NAIVE, SP_NONE)
#undef GC_UF_CASE
    return GCONN_E_UNSUPPORTED;
}

// Threads per block of the finish kernels: the variant's choice, at most 256
// (their launch bounds).
inline int block_of(const Variant& v) { return v.block > 0 && v.block < 256 ? v.block : 256; }

// ---------------------------------------------------------------- CSR path
struct CsrScratch {
    DevBuf counters, active, small, tasks, over;
};

// HB with a union-find (not JTB) and N <= HB_WARP_N: step 1 is fused into
// the initialisation (k_hb_init) and step 2 runs warp-packed.
inline bool hb_fused(const Variant& v, const UFState& s) {
    return v.sample == GCONN_SAMPLE_HB && v.link != GCONN_LINK_JTB && v.hb_n <= HB_WARP_N && !s.W;
}

// mode_dev: a scratch word for the samples' mode label, taken by block 0 of
// the deferred-union kernel while the other blocks run the deferred unions.
template <class OffT>
gconn_status csr_sample(const Variant& v, const UFState& s, const OffT* off, const uint32_t* cols,
                        uint32_t* lmax_dev, unsigned long long* dq_count, uint32_t* lmax_done, uint32_t* mode_dev,
                        cudaStream_t st) {
    uint32_t n = s.n;
    int L, F, S;
    uf_triple(v, &L, &F, &S);
    int B = block_of(v);
    bool sf = s.sf != nullptr;
    bool jtb = v.link == GCONN_LINK_JTB;
    if (v.sample == GCONN_SAMPLE_KOUT) {
        // deferred long unions: capacity n/8 jobs, overflow runs in place
        DevBuf qbuf;
        uint32_t qcap = n / 8 + 64;
        GC_TRY(qbuf.alloc(sizeof(KoutJob) * (size_t)qcap, st));
        JobQueue dq{qbuf.as<KoutJob>(), dq_count, qcap};   // count zeroed by the init kernel
        GC_TRY(dispatch_uf(L, F, S, sf, [&]<int l, int f, int sp, bool w>() {
            auto k = k_kout<l, f, sp, w, OffT>;
            GC_TRY(launch_pdl("kout", k, grid_for(k, KOUT_BLOCK, n), KOUT_BLOCK, 0, st, off, cols, v.k, s, dq,
                              (v.ablation & GCONN_ABL_PLAIN_SAMPLE) != 0));
            auto kj = k_union_jobs<l, f, sp, w>;
            // the retry kernel also yields L_max (block 0: the samples' mode,
            // the last block: its root)
            return launch_pdl("kout_deferred", kj, std::max(2u, grid_for(kj, LMAX_SAMPLES, qcap)), LMAX_SAMPLES, 0, st, s,
                              dq, v.seed, lmax_dev, lmax_done, mode_dev);
        }));
        return GCONN_OK;
    } else if (hb_fused(v, s)) {   // step 1 already done by k_hb_init
        DevBuf qbuf;
        uint32_t qcap = n / 8 + 64;
        GC_TRY(qbuf.alloc(sizeof(KoutJob) * (size_t)qcap, st));
        JobQueue dq{qbuf.as<KoutJob>(), dq_count, qcap};   // count zeroed by the init kernel
        return dispatch_uf(L, F, S, sf, [&]<int l, int f, int sp, bool w>() {
            auto k = k_hb2w<l, f, sp, w, OffT>;
            GC_TRY(launch_pdl("hb2", k, grid_for(k, 256, n), 256, 0, st, off, cols, v.hb_n, s, dq));
            auto kj = k_union_jobs<l, f, sp, w>;
            // the retry kernel also yields L_max (block 0: the samples' mode,
            // the last block: its root)
            return launch_pdl("hb_deferred", kj, std::max(2u, grid_for(kj, LMAX_SAMPLES, qcap)), LMAX_SAMPLES, 0, st, s,
                              dq, v.seed, lmax_dev, lmax_done, mode_dev);
        });
    } else if (v.sample == GCONN_SAMPLE_HB) {
        GC_TRY(launch("hb1", k_hb1<OffT>, grid_for(k_hb1<OffT>, 256, n), 256, 0, st, off, cols, n, s.P, s.sf,
                      s.err));
        if (jtb) {
            UFState sp = s;
            sp.W = nullptr;
            GC_TRY(launch("compress", k_compress<LK_ASYNC>, grid_for(k_compress<LK_ASYNC>, 256, n), 256, 0, st, sp));
            GC_TRY(launch("w_from_p", k_w_from_p, grid_for(k_w_from_p, 256, n), 256, 0, st, n, s.P, s.W));
        }
        GC_TRY(dispatch_uf(L, F, S, sf, [&]<int l, int f, int sp, bool w>() {
            auto k = k_hb2<l, f, sp, w, OffT>;
            return launch("hb2", k, grid_for(k, B, n), B, 0, st, off, cols, v.hb_n, s);
        }));
    } else if (v.sample == GCONN_SAMPLE_BFS) {
        return bfs_sample(v, s, off, cols, lmax_dev, st);   // also yields L_max
    }
    // the full compression after sampling is fused into vertex gathering
    if (jtb)
        return launch_pdl("lmax", k_lmax<LK_JTB>, 1, LMAX_SAMPLES, 0, st, s, v.seed, lmax_dev);
    return launch_pdl("lmax", k_lmax<LK_ASYNC>, 1, LMAX_SAMPLES, 0, st, s, v.seed, lmax_dev);
}

// Runs the sampling phase (unless NONE), L_max, vertex gathering and the
// finish phase of Algorithm 1 on CSR.  Leaves P (or W) final, not finalised.
// Counters of the sampling phase for gconn_cc_csr_stats (Section 4.3, Table 4).
struct CsrStats {
    unsigned long long* d;        // device counters, see k_sample_stats
    cudaEvent_t t_sampled;        // recorded after sampling + L_max + gathering
    cudaEvent_t t_counted;        // recorded after the counting kernel (excluded from the times)
    uint32_t* lmax;               // device scalar, copied out by the caller
};

// After sampling and compression (P[v] = sampled root): vertices labelled
// L_max, sampled components (roots), active vertices and their arcs, arcs
// whose endpoints carry different sampled labels, and arcs the sampling step
// inspected.
template <class OffT>
static __global__ void k_sample_stats(const OffT* __restrict__ off, const uint32_t* __restrict__ cols,
                                      const uint32_t* P, uint32_t n, const uint32_t* lmax_p, int sample, int k,
                                      int hb_n, unsigned long long* c) {
    uint32_t lmax = lmax_p ? *lmax_p : GC_DINF;
    unsigned long long cov = 0, roots = 0, act = 0, act_arcs = 0, inter = 0, insp = 0;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t lv = P[v];
        uint64_t lo = off[v], hi = off[v + 1], deg = hi - lo;
        cov += lv == lmax;
        roots += lv == (uint32_t)v;
        if (lv != lmax && deg) {
            act += 1;
            act_arcs += deg;
        }
        for (uint64_t a = lo; a < hi; ++a) inter += P[cols[a]] != lv;
        if (sample == GCONN_SAMPLE_KOUT) insp += deg < (uint64_t)k ? deg : (uint64_t)k;
        if (sample == GCONN_SAMPLE_HB) insp += (deg > 0) + (lv == (uint32_t)v ? (deg < (uint64_t)hb_n ? deg : hb_n) : 0);
    }
    atomicAdd(c + 0, cov);
    atomicAdd(c + 1, roots);
    atomicAdd(c + 2, act);
    atomicAdd(c + 3, act_arcs);
    atomicAdd(c + 4, inter);
    atomicAdd(c + 5, insp);
}

// With `finalized` non-null, a union-find finish also finalises the labels in
// P (from the gathered lists, k_finalize_gathered) and sets *finalized.
template <class OffT>
gconn_status csr_connect(const Variant& v, const UFState& s, const OffT* off, const uint32_t* cols,
                         cudaStream_t st, CsrStats* stats = nullptr, bool* finalized = nullptr) {
    uint32_t n = s.n;
    if (n == 0) return GCONN_OK;
    CsrScratch sc;
    bool sampled = v.sample != GCONN_SAMPLE_NONE;
    // the pass's counters in one 64-byte header, cleared by the init kernel:
    // [0] L_max, [1..3] gathering counters, [4] the samples' mode label,
    // [8..9] deferred-union count (u64), [10] blocks of the retry kernel done
    // (the last one resolves L_max)
    GC_TRY(sc.counters.alloc(16 * sizeof(uint32_t), st));
    uint32_t* hdr = sc.counters.as<uint32_t>();
    uint32_t* lmax = sampled ? hdr : nullptr;
    uint32_t* cnt = hdr + 1;
    unsigned long long* dq_count = reinterpret_cast<unsigned long long*>(hdr + 8);
    // the rounds-based finishes (SV, LT) sample with Union-Async
    Variant sv = v;
    bool rounds = is_rounds_link(v.link);
    if (rounds) { sv.link = GCONN_LINK_ASYNC; sv.find = GCONN_FIND_NAIVE; sv.splice = 0; }
    bool jtb = sv.link == GCONN_LINK_JTB;
    if (hb_fused(sv, s)) {   // InitLabel and HB step 1 in one pass
        GC_TRY(launch_pdl("init", k_hb_init<OffT>, grid_for(k_hb_init<OffT>, 256, n), 256, 0, st, off, cols, n, s.P,
                          s.H, s.sf, s.err, hdr, 16u));
    } else {
        GC_TRY(init_state(s, st, hdr, 16));
    }
    if (sampled) GC_TRY(csr_sample(sv, s, off, cols, lmax, dq_count, hdr + 10, hdr + 4, st));
    if (v.ablation & GCONN_ABL_NO_VG) {   // measurement form: full compression, then the plain finish
        if (rounds || sv.link == GCONN_LINK_JTB || stats) return GCONN_E_UNSUPPORTED;
        GC_TRY(compress_all(sv, s, st));
        int L, F, S;
        uf_triple(v, &L, &F, &S);
        int B = block_of(v);
        return dispatch_uf(L, F, S, s.sf != nullptr, [&]<int l, int f, int sp, bool w>() {
            auto k = k_finish_plain<l, f, sp, w, OffT>;
            return launch_pdl("finish", k, grid_for(k, B, n), B, 0, st, off, cols, s, (const uint32_t*)lmax);
        });
    }
    // vertex gathering
    // task ids and the task counter are uint32 on the device: clamp (overflowing
    // vertices go to the per-block overflow list)
    uint64_t task_cap = std::min<uint64_t>((uint64_t)n + 1024, 0xFFFFFFFFull);
    uint32_t* active = nullptr;
    if (sampled) {
        GC_TRY(sc.active.alloc(sizeof(uint32_t) * (((size_t)n + 31) / 32), st));
        active = sc.active.as<uint32_t>();
    }
    GC_TRY(sc.small.alloc(sizeof(uint32_t) * (size_t)n, st));
    GC_TRY(sc.tasks.alloc(sizeof(unsigned long long) * task_cap, st));
    GC_TRY(sc.over.alloc(sizeof(uint32_t) * (size_t)n, st));
    uint32_t* small = sc.small.as<uint32_t>();
    unsigned long long* tasks = sc.tasks.as<unsigned long long>();
    uint32_t* over = sc.over.as<uint32_t>();
    bool vec = !jtb && ((uintptr_t)off & 15u) == 0 && ((uintptr_t)s.P & 15u) == 0;
    {
        auto k = jtb ? k_vg<LK_JTB, true, OffT> : vec ? k_vg4<LK_ASYNC, OffT> : k_vg<LK_ASYNC, true, OffT>;
        GC_TRY(launch_pdl("vg", k, grid_for(k, 256, vec ? ((uint64_t)n + 3) / 4 : (uint64_t)n), 256, 0, st, off, s,
                          lmax, active, small, cnt + 0, tasks, (uint32_t)task_cap, cnt + 1, over, cnt + 2));
    }
    if (stats) {
        GC_CUDA(cudaEventRecord(stats->t_sampled, st));
        if (lmax) GC_CUDA(cudaMemcpyAsync(stats->lmax, lmax, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
        if (!jtb)
            GC_TRY(launch("sample_stats", k_sample_stats<OffT>, grid_for(k_sample_stats<OffT>, 256, n), 256, 0, st,
                          off, cols, (const uint32_t*)s.P, n, (const uint32_t*)lmax, v.sample, v.k, v.hb_n, stats->d));
        GC_CUDA(cudaEventRecord(stats->t_counted, st));
    }
    if (rounds) return rounds_csr(v, s, off, cols, active, small, cnt + 0, tasks, cnt + 1, (uint32_t)task_cap,
                                  over, cnt + 2, st);
    int L, F, S;
    uf_triple(v, &L, &F, &S);
    int B = block_of(v);
    GC_TRY(dispatch_uf(L, F, S, s.sf != nullptr, [&]<int l, int f, int sp, bool w>() {
        auto k = k_finish<l, f, sp, w, OffT>;
        return launch_pdl("finish", k, grid_for(k, B, (uint64_t)n * 32), B, 0, st, off, cols, s,
                      (const uint32_t*)active, (const uint32_t*)small, (const uint32_t*)(cnt + 0),
                      (const unsigned long long*)tasks, (const uint32_t*)(cnt + 1), (uint32_t)task_cap,
                      (const uint32_t*)over, (const uint32_t*)(cnt + 2));
    }));
    if (finalized && !jtb) {   // the lists are freed with this call's scratch: finalise now
        GC_TRY(launch_pdl("finalize", k_finalize_gathered, grid_for(k_finalize_gathered, 256, n), 256, 0, st, s,
                          (const uint32_t*)lmax, (const uint32_t*)small, (const uint32_t*)(cnt + 0),
                          (const unsigned long long*)tasks, (const uint32_t*)(cnt + 1), (uint32_t)task_cap,
                          (const uint32_t*)over, (const uint32_t*)(cnt + 2)));
        *finalized = true;
    }
    return GCONN_OK;
}

// --------------------------------------------------------------- drivers
template <class OffT>
static gconn_status static_run(uint32_t n, uint64_t m, const uint32_t* edges, const OffT* off,
                               const uint32_t* cols, uint32_t* labels, uint64_t* forest, uint64_t* forest_count,
                               const gconn_variant* vin, int want_forest, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    bool csr = off != nullptr;
    if (n == 0xFFFFFFFFu) return GCONN_E_INVAL;
    Variant v;
    GC_TRY(resolve_variant(vin, csr ? 1 : 0, want_forest, &v));
    if (want_forest && (!forest || !forest_count)) return GCONN_E_INVAL;
    if (!want_forest && !labels && n) return GCONN_E_INVAL;
    if (csr && !off) return GCONN_E_INVAL;
    if (!csr && m && !edges) return GCONN_E_INVAL;
    if (!csr && want_forest && m >= 0xFFFFFFFFull) return GCONN_E_INVAL;
    if (!csr && m > GC_MAX_COUNT) return GCONN_E_INVAL;
    // edges are read as 8-byte pairs, offsets as whole words
    if (!csr && edges && ((uintptr_t)edges & 7u)) return GCONN_E_INVAL;
    if (csr && ((uintptr_t)off & (sizeof(OffT) - 1))) return GCONN_E_INVAL;
    if (csr && cols && ((uintptr_t)cols & 3u)) return GCONN_E_INVAL;
    if (n == 0) {
        if (!csr && m) return GCONN_E_RANGE;
        if (want_forest) {
            uint64_t z = 0;
            if (is_device_ptr(forest_count)) GC_CUDA(cudaMemcpyAsync(forest_count, &z, 8, cudaMemcpyHostToDevice, st));
            else *forest_count = 0;
        }
        return GCONN_OK;
    }
    int dev = 0;
    GC_CUDA(cudaGetDevice(&dev));
    (void)dev;

    // stage inputs
    DevBuf ebuf, obuf, cbuf, lbuf, pbuf, hbuf, wbuf, sfbuf;
    const uint32_t* d_edges = edges;
    const OffT* d_off = off;
    const uint32_t* d_cols = cols;
    bool any_host = false;
    if (!csr) {
        if (m) {
            bool h = !is_device_ptr(edges);
            any_host |= h;
            // a union-find finish reads every edge once: host edges are read
            // in place where the device can; the round finishes re-read them
            if (is_rounds_link(v.link))
                GC_TRY(stage_in(edges, sizeof(uint32_t) * 2 * m, st, ebuf, (const void**)&d_edges));
            else
                GC_TRY(stage_in_once(edges, sizeof(uint32_t) * 2 * m, st, ebuf, (const void**)&d_edges));
        }
    } else {
        OffT narcs = 0;
        bool oh = !is_device_ptr(off);
        if (!cols) {   // allowed only for a graph without arcs
            if (oh) narcs = off[n];
            else {
                GC_CUDA(cudaMemcpyAsync(&narcs, off + n, sizeof(OffT), cudaMemcpyDeviceToHost, st));
                GC_CUDA(cudaStreamSynchronize(st));
            }
            if (narcs) return GCONN_E_INVAL;
        }
        if (oh) {
            narcs = off[n];
            any_host = true;
            // offsets are read by several kernels: staged; the columns are read
            // in place where the device can (sampling reads k per row, the
            // finish only the active rows)
            GC_TRY(stage_in(off, sizeof(OffT) * ((size_t)n + 1), st, obuf, (const void**)&d_off));
            if (narcs)
                GC_TRY(stage_in_once(cols, sizeof(uint32_t) * (uint64_t)narcs, st, cbuf, (const void**)&d_cols));
        } else if (!is_device_ptr(cols)) {
            GC_CUDA(cudaMemcpyAsync(&narcs, off + n, sizeof(OffT), cudaMemcpyDeviceToHost, st));
            GC_CUDA(cudaStreamSynchronize(st));
            any_host = true;
            if (narcs)
                GC_TRY(stage_in_once(cols, sizeof(uint32_t) * (uint64_t)narcs, st, cbuf, (const void**)&d_cols));
        }
    }
    // parent array: the caller's labels buffer when it is device memory
    uint32_t* P = nullptr;
    bool labels_host = labels && !is_device_ptr(labels);
    any_host |= labels_host;
    if (labels && !labels_host) {
        P = labels;
    } else {
        GC_TRY(pbuf.alloc(sizeof(uint32_t) * (size_t)n, st));
        P = pbuf.as<uint32_t>();
    }
    uint32_t* H = nullptr;
    u64w* W = nullptr;
    uint32_t* sf = nullptr;
    if (v.link == GCONN_LINK_HOOKS) { GC_TRY(hbuf.alloc(sizeof(uint32_t) * (size_t)n, st)); H = hbuf.as<uint32_t>(); }
    if (v.link == GCONN_LINK_JTB) { GC_TRY(wbuf.alloc(sizeof(u64w) * (size_t)n, st)); W = wbuf.as<u64w>(); }
    if (want_forest) { GC_TRY(sfbuf.alloc(sizeof(uint32_t) * (size_t)n, st)); sf = sfbuf.as<uint32_t>(); }
    DevBuf lkbuf;

    UFState s = make_state(n, P, H, W, sf, v);
    if (v.link == GCONN_LINK_REMLOCK) {
        GC_TRY(lkbuf.alloc(sizeof(uint32_t) * (size_t)n, st));
        s.Lk = lkbuf.as<uint32_t>();
        GC_CUDA(cudaMemsetAsync(s.Lk, 0, sizeof(uint32_t) * (size_t)n, st));
    }
    L2Window l2win;
    l2win.apply(st, P, sizeof(uint32_t) * (size_t)n);
    if (!csr) GC_TRY(init_state(s, st));   // csr_connect initialises P and its counters
    if (csr && want_forest)
        GC_TRY(launch("check_arcs", k_check_arcs<OffT>, 1, 1, 0, st, d_off, n, s.err));

    if (!csr) {
        if (is_rounds_link(v.link)) {
            GC_TRY(rounds_coo(v, s, d_edges, nullptr, m, st));
        } else {
            GC_TRY(union_coo(v, s, d_edges, m, 0, st));
        }
    }
    bool finalized = false;
    if (csr) GC_TRY(csr_connect(v, s, d_off, d_cols, st, nullptr, labels ? &finalized : nullptr));
    if (labels) {
        // rounds-based finishes leave P fully compressed and min-rooted
        if (!finalized) GC_TRY(finalize_labels(v, s, P, st));
        if (labels_host) GC_CUDA(cudaMemcpyAsync(labels, P, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost, st));
    }
    if (want_forest) {
        GC_TRY(sf_output(n, sf, forest, forest_count, st));
        any_host |= !is_device_ptr(forest) || !is_device_ptr(forest_count);
    }
    if (any_host) return read_and_clear_err(st);
    return GCONN_OK;
}


}  // namespace gc
