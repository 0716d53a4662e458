"""Benchmark: static connected components on an RMAT scale-22 graph, plus the
incremental insert/query stream, through libgconn on GB300.

One step = one full static CC pass of the two-phase method (sampling, L_max,
vertex gathering, finish, finalisation) over the resident CSR of an RMAT
graph with 2^22 vertices and 2^26 undirected edges (Graph500 a,b,c,d =
.57,.19,.19,.05, ids randomly permuted, self-loops and duplicates kept).
edges/s counts the 2^26 undirected input edges per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torchrun) every rank runs its own replica
graph (seed + rank): the static problem does not shard without an exchange
step, so scaling is weak and there is no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402

SCALE = 22
M_EDGES = 1 << 26
SEED_STATIC = 0x6C0A0002          # per-config seed: base 0x6C0A0001 + config index
SEED_INC = 0x6C0A0005
SEED_BATCH = 0x6C0A0004
SEED_SERVE = 0x6C0A0006
INC_N_SCALE = 24
INC_TOTAL = 1 << 28
L2_FLUSH_BYTES = 256 << 20        # > 126 MB L2
DEFAULT_VARIANT = "kout/remcas/naive/split_one"
# DRAM bytes (read + write) of one k_kout launch per vertex, from an ncu capture
# of the default variant at RMAT scale 20, edge factor 16 (41.984 MB read +
# 0.383 MB written, / 2^20); valid while that kernel is unchanged.
KOUT_DRAM_BYTES_PER_VERTEX = 38.268416e6 / 2 ** 20   # uint32 offsets: 37.789 MB read + 0.479 MB written
KOUT_DRAM_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_kout launch at RMAT scale 20 "
                    "(same variant and edge factor), scaled by the vertex count")


def parse_variant(g, spec: str):
    parts = spec.split("/")
    sample, link = parts[0], parts[1]
    find = parts[2] if len(parts) > 2 else "naive"
    splice = parts[3] if len(parts) > 3 else "none"
    kw = dict(sample=sample, link=link)
    if link == "lt":
        kw["lt"] = find.upper()
    else:
        kw["find"] = find
        kw["splice"] = splice
    return g.make_variant(**kw)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def wait_first(self, timeout=5.0):
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.02)

    def stop(self, t_from=None, t_to=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in self.lines:
            if t_from is not None and not (t_from <= ts <= t_to):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ input build
def make_static_input(rank: int, scale: int = SCALE, m: int = M_EDGES):
    seed = replica_seed(rank)
    e = graphgen.rmat(scale, m, seed)
    n = 1 << scale
    off, cols = graphgen.csr(n, e)
    return n, e, off, cols, seed


def inc_batches(seed: int, total: int = INC_TOTAL, lo: float = 3.0, hi: float = 8.0):
    """Insert-batch sizes floor(10^(lo+(hi-lo)U)) (default: log-uniform in
    [10^3, 10^8]) until `total` (last one truncated)."""
    h = graphgen.hash_fill(seed, 11, 0, 1 << 20)
    sizes, tot = [], 0
    for x in h:
        u = (int(x) >> 11) * 2.0 ** -53
        b = int(10 ** (lo + (hi - lo) * u))
        b = min(b, total - tot)
        sizes.append(b)
        tot += b
        if tot >= total:
            break
    return sizes


# ------------------------------------------------------------ roofline
def alg_bytes(name: str, st: dict):
    """Algorithmic DRAM bytes of one launch of a kernel: what the executed
    variant must move at least once, by the per-unit terms of the method's
    measurement model (random-access sector amplification not counted, nor the
    arcs that sampling avoids):
      init 4n (P[v] = v); k-out sampling 4(n+1) + 4kn (uint32 offsets, k
      columns per vertex); vertex gathering 4n (one read of the labels);
      CSR finish 4 * (arcs of active vertices) + 8 * (active vertices);
      finalisation 8n (read + write); full compression 8n; COO finish 8m.
    Kernels outside the model (the deferred-union retry) count 0."""
    n = st["n"]
    if name == "init":
        return 4 * n
    if name == "kout":
        return 4 * (n + 1) + 4 * st.get("k", 2) * n
    if name == "vg":
        return 4 * n
    if name == "finish":
        return 4 * st.get("active_arcs", 0) + 8 * st.get("active_vertices", 0)
    if name in ("compress", "finalize"):
        return 8 * n
    if name == "union_coo":
        return 8 * st["m"]
    return None


def roofline(bytes_, ms, hbm, peak_src, **extra):
    ach = bytes_ / (ms * 1e-3) / 1e9
    d = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
         "alg_bytes": int(bytes_), "peak_source": peak_src}
    d.update(extra)
    return d


def profile_table(g):
    prof = g.gconn_profile_get()
    return {k: {"launches": c, "ms": ms} for k, (c, ms) in prof.items()}


def pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * p / 100.0
    lo, hi = int(np.floor(k)), int(np.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


# ------------------------------------------------------------ ranks
def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """Slowest rank's time: the whole job is done only when every replica is."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank: int) -> int:
    """Each rank's replica graph: same shape, its own seed."""
    return SEED_STATIC + 1000 * rank


# ------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2008_11839_gb300 as g

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    g.build()
    g.lib()
    dev = torch.device("cuda", local_rank)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    n, e, off, cols, seed = make_static_input(rank, args.scale, args.edges)
    M = args.edges
    deg = np.diff(off).astype(np.int64)
    st = {"n": n, "m": M, "narcs": int(off[-1]), "kout_arcs": int(np.minimum(deg, 2).sum()), "k": 2}
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    off32 = off.astype(np.uint32)                      # 2m < 2^32 arcs: uint32 offsets
    d_off32 = torch.from_numpy(off32.view(np.int32)).to(dev)
    d_cols = torch.from_numpy(cols.view(np.int32)).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    v = parse_variant(g, args.variant)
    stream = torch.cuda.current_stream()
    # the finish's algorithmic bytes need the active set that sampling leaves:
    # one untimed counting pass of the same variant and seed
    try:
        cs = g.gconn_cc_csr_stats(n, d_off, d_cols, labels, v, stream)
        st["active_vertices"], st["active_arcs"] = int(cs.active_vertices), int(cs.active_arcs)
    except g.GconnError:
        pass
    # One static pass is captured once into a CUDA graph.  Every timed kernel
    # adds two event-record nodes, and each serialises the replay for a few
    # microseconds (and breaks the programmatic-launch overlap around it), so
    # three plans of the same pass are replayed: (1) every kernel bracketed,
    # for the per-kernel shares (a separate replay loop); (2) no event nodes:
    # the timed region, timed by events around each replay; (3) one event pair
    # around the dominant kernel, replayed as often right after the timed
    # region, for that kernel's live duration (the roofline).
    def make_plan(select, profiled=True):
        if not profiled:
            return g.gconn_plan_create_cc_csr32(n, d_off32, d_cols, labels, v)
        g.gconn_profile_select(select)
        g.gconn_profile_enable(True)
        p = g.gconn_plan_create_cc_csr32(n, d_off32, d_cols, labels, v)
        g.gconn_profile_enable(False)
        g.gconn_profile_select(None)
        return p

    plan_all = make_plan(None)
    for i in range(args.warmup):
        flush.fill_(i)
        g.gconn_plan_run(plan_all, stream)
        g.gconn_sync(stream)
        g.gconn_profile_sync()
    g.gconn_profile_reset()
    for i in range(args.steps):
        flush.fill_(i + 500)
        g.gconn_plan_run(plan_all, stream)
        g.gconn_sync(stream)
        g.gconn_profile_sync()
    prof_all = profile_table(g)       # per-kernel totals, every kernel bracketed
    g.gconn_profile_reset()
    g.gconn_plan_destroy(plan_all)
    dom_name = max(prof_all.items(), key=lambda kv: kv[1]["ms"])[0] if prof_all else None

    # (2) the timed region: the plain plan (no event nodes) -- the pass a user
    # replays; (3) right after it, the same number of replays of the plan with
    # one event pair around the dominant kernel, for that kernel's live
    # duration (the pair costs the pass its PDL overlap on both sides of the
    # kernel, so it stays out of the timed pass)
    plan = make_plan(None, profiled=False)
    plan_dom = make_plan(dom_name)

    def step():
        g.gconn_plan_run(plan, stream)

    for i in range(args.warmup):
        flush.fill_(i)
        step()
        flush.fill_(i + 100)
        g.gconn_plan_run(plan_dom, stream)
    g.gconn_sync(stream)
    g.gconn_profile_sync()

    # a cheap invariant check here; the labels of the last timed pass are
    # compared bit for bit with the oracle's in the CPU-baseline leg
    lab = labels.cpu().numpy().view(np.uint32)
    ok = bool((lab <= np.arange(n, dtype=np.uint32)).all() and (lab[lab] == lab).all()
              and (lab[e[:4096, 0]] == lab[e[:4096, 1]]).all())

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    g.gconn_profile_reset()
    launches0 = g.gconn_launch_count()
    clocks.start()
    clocks.wait_first()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i + 1000)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = g.gconn_launch_count() - launches0
    lab_timed = labels.cpu().numpy().view(np.uint32).copy()   # the last timed pass's labels
    for i in range(args.steps):      # the dominant kernel's live duration, same workload
        flush.fill_(i + 2000)
        g.gconn_plan_run(plan_dom, stream)
        g.gconn_sync(stream)
        g.gconn_profile_sync()        # the graph's event pair re-records on every replay
    prof = profile_table(g)
    # keep the same step loop running so the 200 ms clock samples see the load
    t_cont = time.perf_counter()
    while time.perf_counter() - t_cont < args.clock_window:
        for i in range(8):
            flush.fill_(i)
            step()
        torch.cuda.synchronize()
    clk = clocks.stop(t0 - 0.05, time.perf_counter())
    g.gconn_profile_reset()
    clk["window"] = (f"timed region + the kernel-timing replays + {args.clock_window:.1f} s continuation "
                     f"of the same step loop")
    g.gconn_sync(stream)
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(x) for s, x in zip(starts, ends)]
    ms = max_over_ranks(float(np.mean(step_ms)), dist, dev)
    g.gconn_plan_destroy(plan)
    g.gconn_plan_destroy(plan_dom)

    # dominant kernel's roofline from its live events in the timed region
    dom = (dom_name, prof[dom_name]) if dom_name in prof else (None, None)
    roof = None
    if dom[0]:
        per_launch_ms = dom[1]["ms"] / max(dom[1]["launches"], 1)
        b = alg_bytes(dom[0], st)
        if b is not None:
            traffic, tsrc = None, None
            if dom[0] == "kout" and args.variant == DEFAULT_VARIANT and args.edges == 16 * n and KOUT_DRAM_BYTES_PER_VERTEX:
                traffic = int(KOUT_DRAM_BYTES_PER_VERTEX * n)
                tsrc = KOUT_DRAM_SOURCE
            roof = roofline(b, per_launch_ms, hbm, peak_src, kernel=dom[0], traffic=traffic, traffic_source=tsrc,
                            alg_bytes_per_launch=b, avg_launch_ms=round(per_launch_ms, 5),
                            bytes_model="4(n+1) + 4kn (k = 2)" if dom[0] == "kout" else None)
    step_share = {k: round(vv["ms"] / max(sum(x["ms"] for x in prof_all.values()), 1e-9), 4)
                  for k, vv in prof_all.items()}
    kernel_us = {k: round(1e3 * vv["ms"] / max(vv["launches"], 1), 2) for k, vv in prof_all.items()}
    # whole-pass algorithmic bytes (every kernel of the pass by the same model)
    # and the input-equivalent bandwidth (8m + 12n) / t, which sampling lets exceed HBM
    pass_b = sum(alg_bytes(name, st) or 0 for name in prof_all)
    pass_roof = roofline(pass_b, ms, hbm, peak_src, kernels=[x for x in prof_all if alg_bytes(x, st)],
                         terms={x: alg_bytes(x, st) for x in prof_all if alg_bytes(x, st)})
    input_eq = {"value": round((8 * M + 12 * n) / (ms * 1e-3) / 1e9, 1), "unit": "GB/s",
                "definition": "(8 m + 12 n) / step time: the bytes an unsampled pass would stream"}

    result = {"metric": "static CC edges/s (RMAT scale 22, 2^26 undirected edges)",
              "value": M * world / (ms * 1e-3), "unit": "edges/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": round(ms, 5),
              "ms_per_step_median": round(float(np.median(step_ms)), 5),
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
              "data": "synthetic", "gpu_launches": int(launches), "labels_invariant_ok": ok,
              "config": {"workload": f"static_cc_rmat_s{args.scale}", "n": n, "m_undirected": M,
                         "arcs_csr": st["narcs"], "rmat_abcd": [0.57, 0.19, 0.19, 0.05], "seed": seed,
                         "variant": args.variant, "input": "CSR (u32 offsets, u32 cols), resident",
                         "launch": "one captured CUDA graph per step (gconn_plan_run)",
                         "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
              "roofline": roof, "pass_roofline": pass_roof, "input_equivalent_bw": input_eq,
              "kernel_share": step_share, "kernel_us": kernel_us,
              "instrumentation": {"timed_region": "plain captured plan, events around each replay only",
                                  "roofline_kernel_duration": f"{args.steps} replays right after the timed region "
                                                              f"of the same plan with one event pair around "
                                                              f"{dom_name}",
                                  "kernel_share": "separate replay loop, every kernel bracketed by events"},
              "clocks": clk,
              "wall_s_timed": round(wall, 4)}

    # end to end through the C ABI with pinned host buffers
    if rank == 0 and not args.no_e2e:
        h_off = torch.from_numpy(off32.view(np.int32)).pin_memory()
        h_cols = torch.from_numpy(cols.view(np.int32)).pin_memory()
        h_lab = torch.empty(n, dtype=torch.int32).pin_memory()
        for _ in range(2):
            g.gconn_cc_csr32(n, h_off, h_cols, h_lab, v, stream)
        tt = []
        for i in range(args.steps):
            flush.fill_(i)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            g.gconn_cc_csr32(n, h_off, h_cols, h_lab, v, stream)   # H2D + kernels + D2H + sync
            tt.append(time.perf_counter() - t1)
        e2e_s = float(np.mean(tt))
        lab_e2e = h_lab.numpy().view(np.uint32)
        staged = os.environ.get("GCONN_HOST_STAGE") == "1"
        # the offsets are copied; the columns are read in place where the
        # device reads host memory (k per row by the sampling, the active rows
        # by the finish), else copied whole
        in_place = 0 if staged else 4 * 2 * n + 4 * st.get("active_arcs", 0)
        copied = int(off32.nbytes + (cols.nbytes if staged else 0))
        result["e2e"] = {"value": M / e2e_s, "unit": "edges/s",
                         "h2d_bytes_per_step": copied + in_place,
                         "d2h_bytes_per_step": int(4 * n), "ms_per_step": round(e2e_s * 1e3, 4),
                         "h2d_breakdown": {"copied": copied, "read_in_place": in_place,
                                           "note": "columns read in place over the host link (cache-line "
                                                   "granularity: the link moves more than these algorithmic "
                                                   "bytes)" if not staged else "all inputs copied"},
                         "labels_equal_device_pass": bool(np.array_equal(lab_e2e, lab_timed))}

    legs = {"rmat_s22": (n, e, lab_timed)}      # final labels, checked against the oracle below
    roof_args = (hbm, peak_src)
    if rank == 0 and not args.no_coo:
        result["static_cc_coo"] = run_c2_coo(g, torch, dev, stream, args, flush, n, e, lab_timed, *roof_args)
    if rank == 0 and not args.no_c1:
        result["static_cc_er_c1"], legs["er_c1"] = run_c1(g, torch, dev, stream, args, flush, *roof_args)
    if rank == 0 and not args.no_c3:
        result["static_cc_grid_paths"], legs["grid_paths"] = run_c3(g, torch, dev, stream, args, flush, *roof_args)
    if rank == 0 and not args.no_incremental:
        result["incremental"] = run_incremental(g, torch, dev, stream, args, *roof_args)
    if rank == 0 and not args.no_batched:
        result["batched"] = run_batched(g, torch, dev, stream, args, *roof_args)
    if rank == 0 and not args.no_forest:
        result["spanning_forest"] = run_forest(g, torch, dev, stream, args, n, M, d_off32, d_cols, labels, flush, st,
                                               *roof_args)
    if rank == 0 and not args.no_serving:
        loads = [float(x) for x in args.serve_loads.split(",")]
        # the incremental workload's scale: 2^28 ops per session, batches of 10^3 - 10^8
        result["serving"] = run_serving(g, torch, args, args.serve_sessions, args.serve_ops, INC_N_SCALE,
                                        (3.0, 8.0), loads, args.serve_reps)
        # many sessions, small requests (10^3 - 10^4): where merging launches pays
        result["serving_small_requests"] = run_serving(g, torch, args, 32, 1 << 20, 20, (3.0, 4.0), loads)
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(n, e, args.cpu_seconds)
        result["cpu_multicore"] = cpu_multicore(n, M, off, cols, args.scale)
        checks = oracle_label_checks(legs)
        result["labels_equal_oracle"] = checks.get("rmat_s22")
        result["oracle_label_checks"] = checks
    if dist:
        dist.destroy_process_group()
    return result


def _time_passes(torch, stream, run, flush, warmup, steps, seed_base):
    """Device time of `run` (one pass), CUDA events on the launching stream,
    L2 flushed before every pass; returns the per-pass milliseconds."""
    for i in range(warmup):
        flush.fill_(seed_base + i)
        run()
    torch.cuda.synchronize()
    ts = []
    for i in range(steps):
        flush.fill_(seed_base + 100 + i)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return ts


def _pass_runner(g, plan_fn, direct_fn):
    """A captured plan where the variant allows one, else direct C-ABI calls."""
    try:
        plan = plan_fn()
    except g.GconnError:
        plan = None
    if plan is not None:
        return plan, (lambda st: g.gconn_plan_run(plan, st)), "captured plan"
    return None, direct_fn, "direct calls"


C2_COO_VARIANTS = ["none/remcas/naive/split_one", "none/async/halve/none", "none/early/naive/none"]


def run_c2_coo(g, torch, dev, stream, args, flush, n, e, lab_ref, hbm, peak_src):
    """The same RMAT graph as the headline pass, as its COO list without
    sampling (the plain method: init, one union per edge, finalisation), one
    captured plan per variant; the roofline on 8m + 12n bytes.  Labels must
    equal the headline pass's (which the CPU-baseline leg compares with the
    oracle)."""
    m = len(e)
    d_e = torch.from_numpy(e.view(np.int32)).to(dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    ref = torch.from_numpy(lab_ref.view(np.int32)).to(dev)
    rows = []
    for spec in C2_COO_VARIANTS:
        v = parse_variant(g, spec)
        plan, run, how = _pass_runner(g, lambda: g.gconn_plan_create_cc(n, m, d_e, lab, v),
                                      lambda st: g.gconn_cc(n, m, d_e, lab, v, st))
        ts = _time_passes(torch, stream, lambda: run(stream), flush, 2, max(3, min(args.steps, 5)), 5000)
        g.gconn_sync(stream)
        if plan is not None:
            g.gconn_plan_destroy(plan)
        ms = float(np.mean(ts))
        rows.append({"variant": spec, "launch": how, "ms": round(ms, 4), "edges_per_s": m / (ms * 1e-3),
                     "roofline": roofline(8 * m + 12 * n, ms, hbm, peak_src, bytes_model="8m + 12n"),
                     "labels_equal_csr_pass": bool(torch.equal(lab, ref))})
    del d_e, lab, ref
    torch.cuda.empty_cache()
    return {"workload": f"static_cc_rmat_s{args.scale}_coo", "n": n, "m_undirected": m,
            "input": "COO (uint32 pairs), resident, no sampling", "l2": "flushed between passes", "rows": rows}


def run_c1(g, torch, dev, stream, args, flush, hbm, peak_src):
    """ER G(n, m), n = 65,536, m = 2^20 (loops and duplicates kept), COO,
    Union-Rem-CAS + FullShortcut without sampling, as one captured plan.  The
    inputs fit in L2 (8 MiB), so the pass is launch- and latency-bound; the
    fraction is reported for completeness."""
    n, m = 65_536, 1 << 20
    e = graphgen.er(n, m, 0x6C0A0001)
    d_e = torch.from_numpy(e.view(np.int32)).to(dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    v = g.make_variant(link="remcas", find="fullshortcut", splice="splice")
    plan, run, how = _pass_runner(g, lambda: g.gconn_plan_create_cc(n, m, d_e, lab, v),
                                  lambda st: g.gconn_cc(n, m, d_e, lab, v, st))
    ts = _time_passes(torch, stream, lambda: run(stream), flush, args.warmup, max(args.steps, 5), 3000)
    g.gconn_sync(stream)
    if plan is not None:
        g.gconn_plan_destroy(plan)
    ms = float(np.mean(ts))
    b = 8 * m + 12 * n
    res = {"workload": "static_cc_er_n65536_m1048576", "variant": "none/remcas/fullshortcut/splice",
           "input": "COO (uint32 pairs), resident", "launch": how, "ms": round(ms, 5),
           "ms_median": round(float(np.median(ts)), 5), "edges_per_s": m / (ms * 1e-3),
           "roofline": roofline(b, ms, hbm, peak_src, bytes_model="8m + 12n (COO finish + init + finalisation)",
                                note="inputs fit in L2: launch- and latency-bound")}
    return res, (n, e, lab.cpu().numpy().view(np.uint32).copy())


C3_VARIANTS = [("coo", "none/remcas/naive/split_one"), ("csr", "kout/remcas/naive/split_one"),
               ("csr", "bfs/async/naive/none"), ("coo", "none/sv/naive/none"), ("coo", "none/lt/PRF/none")]


def run_c3(g, torch, dev, stream, args, flush, hbm, peak_src):
    """The high-diameter workload: a 4096 x 4096 grid with 5 % of its edges
    removed plus 64 randomly permuted paths of 2^18 vertices (n = 2^25,
    m = 48.6 M, edge order shuffled), as COO and as CSR; one row per
    sampling / finish variant.  Every variant's labels must equal the first
    variant's (compared on the device); the first is compared with the
    oracle in the CPU-baseline leg."""
    n, e = graphgen.grid_paths(4096, 0.05, 64, 1 << 18, 0x6C0A0003)
    m = len(e)
    off, cols = graphgen.csr(n, e)
    d_e = torch.from_numpy(e.view(np.int32)).to(dev)
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    d_off32 = torch.from_numpy(off.astype(np.uint32).view(np.int32)).to(dev)
    d_cols = torch.from_numpy(cols.view(np.int32)).to(dev)
    deg = np.diff(off.astype(np.int64))
    first = None
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    rows = []
    for kind, spec in C3_VARIANTS:
        v = parse_variant(g, spec)
        if kind == "coo":
            plan, run, how = _pass_runner(g, lambda: g.gconn_plan_create_cc(n, m, d_e, lab, v),
                                          lambda st: g.gconn_cc(n, m, d_e, lab, v, st))
        else:
            plan, run, how = _pass_runner(g, lambda: g.gconn_plan_create_cc_csr32(n, d_off32, d_cols, lab, v),
                                          lambda st: g.gconn_cc_csr32(n, d_off32, d_cols, lab, v, st))
        ts = _time_passes(torch, stream, lambda: run(stream), flush, 2, max(3, min(args.steps, 5)), 4000)
        g.gconn_sync(stream)
        if plan is not None:
            g.gconn_plan_destroy(plan)
        ms = float(np.mean(ts))
        row = {"input": kind, "variant": spec, "launch": how, "ms": round(ms, 4), "edges_per_s": m / (ms * 1e-3),
               "input_equivalent_gbs": round((8 * m + 12 * n) / (ms * 1e-3) / 1e9, 1)}
        sample = spec.split("/")[0]
        link = spec.split("/")[1]
        if kind == "coo" and link not in ("sv", "lt"):
            row["roofline"] = roofline(8 * m + 12 * n, ms, hbm, peak_src, bytes_model="8m + 12n")
        elif kind == "coo":
            row["roofline_lower_bound"] = roofline(8 * m + 12 * n, ms, hbm, peak_src,
                                                   bytes_model="8m + 12n: one edge pass (the rounds re-read the "
                                                               "edges and labels every round)")
        else:
            try:
                stt = g.gconn_cc_csr_stats(n, d_off, d_cols, lab, v, stream)
                act_v, act_a, lmax = int(stt.active_vertices), int(stt.active_arcs), int(stt.lmax)
                if sample == "kout":
                    samp = 4 * (n + 1) + 8 * n
                else:   # BFS: 4 bytes per arc of the reached component
                    hl = lab.cpu().numpy().view(np.uint32)
                    samp = 4 * int(deg[hl == lmax].sum()) if lmax < n else 0
                b = 4 * n + samp + 4 * n + 4 * act_a + 8 * act_v + 8 * n
                row["roofline"] = roofline(b, ms, hbm, peak_src, active_vertices=act_v, active_arcs=act_a,
                                           bytes_model="init 4n + sampling + VG 4n + finish + finalise 8n")
            except g.GconnError as ex:
                row["roofline"] = None
                row["stats_error"] = str(ex)
        if first is None:
            first = lab.clone()
            row["labels"] = "compared with the oracle (CPU-baseline leg)"
        else:
            row["labels_equal_first_variant"] = bool(torch.equal(lab, first))
        rows.append(row)
    res = {"workload": "static_cc_grid4096_paths64x2^18", "n": n, "m_undirected": m,
           "input": "COO (uint32 pairs) and CSR (u32 offsets), resident", "l2": "flushed between passes",
           "rows": rows}
    out = (n, e, first.cpu().numpy().view(np.uint32).copy())
    del d_e, d_off, d_off32, d_cols, lab, first
    torch.cuda.empty_cache()
    return res, out


def run_incremental(g, torch, dev, stream, args, hbm, peak_src):
    """The insert/query stream on n = 2^24: 2^28 RMAT scale-24 insertions in
    batches of log-uniform size in [10^3, 10^8], each followed by a query
    batch of the same size of uniform random pairs.  Stream s of the
    args.inc_seeds streams draws its own batch-size sequence and relabels the
    vertices of the same edge multiset by its own seeded permutation (done on
    the device, outside the timed batches), so per-batch latencies can be
    pooled per batch-size decade; one extra pass of stream 0 warms up."""
    n = 1 << INC_N_SCALE
    perm = graphgen.permutation(n, SEED_INC, 6)
    total = INC_TOTAL
    ins0 = torch.empty((total, 2), dtype=torch.int32, device=dev)
    qry = torch.empty((total, 2), dtype=torch.int32, device=dev)
    chunk = 1 << 25
    buf = np.empty((chunk, 2), np.uint32)
    if args.inc_gen == "ba":    # growth stream: vertex v arrives with total / n edges to earlier vertices
        ba = graphgen.ba(n, total // n, SEED_INC)
        ins0.copy_(torch.from_numpy(ba.view(np.int32)))
        del ba
    for s in range(0, total, chunk):
        c = min(chunk, total - s)
        if args.inc_gen != "ba":
            graphgen.rmat_range(INC_N_SCALE, s, c, SEED_INC, perm=perm, out=buf[:c])
            ins0[s:s + c].copy_(torch.from_numpy(buf[:c].view(np.int32)))
        graphgen.pairs_range(n, s, c, SEED_INC, out=buf[:c])
        qry[s:s + c].copy_(torch.from_numpy(buf[:c].view(np.int32)))
    ins = torch.empty_like(ins0)
    out = torch.empty(total, dtype=torch.uint8, device=dev)
    v = parse_variant(g, "none/" + args.inc_variant)
    recs = []                                   # (batch size, insert ms, query ms)
    nseeds = max(1, args.inc_seeds)
    for rep in range(nseeds + 1):               # rep 0 warms up on stream 0
        si = max(rep - 1, 0)
        sizes = inc_batches(SEED_INC + si)
        if si == 0:
            ins.copy_(ins0)
        else:                                   # relabel: ins = pi_s[ins0], chunked
            pi = torch.from_numpy(graphgen.permutation(n, SEED_INC + si, 7).view(np.int32)).to(dev).long()
            for s in range(0, total, chunk):
                ins[s:s + chunk] = pi[ins0[s:s + chunk].long()].int()
            del pi
        inc = g.Incremental(n, v, stream)
        evs = []
        s = 0
        torch.cuda.synchronize()
        for b in sizes:
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            inc.insert(ins[s:s + b], stream)
            e1.record(stream)
            inc.query(qry[s:s + b], out[s:s + b], stream)
            e2.record(stream)
            evs.append((b, e0, e1, e2))
            s += b
        torch.cuda.synchronize()
        g.gconn_sync(stream)
        inc.close()
        if rep > 0:
            recs += [(b, a.elapsed_time(b_), b_.elapsed_time(c)) for (b, a, b_, c) in evs]
    ins_ms = [r[1] for r in recs]
    q_ms = [r[2] for r in recs]
    per_decade = {}
    for d in range(3, 9):
        sel = [r for r in recs if 10 ** d <= r[0] < 10 ** (d + 1)]
        if sel:
            per_decade[f"1e{d}"] = {"batches": len(sel),
                                    "insert_ms_p50": round(pct([r[1] for r in sel], 50), 4),
                                    "insert_ms_p99": round(pct([r[1] for r in sel], 99), 4),
                                    "query_ms_p50": round(pct([r[2] for r in sel], 50), 4),
                                    "query_ms_p99": round(pct([r[2] for r in sel], 99), 4)}
    small = [r for r in recs if r[0] < 1000]
    if small:
        per_decade["<1e3 (truncated last batch)"] = {"batches": len(small)}
    res = {"n": n, "generator": "Barabasi-Albert, d = %d" % (total // n) if args.inc_gen == "ba"
           else "RMAT scale 24 (Graph500 a, b, c), relabelled",
           "inserts_per_stream": total, "queries_per_stream": total, "streams": nseeds,
           "batches": len(recs), "variant": args.inc_variant,
           "updates_per_s": nseeds * total / (sum(ins_ms) * 1e-3),
           "queries_per_s": nseeds * total / (sum(q_ms) * 1e-3),
           "ops_per_s": 2 * nseeds * total / ((sum(ins_ms) + sum(q_ms)) * 1e-3),
           "insert_batch_ms_p50": round(pct(ins_ms, 50), 4), "insert_batch_ms_p99": round(pct(ins_ms, 99), 4),
           "query_batch_ms_p50": round(pct(q_ms, 50), 4), "query_batch_ms_p99": round(pct(q_ms, 99), 4),
           "per_batch_size_decade": per_decade,
           "batch_sizes_min_max": [min(r[0] for r in recs), max(r[0] for r in recs)],
           "latency": "device time per batch, CUDA events on the launching stream",
           "inputs": "resident in HBM"}
    # 8 bytes per inserted pair, 9 per query (its pair and its answer byte)
    res["roofline_insert"] = roofline(8 * nseeds * total, sum(ins_ms), hbm, peak_src, bytes_model="8 B per insert")
    res["roofline_query"] = roofline(9 * nseeds * total, sum(q_ms), hbm, peak_src,
                                     bytes_model="9 B per query (pair + answer byte)")
    del ins, ins0, qry, out
    torch.cuda.empty_cache()
    return res


def run_forest(g, torch, dev, stream, args, n, M, d_off, d_cols, labels, flush, st, hbm, peak_src):
    """Spanning forest (Algorithm 2) of the same RMAT graph through
    gconn_spanning_forest_csr with device buffers; the forest must have
    n - c edges (c = components of the timed CC pass)."""
    v = parse_variant(g, args.variant)
    forest = torch.empty(n, dtype=torch.int64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    plan = g.gconn_plan_create_forest_csr32(n, d_off, d_cols, forest, count, None, v)
    for i in range(args.warmup):
        flush.fill_(i)
        g.gconn_plan_run(plan, stream)
    g.gconn_sync(stream)
    ts = []
    for i in range(args.steps):
        flush.fill_(i + 700)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.gconn_plan_run(plan, stream)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    g.gconn_sync(stream)
    g.gconn_plan_destroy(plan)
    comps = int(torch.unique(labels).numel())
    cnt = int(count.item())
    ms = float(np.mean(ts))
    pass_b = sum(alg_bytes(k, st) for k in ("init", "kout", "vg", "finish")) + 4 * n + 8 * cnt
    return {"edges_per_s": M / (ms * 1e-3), "ms": round(ms, 5), "ms_median": round(float(np.median(ts)), 5),
            "roofline": roofline(pass_b, ms, hbm, peak_src,
                                 bytes_model="init 4n + k-out 4(n+1) + 8n + VG 4n + finish + forest slots 4n "
                                             "+ forest ids 8(n - c)"),
            "forest_edges": cnt, "components": comps, "count_is_n_minus_c": cnt == n - comps,
            "variant": args.variant, "output": "arc positions of the forest edges (int64), compacted on device",
            "launch": "one captured plan per pass (gconn_plan_create_forest_csr)"}


def run_batched(g, torch, dev, stream, args, hbm, peak_src):
    """4,096 independent graphs (n log-uniform in [256, 65,536], average
    degree uniform in [4, 32], half ER half RMAT) in one captured plan,
    against one gconn_cc launch sequence per graph; both must agree exactly."""
    G = 4096
    vo, eo, e = graphgen.batched(G, SEED_BATCH)
    d_vo = torch.from_numpy(vo.view(np.int64)).to(dev)
    d_eo = torch.from_numpy(eo.view(np.int64)).to(dev)
    d_e = torch.from_numpy(e.view(np.int32)).to(dev)
    lab = torch.empty(int(vo[-1]), dtype=torch.int32, device=dev)
    lab2 = torch.empty(int(vo[-1]), dtype=torch.int32, device=dev)
    t0 = time.perf_counter()
    tune = g.gconn_batch_autotune(G, vo, eo, d_e, lab, stream)
    tune_s = time.perf_counter() - t0
    h = g.gconn_batch_create(G, d_vo, d_eo, d_e, lab, tune, stream)
    for _ in range(args.warmup):
        g.gconn_batch_run(h, stream)
    g.gconn_sync(stream)
    ts = []
    for i in range(max(args.steps, 3)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.gconn_batch_run(h, stream)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    g.gconn_sync(stream)
    ms = float(np.mean(ts))
    # the plain form: one gconn_cc call per graph on the same stream
    vol, eol = vo.tolist(), eo.tolist()
    v = g.make_variant(link="remcas", splice="split_one")

    def per_graph():
        for gi in range(G):
            n = vol[gi + 1] - vol[gi]
            m = eol[gi + 1] - eol[gi]
            g.gconn_cc(n, m, d_e[eol[gi]:eol[gi + 1]], lab2[vol[gi]:vol[gi + 1]], v, stream)
    per_graph()
    g.gconn_sync(stream)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    per_graph()
    b.record(stream)
    b.synchronize()
    ms_pg = a.elapsed_time(b)
    g.gconn_sync(stream)
    same = bool(torch.equal(lab, lab2))
    g.gconn_batch_destroy(h)
    m_tot = int(eo[-1])
    res = {"graphs": G, "vertices": int(vo[-1]), "edges": m_tot, "ms": round(ms, 4),
           "edges_per_s": m_tot / (ms * 1e-3), "graphs_per_s": G / (ms * 1e-3),
           "per_graph_launches_ms": round(ms_pg, 3), "per_graph_edges_per_s": m_tot / (ms_pg * 1e-3),
           "speedup_vs_per_graph": round(ms_pg / ms, 2), "identical_labels": same,
           "roofline": roofline(8 * m_tot + 4 * int(vo[-1]), ms, hbm, peak_src,
                                bytes_model="8m + 4n (edges read once, labels written once)"),
           "tune": tune.as_dict(), "autotune_s": round(tune_s, 2),
           "launch": "one CUDA graph replay (a persistent kernel per size class on forked streams)"}
    del d_e, lab, lab2
    torch.cuda.empty_cache()
    return res


def rmat_stream(scale, total, seed, perm, threads=16, out=None):
    """Edges [0, total) of the seeded RMAT stream, generated in parallel
    chunks (the C generator releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    out = np.empty((total, 2), np.uint32) if out is None else out
    chunk = -(-total // threads)
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda s0: graphgen.rmat_range(scale, s0, min(chunk, total - s0), seed, perm=perm,
                                                   out=out[s0:s0 + min(chunk, total - s0)]),
                    range(0, total, chunk)))
    return out


def host_array(shape, dtype, pinned):
    """A host array, page-locked when asked (a serving frontend's receive buffers)."""
    if not pinned:
        return np.empty(shape, dtype)
    import torch
    tdt = {np.dtype(np.uint32): torch.int32, np.dtype(np.uint8): torch.uint8}[np.dtype(dtype)]
    return torch.empty(shape, dtype=tdt, pin_memory=True).numpy().view(dtype)


def serving_trace(sessions, n_scale, total, seed, pinned=False, law=(3.0, 8.0)):
    """Per session s: its own RMAT scale-24 insert stream (seed + s) and as
    many uniform query pairs, cut into insert batches of log-uniform size in
    [10^3, 10^8] (the incremental workload's law), each followed by a query
    batch of the same size; requests are (op, pairs) in session order.  Also
    returns one answer buffer per session (a query request's answers go to
    its slice)."""
    n = 1 << n_scale
    perm = graphgen.permutation(n, seed, 6)
    out, answers = [], []
    for s in range(sessions):
        ins = rmat_stream(n_scale, total, seed + s, perm, out=host_array((total, 2), np.uint32, pinned))
        qry = graphgen.pairs_range(n, 0, total, seed + s, out=host_array((total, 2), np.uint32, pinned))
        answers.append(host_array(total, np.uint8, pinned))
        reqs, a = [], 0
        for b in inc_batches(seed + s, total, *law):
            reqs.append((0, ins[a:a + b], a))
            reqs.append((1, qry[a:a + b], a))
            a += b
        out.append(reqs)
    return n, out, answers


def run_serving(g, torch, args, sessions, ops, n_scale, law, loads, reps=1):
    """Continuous batching at the incremental workload's scale, open loop.
    S sessions (n = 2^24 each, Union-Early), each with its own stream of 2^28
    RMAT insertions and 2^28 query pairs in batches of log-uniform size in
    [10^3, 10^8], in page-locked host buffers (a frontend's receive buffers).
    Requests ARRIVE by a seeded Poisson process per session at an offered
    load (ops/s, a fraction of what the plain loop sustains back to back) and
    are either (plain) executed one at a time in arrival order by
    synchronous gconn_inc_* calls, or (served) submitted at arrival to one
    gconn_server, which admits them as slots and staging memory free up and
    overlaps different sessions' work.  Latency is arrival to answer on the
    host clock; every query answer must be identical."""
    S = sessions
    n, trace, answers = serving_trace(S, n_scale, ops, SEED_SERVE, pinned=True, law=law)
    v = g.make_variant(link="early")
    total_ops = sum(len(a) for reqs in trace for _, a, _ in reqs)
    nreq = sum(len(r) for r in trace)

    def out_of(s, r):
        _, a, off = trace[s][r]
        return answers[s][off:off + len(a)]

    def same_as(ref):
        return all(trace[s][r][0] == 0 or np.array_equal(out_of(s, r), ref[s][r])
                   for s in range(S) for r in range(len(trace[s])))

    def plain_run(arrivals):
        """One thread, arrival order; arrivals None = back to back."""
        hs = [g.gconn_inc_create(n, v) for _ in range(S)]
        torch.cuda.synchronize()
        order = sorted((arrivals[s][r] if arrivals else 0.0, s, r) for s in range(S) for r in range(len(trace[s])))
        lat = []
        t0 = time.perf_counter()
        for at, s, r in order:
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            op, a, _ = trace[s][r]
            if op == 0:
                g.gconn_inc_insert_batch(hs[s], len(a), a)
            else:
                g.gconn_inc_query(hs[s], len(a), a, out_of(s, r))
            lat.append((time.perf_counter() - t0 - at) * 1e3)
        span = time.perf_counter() - t0 - (order[0][0] if arrivals else 0.0)
        for h in hs:
            g.gconn_inc_destroy(h)
        return lat, span

    def served_run(arrivals):
        """One submitter thread (all sessions, arrival order) and one thread
        that waits for the tickets in submission order; latency comes from
        the server's own clock (submit to answer) plus the submitter's lag."""
        srv = g.gconn_server_create()
        sids = [g.gconn_server_open_session(srv, n, v) for _ in range(S)]
        order = sorted((arrivals[s][r], s, r) for s in range(S) for r in range(len(trace[s])))
        tickets, lat = [], []
        cv = threading.Condition()
        t0 = time.perf_counter()

        def submitter():
            for at, s, r in order:
                now = time.perf_counter() - t0
                if at > now:
                    time.sleep(at - now)
                op, a, _ = trace[s][r]
                lag = (time.perf_counter() - t0 - at) * 1e3
                t = g.gconn_server_submit(srv, sids[s], g.GCONN_OP_INSERT if op == 0 else g.GCONN_OP_QUERY,
                                          len(a), a, out_of(s, r) if op == 1 else None)
                with cv:
                    tickets.append((t, lag))
                    cv.notify_all()

        def waiter():
            for i in range(len(order)):
                with cv:
                    cv.wait_for(lambda: len(tickets) > i)
                    t, lag = tickets[i]
                lat.append(g.gconn_server_wait(srv, t) + lag)

        th = [threading.Thread(target=submitter), threading.Thread(target=waiter)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        span = time.perf_counter() - t0 - order[0][0]
        st = g.gconn_server_stats(srv)
        g.gconn_server_destroy(srv)
        return lat, span, st

    # the plain loop back to back: its answers are the reference and its
    # capacity sets the offered loads
    _, span0 = plain_run(None)
    ref = [[out_of(s, r).copy() if trace[s][r][0] == 1 else None for r in range(len(trace[s]))] for s in range(S)]
    cap_ops = total_ops / span0
    rng = np.random.default_rng(SEED_SERVE)
    rows, identical = [], True
    for frac in loads:
        rate = frac * cap_ops                                   # offered ops/s, all sessions
        # `reps` independent arrival draws over the same trace, latencies pooled
        pl, sl, ps, ss, launches, groups, same, p50s = [], [], 0.0, 0.0, 0, 0, True, []
        for _ in range(reps):
            arrivals = []
            for s in range(S):                                  # Poisson, mean request size per session
                mean_ops = sum(len(a) for _, a, _ in trace[s]) / len(trace[s])
                gaps = rng.exponential(mean_ops * S / rate, len(trace[s]))
                arrivals.append(list(np.cumsum(gaps)))
            for buf in answers:
                buf.fill(2)
            l1, s1 = plain_run(arrivals)
            same &= same_as(ref)
            for buf in answers:
                buf.fill(2)
            l2, s2, st = served_run(arrivals)
            same &= same_as(ref)
            pl += l1
            sl += l2
            ps += s1
            ss += s2
            launches += st["launches"]
            groups += st["groups"]
            p50s.append([round(pct(l1, 50), 3), round(pct(l2, 50), 3)])
        identical &= same
        rows.append({"offered_load_of_plain_capacity": frac, "offered_ops_per_s": rate,
                     "plain": {"ops_per_s": reps * total_ops / ps, "latency_ms_p50": round(pct(pl, 50), 3),
                               "latency_ms_p99": round(pct(pl, 99), 3)},
                     "served": {"ops_per_s": reps * total_ops / ss, "latency_ms_p50": round(pct(sl, 50), 3),
                                "latency_ms_p99": round(pct(sl, 99), 3), "launches": launches, "groups": groups},
                     "p50_plain_served_per_draw": p50s, "identical_answers": same})
    return {"sessions": S, "n_per_session": n, "requests": nreq, "ops": total_ops,
            "ops_per_session": ops, "batch_law": f"log-uniform sizes in [1e{law[0]:g}, 1e{law[1]:g}], insert then query",
            "plain_capacity_ops_per_s": cap_ops, "loads": rows, "identical_answers": identical,
            "arrivals": f"open loop: seeded Poisson per session at the offered load; {reps} draws per load, "
                        f"latencies pooled",
            "latency": "host clock, arrival to answers in the client's buffer",
            "inputs": "page-locked host memory (requests and answers)"}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_multicore(n, m, off, cols, scale):
    """The multicore CPU baseline (k-out sampling + lock-free union-find on all
    host cores) on the whole graph; best of 3 runs."""
    import cpu_baseline as cb
    lab = np.empty(n, np.uint32)
    cb.cc_csr(n, off, cols, out=lab)
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        cb.cc_csr(n, off, cols, out=lab)
        ts.append(time.perf_counter() - t0)
    dt = min(ts)
    return {"value": m / dt, "unit": "edges/s", "cores": cb.max_threads(), "kind": "multicore baseline",
            "method": "k-out (k=2) + L_max skip + lock-free Rem-CAS union-find, OpenMP",
            "sample": f"whole RMAT s{scale} CSR ({n} vertices, {m} undirected edges), best of 3",
            "ms": round(dt * 1e3, 3), "cpu_model": cpu_model()}


def cpu_baseline(n, e, seconds):
    """The oracle (sequential union-find, one host core) on the first m_s
    edges of the same edge list, m_s sized for about `seconds` of work."""
    import oracle
    m_s = 1 << 20
    t0 = time.perf_counter()
    oracle.cc_uf(n, e[:m_s])
    dt = time.perf_counter() - t0
    while dt < seconds / 4 and m_s < len(e):
        m_s = min(len(e), m_s * 4)
        t0 = time.perf_counter()
        oracle.cc_uf(n, e[:m_s])
        dt = time.perf_counter() - t0
    runs = [dt]   # the sample size is final: repeat it for about seconds / 4 in all, report the median
    while sum(runs) < seconds / 4 and len(runs) < 15:
        t0 = time.perf_counter()
        oracle.cc_uf(n, e[:m_s])
        runs.append(time.perf_counter() - t0)
    dt = float(np.median(runs))
    return {"value": m_s / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"first {m_s} edges of the RMAT s22 COO list, all {n} vertices; O1 union-find incl. "
                      f"min-id canonicalisation; median of {len(runs)} runs", "seconds": round(dt, 3),
            "runs": len(runs), "host_cores_available": os.cpu_count(), "oracle_threads": 1,
            "cpu_model": cpu_model()}


def oracle_label_checks(legs: dict) -> dict:
    """The labels each timed leg ended with against the oracle's (O1 on the
    whole graph), bit for bit: part of the CPU-baseline leg, the one place
    the benchmark runs the oracle beside the GPU path."""
    import oracle
    out = {}
    for name, (n, e, lab) in legs.items():
        t0 = time.perf_counter()
        ref = oracle.cc_uf(n, e)
        out[name] = bool(np.array_equal(ref, lab))
        out[name + "_oracle_s"] = round(time.perf_counter() - t0, 2)
    return out


# ------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The oracle timed as it stands on the host cores (rank 0 only)."""
    if rank != 0:
        return None
    import oracle
    n = 1 << SCALE
    e = graphgen.rmat(SCALE, M_EDGES, SEED_STATIC)
    m_s = min(M_EDGES, args.ref_edges)
    for _ in range(args.warmup):
        oracle.cc_uf(n, e[:m_s])
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.cc_uf(n, e[:m_s])
        ts.append(time.perf_counter() - t0)
    val = m_s / float(np.mean(ts))
    return {"impl": "reference", "metric": "static CC edges/s (RMAT scale 22, 2^26 undirected edges)",
            "value": val, "unit": "edges/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(float(np.mean(ts)) * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "static_cc_rmat_s22", "n": n, "m_undirected": M_EDGES, "seed": SEED_STATIC},
            "cpu_baseline": {"value": val, "unit": "edges/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {m_s} edges of the RMAT s22 COO list per step"},
            "e2e": {"value": val, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


SWEEP_LINKS = ([("async", f, "none") for f in ["naive", "compress", "split", "halve", "fullshortcut"]]
               + [("hooks", f, "none") for f in ["naive", "compress", "split", "halve"]]
               + [("early", f, "none") for f in ["naive", "compress", "split", "halve"]]
               + [("remcas", f, s) for f in ["naive", "split", "halve"] for s in ["split_one", "halve_one", "splice"]]
               + [("remlock", "naive", s) for s in ["split_one", "halve_one"]]
               + [("afforest", "naive", "none"), ("eclcc", "naive", "none")]
               + [("jtb", f, "none") for f in ["naive", "twotrysplit"]]
               + [("lp", "naive", "none"), ("stergiou", "naive", "none")]
               + [("sv", "naive", "none")]
               + [("lt", r, "none") for r in ["PRF", "PRS", "CRFA", "PUF", "EUF", "CUFA"]])


def run_sweep(args):
    """Sampling x linking x compression on a CSR graph (the RMAT scale-22
    workload, or with --sweep-graph grid_paths the high-diameter one); every
    variant's labels are compared bit for bit with the oracle's."""
    import torch
    import oracle
    import paper_2008_11839_gb300 as g
    g.build()
    dev = torch.device("cuda", 0)
    if args.sweep_graph == "grid_paths":
        n, e = graphgen.grid_paths(4096, 0.05, 64, 1 << 18, 0x6C0A0003)
        off, cols = graphgen.csr(n, e)
    else:
        n, e, off, cols, seed = make_static_input(0)
    m_und = len(e)
    ref = oracle.cc_uf(n, e)
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    d_cols = torch.from_numpy(cols.view(np.int32)).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    samples = args.sweep_samples.split(",")
    rows = []
    for sample in samples:
        for link, f, sp in SWEEP_LINKS:
            spec = f"{sample}/{link}/{f}/{sp}"
            if args.sweep_graph == "grid_paths" and sample == "none" and link == "lp":
                # label propagation needs about as many rounds as the paths are long (2^18):
                # beyond the round cap
                rows.append({"variant": spec, "skipped": "rounds ~ path length (2^18) exceed the round cap"})
                print(json.dumps(rows[-1]), flush=True)
                continue
            v = parse_variant(g, spec)
            plan = None
            try:
                try:      # a captured plan where the variant allows one (no host round trip in the pass)
                    plan = g.gconn_plan_create_cc_csr(n, d_off, d_cols, labels, v)
                except g.GconnError:
                    plan = None

                def run():
                    if plan is not None:
                        g.gconn_plan_run(plan, stream)
                    else:
                        g.gconn_cc_csr(n, d_off, d_cols, labels, v, stream)
                for i in range(3):
                    flush.fill_(i)
                    run()
                g.gconn_sync(stream)
                exact = bool((labels.cpu().numpy().view(np.uint32) == ref).all())
                ts = []
                for i in range(args.sweep_steps):
                    flush.fill_(i)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    run()
                    b.record(stream)
                    b.synchronize()
                    ts.append(a.elapsed_time(b))
                g.gconn_sync(stream)
                ms = float(np.median(ts))
                row = {"variant": spec, "ms": round(ms, 4), "edges_per_s": m_und / (ms * 1e-3), "exact": exact,
                       "input_equivalent_gbs": round((8 * m_und + 12 * n) / (ms * 1e-3) / 1e9, 1),
                       "launch": "captured plan" if plan is not None else "direct calls"}
            except g.GconnError as ex:
                row = {"variant": spec, "error": str(ex)}
            if plan is not None:
                g.gconn_plan_destroy(plan)
            rows.append(row)
            print(json.dumps(row), flush=True)
    ok = [r for r in rows if "ms" in r]
    rows = [r for r in rows if "skipped" not in r]
    ok.sort(key=lambda r: r["ms"])
    print(json.dumps({"sweep_best": ok[:10], "all_exact": all(r["exact"] for r in ok), "variants": len(rows)}))


def run_ablation(args):
    """The contribution of the GB300 forms of the paper's GPU optimisations
    (Section 3.3: coalesced / reorganised sampling reads, vertex gathering) on
    the RMAT s22 CSR: the default pass against its plain forms, each as a
    captured plan, labels checked against the oracle."""
    import torch
    import oracle
    import paper_2008_11839_gb300 as g
    g.build()
    dev = torch.device("cuda", 0)
    n, e, off, cols, seed = make_static_input(0, args.scale, args.edges)
    ref = oracle.cc_uf(n, e)
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    d_cols = torch.from_numpy(cols.view(np.int32)).to(dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    forms = [(0, "library kernels"), (1, "plain k-out (thread per vertex)"),
             (2, "no vertex gathering (thread-per-vertex finish)"), (3, "both plain")]
    rows = []
    for spec in args.ablation_variants.split(","):
        for bits, what in forms:
            v = parse_variant(g, spec)
            v.ablation = bits
            plan = g.gconn_plan_create_cc_csr(n, d_off, d_cols, labels, v)
            for i in range(3):
                flush.fill_(i)
                g.gconn_plan_run(plan, stream)
            g.gconn_sync(stream)
            exact = bool((labels.cpu().numpy().view(np.uint32) == ref).all())
            ts = []
            for i in range(args.steps):
                flush.fill_(i + 300)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g.gconn_plan_run(plan, stream)
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            g.gconn_sync(stream)
            g.gconn_plan_destroy(plan)
            ms = float(np.median(ts))
            row = {"variant": spec, "ablation": bits, "form": what, "ms": round(ms, 4),
                   "edges_per_s": args.edges / (ms * 1e-3), "exact": exact}
            rows.append(row)
            print(json.dumps(row), flush=True)


def run_stats(args):
    """Sampling quality on the RMAT s22 graph (the paper's Table 4 columns):
    Cov, IC, Time % and arcs inspected, per sampling method."""
    import torch
    import paper_2008_11839_gb300 as g
    g.build()
    dev = torch.device("cuda", 0)
    n, e, off, cols, seed = make_static_input(0, args.scale, args.edges)
    d_off = torch.from_numpy(off.view(np.int64)).to(dev)
    d_cols = torch.from_numpy(cols.view(np.int32)).to(dev)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    for spec in args.stats_variants.split(","):
        v = parse_variant(g, spec)
        for _ in range(2):                   # warm, then report the second run
            st = g.gconn_cc_csr_stats(n, d_off, d_cols, lab, v)
        d = st.as_dict()
        d["variant"] = spec
        print(json.dumps(d), flush=True)


def run_ratio_sweep(args):
    """Mixed batches (Algorithm 3) at several insert:query ratios x: the
    high-diameter grid + paths edges, shuffled, with 1/x random queries per
    insert mixed in, in batches of 2^22 operations (Section 4.4's experiment)."""
    import torch
    import paper_2008_11839_gb300 as g
    g.build()
    dev = torch.device("cuda", 0)
    n, e = graphgen.grid_paths(4096, 0.05, 64, 1 << 18, 0x6C0A0003)
    m = len(e)
    stream = torch.cuda.current_stream()
    for x in [8.0, 4.0, 2.0, 1.0, 0.5, 0.25]:
        q = int(m / x)
        pairs = np.empty((m + q, 2), np.uint32)
        pairs[:m] = e
        graphgen.pairs_range(n, 0, q, 0x6C0A0007, out=pairs[m:])
        isq = np.zeros(m + q, np.uint8)
        isq[m:] = 1
        perm = graphgen.permutation(m + q, 0x6C0A0008, 6).astype(np.int64)
        d_pairs = torch.from_numpy(pairs[perm].view(np.int32)).to(dev)
        d_isq = torch.from_numpy(isq[perm]).to(dev)
        total = m + q
        B = 1 << 22
        bits = torch.empty((B + 31) // 32, dtype=torch.int32, device=dev)
        for v_spec in args.ratio_variants.split(","):
            v = parse_variant(g, "none/" + v_spec)
            h = g.gconn_inc_create(n, v, stream)
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for s in range(0, total, B):
                c = min(B, total - s)
                g.gconn_inc_process_batch(h, c, d_pairs[s:s + c], d_isq[s:s + c], bits, stream)
            b_.record(stream)
            b_.synchronize()
            g.gconn_sync(stream)
            ms = a.elapsed_time(b_)
            g.gconn_inc_destroy(h)
            print(json.dumps({"ratio_insert_to_query": x, "variant": v_spec, "ops": total, "inserts": m,
                              "ms": round(ms, 3), "ops_per_s": total / (ms * 1e-3)}), flush=True)
        del d_pairs, d_isq
        torch.cuda.empty_cache()


def run_edge_inspect(args):
    """Section 4.4's edges-inspected figure: the first 2^24 edges of the RMAT
    scale-24 insert stream, inserted into a fresh n = 2^24 handle in batches of
    one size per decade 10^3 .. 10^7; per batch size and finish, the edge
    inspections the handle counted (each edge once for union-find, every
    round re-reads the whole batch for SV / Liu-Tarjan) and the device time."""
    import torch
    import paper_2008_11839_gb300 as g
    g.build()
    dev = torch.device("cuda", 0)
    n = 1 << INC_N_SCALE
    total = 1 << 24
    perm = graphgen.permutation(n, SEED_INC, 6)
    e = graphgen.rmat_range(INC_N_SCALE, 0, total, SEED_INC, perm=perm)
    d_e = torch.from_numpy(e.view(np.int32)).to(dev)
    stream = torch.cuda.current_stream()
    for v_spec in args.inspect_variants.split(","):
        v = parse_variant(g, "none/" + v_spec)
        for b in [10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7]:
            inc = g.Incremental(n, v, stream)
            per_batch = []
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for s in range(0, total, b):
                inc.insert(d_e[s:min(total, s + b)])
                per_batch.append(inc.edges_inspected()[0])
            z.record(stream)
            z.synchronize()
            g.gconn_sync(stream)
            insp = inc.edges_inspected()[1]
            inc.close()
            print(json.dumps({"variant": v_spec, "batch": b, "batches": len(per_batch), "edges": total,
                              "inspected": insp, "inspected_per_edge": round(insp / total, 3),
                              "max_batch_inspections_per_edge": round(max(x / min(b, total) for x in per_batch), 3),
                              "ms": round(a.elapsed_time(z), 3)}), flush=True)


def run_inc_probe(args):
    """One insert batch and one query batch of args.inc_probe pairs on an
    n = 2^24 handle that already holds the first 2^27 edges of the RMAT
    scale-24 insert stream (a realistic forest): the launches a kernel
    profile of the incremental path captures (the prefix is the first
    insert launch, the probe batch the second)."""
    import torch
    import paper_2008_11839_gb300 as g
    g.build()
    dev = torch.device("cuda", 0)
    n = 1 << INC_N_SCALE
    perm = graphgen.permutation(n, SEED_INC, 6)
    pre, b = 1 << 27, args.inc_probe
    e = rmat_stream(INC_N_SCALE, pre + b, SEED_INC, perm)
    d_e = torch.from_numpy(e.view(np.int32)).to(dev)
    q = torch.from_numpy(graphgen.pairs_range(n, 0, b, SEED_INC).view(np.int32)).to(dev)
    out = torch.empty(b, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    # the eager initialisation a handle pays once (P[v] = v over n = 2^24):
    # the cost a lazy per-vertex initialisation would trade for a check on
    # every access
    init_ms = []
    for _ in range(6):
        g.gconn_profile_reset()
        g.gconn_profile_select("init")
        g.gconn_profile_enable(True)
        h = g.Incremental(n, parse_variant(g, "none/early/naive"), stream)
        g.gconn_profile_enable(False)
        g.gconn_profile_select(None)
        torch.cuda.synchronize()
        g.gconn_profile_sync()
        prof = g.gconn_profile_get()
        h.close()
        if "init" in prof:
            init_ms.append(prof["init"][1])
    g.gconn_profile_reset()
    print(json.dumps({"eager_init": {"n": n, "ms_median": round(float(np.median(init_ms[1:])), 4) if init_ms else None,
                                     "bytes": 4 * n, "runs": len(init_ms) - 1}}), flush=True)
    rows = []
    for spec in args.inc_probe_variants.split(","):
        inc = g.Incremental(n, parse_variant(g, "none/" + spec), stream)
        inc.query(q[:1024], out[:1024], stream)        # first launches load the kernels' code
        inc.insert(d_e[:pre], stream)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        inc.insert(d_e[pre:pre + b], stream)
        ev[1].record(stream)
        inc.query(q, out, stream)
        ev[2].record(stream)
        torch.cuda.synchronize()
        g.gconn_sync(stream)
        inc.close()
        ti, tq = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        rows.append({"variant": spec, "batch": b, "insert_ms": round(ti, 4), "query_ms": round(tq, 4),
                     "updates_per_s": b / (ti * 1e-3), "queries_per_s": b / (tq * 1e-3)})
        print(json.dumps(rows[-1]), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default=DEFAULT_VARIANT)
    ap.add_argument("--inc-variant", default="early/naive", help="link/find[/splice] of the incremental handle")
    ap.add_argument("--inc-seeds", type=int, default=8, help="independent insert/query streams (latency pooling)")
    ap.add_argument("--inc-gen", choices=["rmat", "ba"], default="rmat",
                    help="insert-stream generator: RMAT (default) or Barabasi-Albert growth")
    ap.add_argument("--no-incremental", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-forest", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--inc-probe", type=int, default=0,
                    help="time one insert and one query batch of this size after a 2^27-edge prefix")
    ap.add_argument("--inc-probe-variants", default="early/naive")
    ap.add_argument("--serve-sessions", type=int, default=2)
    ap.add_argument("--serve-reps", type=int, default=5,
                    help="arrival draws per offered load at the incremental workload's scale (latencies pooled)")
    ap.add_argument("--serve-ops", type=int, default=1 << 28, help="insertions (and queries) per serving session")
    ap.add_argument("--serve-loads", default="0.3,0.6,0.9,1.2",
                    help="offered loads as fractions of the plain loop's back-to-back throughput")
    ap.add_argument("--no-c1", action="store_true", help="skip the ER n=65,536 COO leg")
    ap.add_argument("--no-coo", action="store_true", help="skip the headline graph's COO no-sampling rows")
    ap.add_argument("--no-c3", action="store_true", help="skip the grid + paths leg")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-edges", type=int, default=M_EDGES)
    ap.add_argument("--clock-window", type=float, default=1.0)
    ap.add_argument("--scale", type=int, default=SCALE, help="RMAT scale (default: the scale-22 workload)")
    ap.add_argument("--edges", type=int, default=M_EDGES, help="undirected edges (default 2^26)")
    ap.add_argument("--sweep", action="store_true", help="time every sampling x finish variant (RMAT s22)")
    ap.add_argument("--ablation", action="store_true", help="library kernels vs their plain forms (RMAT s22)")
    ap.add_argument("--ablation-variants", default="kout/remcas/naive/split_one,kout/early/naive/none,"
                                                   "hb/remcas/naive/split_one")
    ap.add_argument("--sweep-samples", default="none,kout,hb,bfs")
    ap.add_argument("--sweep-graph", choices=["rmat", "grid_paths"], default="rmat")
    ap.add_argument("--sweep-steps", type=int, default=5)
    ap.add_argument("--stats", action="store_true", help="sampling Cov / IC / Time %% per sampling method")
    ap.add_argument("--ratio-sweep", action="store_true", help="mixed batches at several insert:query ratios")
    ap.add_argument("--ratio-variants", default="early/naive,async/halve,remcas/naive/split_one")
    ap.add_argument("--edge-inspect", action="store_true",
                    help="edge inspections per insert batch size (SV, Liu-Tarjan PRS, union-find)")
    ap.add_argument("--inspect-variants", default="sv,lt/PRS,early/naive")
    ap.add_argument("--stats-variants", default="kout/remcas/naive/split_one,hb/remcas/naive/split_one,"
                                                 "bfs/remcas/naive/split_one,none/remcas/naive/split_one")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.sweep:
        run_sweep(args)
        return
    if args.ablation:
        run_ablation(args)
        return
    if args.stats:
        run_stats(args)
        return
    if args.ratio_sweep:
        run_ratio_sweep(args)
        return
    if args.edge_inspect:
        run_edge_inspect(args)
        return
    if args.inc_probe:
        run_inc_probe(args)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
