"""ctypes binding of libgconn (include/gconn.h).  Argument marshalling only:
every step of connectivity runs in the library's CUDA kernels.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; their data pointers
are passed straight through, so device tensors stay on the device.  A stream
argument of None means torch's current CUDA stream.  Non-OK statuses raise
GconnError.  If libgconn.so has not been built, every call raises
GconnUnavailable: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgconn.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gconn.h")

# status codes
GCONN_OK = 0
GCONN_E_INVAL = 1
GCONN_E_RANGE = 2
GCONN_E_NOMEM = 3
GCONN_E_UNSUPPORTED = 4
GCONN_E_NONCONVERGED = 5
GCONN_E_CUDA = 6
GCONN_NOALLOC_MAX_N = 1 << 20
# variant enums
GCONN_SAMPLE_NONE, GCONN_SAMPLE_KOUT, GCONN_SAMPLE_HB, GCONN_SAMPLE_BFS = 0, 1, 2, 3
(GCONN_LINK_ASYNC, GCONN_LINK_HOOKS, GCONN_LINK_EARLY, GCONN_LINK_REMCAS, GCONN_LINK_JTB,
 GCONN_LINK_SV, GCONN_LINK_LT, GCONN_LINK_REMLOCK, GCONN_LINK_ECLCC, GCONN_LINK_AFFOREST, GCONN_LINK_LP,
 GCONN_LINK_STERGIOU) = range(12)
(GCONN_FIND_NAIVE, GCONN_FIND_COMPRESS, GCONN_FIND_SPLIT, GCONN_FIND_HALVE, GCONN_FIND_TWOTRYSPLIT,
 GCONN_FIND_FULLSHORTCUT) = range(6)
GCONN_SPLICE_NONE, GCONN_SPLICE_SPLIT_ONE, GCONN_SPLICE_HALVE_ONE, GCONN_SPLICE_SPLICE = 0, 1, 2, 3
GCONN_LT_CONNECT, GCONN_LT_PARENT, GCONN_LT_EXTENDED = 0, 1, 2
GCONN_LT_ROOTUPDATE, GCONN_LT_FULLSHORTCUT, GCONN_LT_ALTER = 4, 8, 16

SAMPLES = {"none": 0, "kout": 1, "hb": 2, "bfs": 3}
LINKS = {"async": 0, "hooks": 1, "early": 2, "remcas": 3, "jtb": 4, "sv": 5, "lt": 6, "remlock": 7,
         "eclcc": 8, "afforest": 9, "lp": 10, "stergiou": 11}
FINDS = {"naive": 0, "compress": 1, "split": 2, "halve": 3, "twotrysplit": 4, "fullshortcut": 5}
SPLICES = {"none": 0, "split_one": 1, "halve_one": 2, "splice": 3}


def lt_rules(name: str) -> int:
    """Liu-Tarjan rule bits from an appendix name such as 'PRFA'."""
    name = name.upper()
    bits = {"C": GCONN_LT_CONNECT, "P": GCONN_LT_PARENT, "E": GCONN_LT_EXTENDED}[name[0]]
    if name[1] == "R":
        bits |= GCONN_LT_ROOTUPDATE
    if name[2] == "F":
        bits |= GCONN_LT_FULLSHORTCUT
    if name.endswith("A"):
        bits |= GCONN_LT_ALTER
    return bits


class gconn_variant(ctypes.Structure):
    _fields_ = [("sample", ctypes.c_int32), ("k", ctypes.c_int32), ("hb_n", ctypes.c_int32),
                ("link", ctypes.c_int32), ("find", ctypes.c_int32), ("splice", ctypes.c_int32),
                ("lt_rules", ctypes.c_int32), ("block", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("iter_cap", ctypes.c_uint32), ("ablation", ctypes.c_uint32)]


GCONN_BATCH_CLASSES = 4


class gconn_batch_tune(ctypes.Structure):
    _fields_ = [("class_max_n", ctypes.c_uint32 * GCONN_BATCH_CLASSES),
                ("block", ctypes.c_int32 * GCONN_BATCH_CLASSES),
                ("link", ctypes.c_int32 * GCONN_BATCH_CLASSES),
                ("find", ctypes.c_int32 * GCONN_BATCH_CLASSES)]

    def as_dict(self):
        return {"class_max_n": list(self.class_max_n), "block": list(self.block),
                "link": list(self.link), "find": list(self.find)}


GCONN_OP_INSERT, GCONN_OP_QUERY = 0, 1
GCONN_ABL_PLAIN_SAMPLE, GCONN_ABL_NO_VG = 1, 2


class gconn_server_config(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32),
                ("coalesce_pairs", ctypes.c_uint32), ("slot_pairs", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class gconn_sample_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("n", "arcs", "lmax_vertices", "sampled_components",
                                               "active_vertices", "active_arcs", "inter_component_arcs",
                                               "sample_arcs_inspected", "lmax")] + \
               [("sample_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["cov"] = self.lmax_vertices / max(self.n, 1)
        d["ic"] = self.inter_component_arcs / max(self.arcs, 1)
        d["time_pct"] = self.sample_ms / self.total_ms if self.total_ms else 0.0
        return d


class GconnError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _status_text(status)
        super().__init__(f"{what}: {msg} (status {status})" if what else f"{msg} (status {status})")


class GconnUnavailable(ImportError):
    pass


_lock = threading.Lock()
_lib = None

_vp, _u32, _u64, _i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_SIGS = {
    "gconn_variant_default": (_i32, [ctypes.POINTER(gconn_variant)]),
    "gconn_variant_check": (_i32, [ctypes.POINTER(gconn_variant), _i32, _i32]),
    "gconn_cc": (_i32, [_u32, _u64, _vp, _vp, ctypes.POINTER(gconn_variant), _vp]),
    "gconn_cc_csr": (_i32, [_u32, _vp, _vp, _vp, ctypes.POINTER(gconn_variant), _vp]),
    "gconn_cc_csr32": (_i32, [_u32, _vp, _vp, _vp, ctypes.POINTER(gconn_variant), _vp]),
    "gconn_spanning_forest": (_i32, [_u32, _u64, _vp, _vp, _vp, _vp, ctypes.POINTER(gconn_variant), _vp]),
    "gconn_spanning_forest_csr": (_i32, [_u32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(gconn_variant), _vp]),
    "gconn_spanning_forest_csr32": (_i32, [_u32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(gconn_variant), _vp]),
    "gconn_inc_create": (_i32, [_u32, ctypes.POINTER(gconn_variant), _vp, ctypes.POINTER(_vp)]),
    "gconn_inc_insert_batch": (_i32, [_vp, _u64, _vp, _vp]),
    "gconn_inc_query": (_i32, [_vp, _u64, _vp, _vp, _vp]),
    "gconn_inc_labels": (_i32, [_vp, _vp, _vp]),
    "gconn_inc_edges_inspected": (_i32, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "gconn_inc_process_batch": (_i32, [_vp, _u64, _vp, _vp, _vp, _vp]),
    "gconn_inc_destroy": (_i32, [_vp]),
    "gconn_cc_csr_noalloc": (_i32, [_u32, _vp, _vp, _vp, ctypes.POINTER(gconn_variant), _vp]),
    "gconn_batch_tune_default": (_i32, [ctypes.POINTER(gconn_batch_tune)]),
    "gconn_cc_batched": (_i32, [_u32, _vp, _vp, _vp, _vp, ctypes.POINTER(gconn_batch_tune), _vp]),
    "gconn_batch_create": (_i32, [_u32, _vp, _vp, _vp, _vp, ctypes.POINTER(gconn_batch_tune), _vp,
                                  ctypes.POINTER(_vp)]),
    "gconn_batch_run": (_i32, [_vp, _vp]),
    "gconn_batch_destroy": (_i32, [_vp]),
    "gconn_batch_autotune": (_i32, [_u32, _vp, _vp, _vp, _vp, ctypes.POINTER(gconn_batch_tune), _vp]),
    "gconn_plan_create_cc": (_i32, [_u32, _u64, _vp, _vp, ctypes.POINTER(gconn_variant), ctypes.POINTER(_vp)]),
    "gconn_plan_create_cc_csr": (_i32, [_u32, _vp, _vp, _vp, ctypes.POINTER(gconn_variant), ctypes.POINTER(_vp)]),
    "gconn_plan_create_forest_csr": (_i32, [_u32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(gconn_variant),
                                            ctypes.POINTER(_vp)]),
    "gconn_plan_create_cc_csr32": (_i32, [_u32, _vp, _vp, _vp, ctypes.POINTER(gconn_variant),
                                          ctypes.POINTER(_vp)]),
    "gconn_plan_create_forest_csr32": (_i32, [_u32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(gconn_variant),
                                              ctypes.POINTER(_vp)]),
    "gconn_plan_run": (_i32, [_vp, _vp]),
    "gconn_plan_destroy": (_i32, [_vp]),
    "gconn_profile_sync": (_i32, []),
    "gconn_server_config_default": (_i32, [ctypes.POINTER(gconn_server_config)]),
    "gconn_server_create": (_i32, [ctypes.POINTER(gconn_server_config), ctypes.POINTER(_vp)]),
    "gconn_server_open_session": (_i32, [_vp, _u32, ctypes.POINTER(gconn_variant), ctypes.POINTER(_u32)]),
    "gconn_server_submit": (_i32, [_vp, _u32, _i32, _u64, _vp, _vp, ctypes.POINTER(_u64)]),
    "gconn_server_wait": (_i32, [_vp, _u64, ctypes.POINTER(ctypes.c_double)]),
    "gconn_server_labels": (_i32, [_vp, _u32, _vp]),
    "gconn_server_close_session": (_i32, [_vp, _u32]),
    "gconn_server_stats": (_i32, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "gconn_server_destroy": (_i32, [_vp]),
    "gconn_cc_csr_stats": (_i32, [_u32, _vp, _vp, _vp, ctypes.POINTER(gconn_variant),
                                  ctypes.POINTER(gconn_sample_stats), _vp]),
    "gconn_sync": (_i32, [_vp]),
    "gconn_status_str": (ctypes.c_char_p, [_i32]),
    "gconn_launch_count": (_u64, []),
    "gconn_release_cached": (_i32, []),
    "gconn_profile_enable": (_i32, [_i32]),
    "gconn_profile_select": (_i32, [ctypes.c_char_p]),
    "gconn_profile_reset": (_i32, []),
    "gconn_profile_get": (_i32, [_i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_u64),
                                 ctypes.POINTER(ctypes.c_double)]),
}


def declared_symbols(header: str = HEADER):
    """Names of every function declared in include/gconn.h."""
    txt = open(header).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gconn_[a-z0-9_]+)\s*\(", txt)))


def lib():
    """The loaded libgconn (raises GconnUnavailable when it is not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise GconnUnavailable(f"{LIB_PATH} is not built; run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name, None)
                if f is None:
                    continue
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _status_text(status: int) -> str:
    try:
        return lib().gconn_status_str(status).decode()
    except Exception:
        return "error"


def ptr(x):
    """Data pointer of a torch tensor / numpy array (None stays NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr() or None
    if hasattr(x, "ctypes"):
        return x.ctypes.data or None
    if isinstance(x, int):
        return x or None
    raise TypeError(f"cannot take a pointer of {type(x)}")


def stream_handle(stream=None):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream or None
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream or None
    return getattr(stream, "cuda_stream", None) or None


def check(status: int, what: str = "") -> None:
    if status != GCONN_OK:
        raise GconnError(status, what)


def make_variant(sample="none", link="async", find="naive", splice="none", lt="PRF", k=2, hb_n=4,
                 block=0, seed=0x6C0A0001, iter_cap=0, ablation=0) -> gconn_variant:
    v = gconn_variant()
    check(lib().gconn_variant_default(ctypes.byref(v)), "gconn_variant_default")
    v.sample = SAMPLES[sample] if isinstance(sample, str) else int(sample)
    v.link = LINKS[link] if isinstance(link, str) else int(link)
    v.find = FINDS[find] if isinstance(find, str) else int(find)
    v.splice = SPLICES[splice] if isinstance(splice, str) else int(splice)
    v.lt_rules = lt_rules(lt) if isinstance(lt, str) else int(lt)
    v.k, v.hb_n, v.block, v.seed, v.iter_cap, v.ablation = k, hb_n, block, seed, iter_cap, ablation
    return v


def _vref(v):
    return None if v is None else ctypes.byref(v)


# ------------------------------------------------------- same-name wrappers

def gconn_variant_default() -> gconn_variant:
    v = gconn_variant()
    check(lib().gconn_variant_default(ctypes.byref(v)), "gconn_variant_default")
    return v


def gconn_variant_check(v, input_kind: int, want_forest: int) -> int:
    return int(lib().gconn_variant_check(ctypes.byref(v), input_kind, want_forest))


def gconn_cc(n, m, edges, labels, variant=None, stream=None):
    check(lib().gconn_cc(n, m, ptr(edges), ptr(labels), _vref(variant), stream_handle(stream)), "gconn_cc")


def gconn_cc_csr(n, offsets, cols, labels, variant=None, stream=None):
    check(lib().gconn_cc_csr(n, ptr(offsets), ptr(cols), ptr(labels), _vref(variant), stream_handle(stream)),
          "gconn_cc_csr")


def gconn_cc_csr32(n, offsets, cols, labels, variant=None, stream=None):
    """gconn_cc_csr with uint32 offsets (fewer than 2^32 arcs)."""
    check(lib().gconn_cc_csr32(n, ptr(offsets), ptr(cols), ptr(labels), _vref(variant), stream_handle(stream)),
          "gconn_cc_csr32")


def gconn_cc_csr_noalloc(n, offsets, cols, labels, variant=None, stream=None):
    """gconn_cc_csr without device allocation (device buffers, n <= 2^20)."""
    check(lib().gconn_cc_csr_noalloc(n, ptr(offsets), ptr(cols), ptr(labels), _vref(variant),
                                     stream_handle(stream)), "gconn_cc_csr_noalloc")


def gconn_batch_tune_default() -> gconn_batch_tune:
    t = gconn_batch_tune()
    check(lib().gconn_batch_tune_default(ctypes.byref(t)), "gconn_batch_tune_default")
    return t


def gconn_cc_batched(G, vtx_off, edge_off, edges, labels, tune=None, stream=None):
    check(lib().gconn_cc_batched(G, ptr(vtx_off), ptr(edge_off), ptr(edges), ptr(labels), _vref(tune),
                                 stream_handle(stream)), "gconn_cc_batched")


def gconn_batch_create(G, vtx_off, edge_off, edges, labels, tune=None, stream=None):
    h = ctypes.c_void_p()
    check(lib().gconn_batch_create(G, ptr(vtx_off), ptr(edge_off), ptr(edges), ptr(labels), _vref(tune),
                                   stream_handle(stream), ctypes.byref(h)), "gconn_batch_create")
    return h


def gconn_batch_run(h, stream=None):
    check(lib().gconn_batch_run(h, stream_handle(stream)), "gconn_batch_run")


def gconn_batch_destroy(h):
    check(lib().gconn_batch_destroy(h), "gconn_batch_destroy")


def gconn_batch_autotune(G, vtx_off, edge_off, edges, labels, stream=None) -> gconn_batch_tune:
    t = gconn_batch_tune()
    check(lib().gconn_batch_autotune(G, ptr(vtx_off), ptr(edge_off), ptr(edges), ptr(labels), ctypes.byref(t),
                                     stream_handle(stream)), "gconn_batch_autotune")
    return t


def gconn_spanning_forest(n, m, edges, forest, forest_count, labels=None, variant=None, stream=None):
    check(lib().gconn_spanning_forest(n, m, ptr(edges), ptr(forest), ptr(forest_count), ptr(labels),
                                      _vref(variant), stream_handle(stream)), "gconn_spanning_forest")


def gconn_spanning_forest_csr(n, offsets, cols, forest, forest_count, labels=None, variant=None, stream=None):
    check(lib().gconn_spanning_forest_csr(n, ptr(offsets), ptr(cols), ptr(forest), ptr(forest_count),
                                          ptr(labels), _vref(variant), stream_handle(stream)),
          "gconn_spanning_forest_csr")


def gconn_spanning_forest_csr32(n, offsets, cols, forest, forest_count, labels=None, variant=None, stream=None):
    check(lib().gconn_spanning_forest_csr32(n, ptr(offsets), ptr(cols), ptr(forest), ptr(forest_count), ptr(labels),
                                            _vref(variant), stream_handle(stream)), "gconn_spanning_forest_csr32")


def gconn_inc_create(n, variant=None, stream=None):
    h = ctypes.c_void_p()
    check(lib().gconn_inc_create(n, _vref(variant), stream_handle(stream), ctypes.byref(h)), "gconn_inc_create")
    return h


def gconn_inc_insert_batch(h, b, edges, stream=None):
    check(lib().gconn_inc_insert_batch(h, b, ptr(edges), stream_handle(stream)), "gconn_inc_insert_batch")


def gconn_inc_query(h, q, pairs, connected, stream=None):
    check(lib().gconn_inc_query(h, q, ptr(pairs), ptr(connected), stream_handle(stream)), "gconn_inc_query")


def gconn_inc_process_batch(h, b, pairs, is_query, result_bits, stream=None):
    check(lib().gconn_inc_process_batch(h, b, ptr(pairs), ptr(is_query), ptr(result_bits), stream_handle(stream)),
          "gconn_inc_process_batch")


def gconn_inc_edges_inspected(h):
    """(inspections of the last insert / mixed batch, total since creation)."""
    last, total = _u64(0), _u64(0)
    check(lib().gconn_inc_edges_inspected(h, ctypes.byref(last), ctypes.byref(total)), "gconn_inc_edges_inspected")
    return last.value, total.value


def gconn_inc_labels(h, labels, stream=None):
    check(lib().gconn_inc_labels(h, ptr(labels), stream_handle(stream)), "gconn_inc_labels")


def gconn_inc_destroy(h):
    check(lib().gconn_inc_destroy(h), "gconn_inc_destroy")


def gconn_plan_create_cc(n, m, edges, labels, variant=None):
    h = ctypes.c_void_p()
    check(lib().gconn_plan_create_cc(n, m, ptr(edges), ptr(labels), _vref(variant), ctypes.byref(h)),
          "gconn_plan_create_cc")
    return h


def gconn_plan_create_cc_csr(n, offsets, cols, labels, variant=None):
    h = ctypes.c_void_p()
    check(lib().gconn_plan_create_cc_csr(n, ptr(offsets), ptr(cols), ptr(labels), _vref(variant), ctypes.byref(h)),
          "gconn_plan_create_cc_csr")
    return h


def gconn_plan_create_forest_csr(n, offsets, cols, forest, forest_count, labels=None, variant=None):
    h = ctypes.c_void_p()
    check(lib().gconn_plan_create_forest_csr(n, ptr(offsets), ptr(cols), ptr(forest), ptr(forest_count), ptr(labels),
                                             _vref(variant), ctypes.byref(h)), "gconn_plan_create_forest_csr")
    return h


def gconn_plan_create_cc_csr32(n, offsets, cols, labels, variant=None):
    h = ctypes.c_void_p()
    check(lib().gconn_plan_create_cc_csr32(n, ptr(offsets), ptr(cols), ptr(labels), _vref(variant),
                                           ctypes.byref(h)), "gconn_plan_create_cc_csr32")
    return h


def gconn_plan_create_forest_csr32(n, offsets, cols, forest, forest_count, labels=None, variant=None):
    h = ctypes.c_void_p()
    check(lib().gconn_plan_create_forest_csr32(n, ptr(offsets), ptr(cols), ptr(forest), ptr(forest_count),
                                               ptr(labels), _vref(variant), ctypes.byref(h)),
          "gconn_plan_create_forest_csr32")
    return h


def gconn_plan_run(h, stream=None):
    check(lib().gconn_plan_run(h, stream_handle(stream)), "gconn_plan_run")


def gconn_plan_destroy(h):
    check(lib().gconn_plan_destroy(h), "gconn_plan_destroy")


def gconn_profile_sync():
    check(lib().gconn_profile_sync(), "gconn_profile_sync")


def gconn_server_config_default() -> gconn_server_config:
    c = gconn_server_config()
    check(lib().gconn_server_config_default(ctypes.byref(c)), "gconn_server_config_default")
    return c


def gconn_server_create(cfg=None):
    h = ctypes.c_void_p()
    check(lib().gconn_server_create(_vref(cfg), ctypes.byref(h)), "gconn_server_create")
    return h


def gconn_server_open_session(h, n, variant=None) -> int:
    sid = ctypes.c_uint32()
    check(lib().gconn_server_open_session(h, n, _vref(variant), ctypes.byref(sid)), "gconn_server_open_session")
    return int(sid.value)


def gconn_server_submit(h, session, op, count, pairs, result=None) -> int:
    t = ctypes.c_uint64()
    check(lib().gconn_server_submit(h, session, op, count, ptr(pairs), ptr(result), ctypes.byref(t)),
          "gconn_server_submit")
    return int(t.value)


def gconn_server_wait(h, ticket) -> float:
    ms = ctypes.c_double()
    check(lib().gconn_server_wait(h, ticket, ctypes.byref(ms)), "gconn_server_wait")
    return float(ms.value)


def gconn_server_labels(h, session, labels):
    check(lib().gconn_server_labels(h, session, ptr(labels)), "gconn_server_labels")


def gconn_server_close_session(h, session):
    check(lib().gconn_server_close_session(h, session), "gconn_server_close_session")


def gconn_server_stats(h):
    a, b_, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().gconn_server_stats(h, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)), "gconn_server_stats")
    return {"launches": int(a.value), "groups": int(b_.value), "requests": int(c.value)}


def gconn_server_destroy(h):
    check(lib().gconn_server_destroy(h), "gconn_server_destroy")


def gconn_cc_csr_stats(n, offsets, cols, labels, variant=None, stream=None) -> gconn_sample_stats:
    out = gconn_sample_stats()
    check(lib().gconn_cc_csr_stats(n, ptr(offsets), ptr(cols), ptr(labels), _vref(variant), ctypes.byref(out),
                                   stream_handle(stream)), "gconn_cc_csr_stats")
    return out


def gconn_sync(stream=None):
    check(lib().gconn_sync(stream_handle(stream)), "gconn_sync")


def gconn_status_str(status: int) -> str:
    return lib().gconn_status_str(status).decode()


def gconn_launch_count() -> int:
    return int(lib().gconn_launch_count())


def gconn_release_cached():
    check(lib().gconn_release_cached(), "gconn_release_cached")


def gconn_profile_enable(on: bool = True):
    check(lib().gconn_profile_enable(1 if on else 0), "gconn_profile_enable")


def gconn_profile_select(names=None):
    """Time only the named kernels (comma-separated string or list); None: all."""
    if names is not None and not isinstance(names, str):
        names = ",".join(names)
    check(lib().gconn_profile_select(None if names is None else names.encode()), "gconn_profile_select")


def gconn_profile_reset():
    check(lib().gconn_profile_reset(), "gconn_profile_reset")


def gconn_profile_get():
    """All per-kernel totals as {name: (launches, total_ms)}."""
    out = {}
    i = 0
    L = lib()
    while True:
        name = ctypes.c_char_p()
        cnt = ctypes.c_uint64()
        ms = ctypes.c_double()
        if L.gconn_profile_get(i, ctypes.byref(name), ctypes.byref(cnt), ctypes.byref(ms)) != GCONN_OK:
            break
        out[name.value.decode()] = (int(cnt.value), float(ms.value))
        i += 1
    return out
