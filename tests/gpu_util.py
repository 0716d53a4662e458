"""Helpers for the GPU parity tests: device copies of seeded inputs and
calls through the C ABI (via the ctypes binding)."""
import numpy as np

import graphgen

UF_COMBOS = []
for _l in ["async", "hooks", "early"]:
    for _f in ["naive", "compress", "split", "halve"]:
        UF_COMBOS.append((_l, _f, "none"))
for _f in ["naive", "split", "halve"]:
    for _s in ["split_one", "halve_one", "splice"]:
        UF_COMBOS.append(("remcas", _f, _s))
UF_COMBOS += [("jtb", "naive", "none"), ("jtb", "twotrysplit", "none")]
for _f in ["naive", "split", "halve"]:
    for _s in ["split_one", "halve_one", "splice"]:
        UF_COMBOS.append(("remlock", _f, _s))
UF_COMBOS += [("afforest", "naive", "none"), ("eclcc", "naive", "none")]

LT_ALL = ["CUSA", "CRSA", "PUSA", "PRSA", "PUS", "PRS", "EUSA", "EUS",
          "CUFA", "CRFA", "PUFA", "PRFA", "PUF", "PRF", "EUFA", "EUF"]
LT_ROOT = ["CRSA", "PRSA", "PRS", "CRFA", "PRFA", "PRF"]


UF_FOREST = [c for c in UF_COMBOS if not (c[0] in ("remcas", "remlock") and c[2] == "splice")]


def combo_id(c):
    return "-".join(c)


def dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    elif a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def small_graphs():
    """Seeded inputs that span several tiles with a ragged tail, plus the
    degenerate shapes of the method."""
    out = []
    out.append(("er", 5003, graphgen.er(5003, 12345, 1)))
    out.append(("er_sparse", 20011, graphgen.er(20011, 9001, 2)))
    out.append(("rmat12", 4096, graphgen.rmat(12, 30001, 3)))
    n, e = graphgen.grid_paths(40, 0.05, 6, 700, 4)
    out.append(("grid_paths", n, e))
    k = 3001
    path = np.stack([np.arange(k - 1, 0, -1), np.arange(k - 2, -1, -1)], 1).astype(np.uint32)
    out.append(("rev_path", k, path))
    star = np.stack([np.full(4000, 4000), np.arange(4000)], 1).astype(np.uint32)
    out.append(("star_hi_center", 4001, star))
    out.append(("empty", 777, np.zeros((0, 2), np.uint32)))
    loops = np.stack([np.arange(500), np.arange(500)], 1).astype(np.uint32)
    out.append(("self_loops", 500, loops))
    dup = np.tile(np.array([[7, 3], [3, 7], [1, 2]], np.uint32), (1000, 1))
    out.append(("duplicates", 10, dup))
    out.append(("one_vertex", 1, np.zeros((3, 2), np.uint32)))
    return out
