import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libgconn")
    config.addinivalue_line("markers", "slow: long-running full-size check")


def golden_path(name: str) -> str:
    return os.path.join(ROOT, "tests", "golden", name)


def read_cc_golden(name: str):
    """Parse a tests/golden/cc_*.txt fixture -> (n, edges list, labels list)."""
    n, edges, labels, in_edges = None, [], None, False
    with open(golden_path(name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("n "):
                n = int(line.split()[1])
            elif line == "edges":
                in_edges = True
            elif line.startswith("labels"):
                labels = [int(x) for x in line.split()[1:]]
                in_edges = False
            elif in_edges:
                u, v = line.split()
                edges.append((int(u), int(v)))
    return n, edges, labels


def read_inc_golden(name: str):
    """Parse tests/golden/inc_*.txt -> (n, ops, final labels)."""
    n, ops, labels = None, [], None
    with open(golden_path(name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t = line.split()
            if t[0] == "n":
                n = int(t[1])
            elif t[0] == "insert":
                ops.append(("insert", int(t[1]), int(t[2])))
            elif t[0] == "query":
                ops.append(("query", int(t[1]), int(t[2]), int(t[3])))
            elif t[0] == "labels":
                labels = [int(x) for x in t[1:]]
    return n, ops, labels
