"""Host logic of bench.py's edge-inspection sweep, run on CPU with a stand-in
for the incremental handle (the real handle needs a GPU): one JSON line per
(finish, batch size) with the counts the handle reports."""
import json
import sys
import types


def test_edge_inspect_lines(monkeypatch, capsys):
    import torch
    import bench

    class FakeInc:   # reports 3 inspections per inserted edge
        def __init__(self, n, v, stream):
            self.last = self.total = 0

        def insert(self, e):
            self.last = 3 * int(e.shape[0])
            self.total += self.last

        def edges_inspected(self):
            return self.last, self.total

        def close(self):
            pass

    class Ev:
        def __init__(self, enable_timing=True):
            pass

        def record(self, stream=None):
            pass

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return 2.0

    fake = types.SimpleNamespace(build=lambda: None, Incremental=FakeInc, gconn_sync=lambda stream=None: None,
                                 make_variant=lambda **kw: kw)
    monkeypatch.setitem(sys.modules, "paper_2008_11839_gb300", fake)
    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda: None)
    real_device = torch.device
    monkeypatch.setattr(torch, "device", lambda *a: real_device("cpu"))
    monkeypatch.setattr(bench, "INC_N_SCALE", 10)
    bench.run_edge_inspect(types.SimpleNamespace(inspect_variants="sv,lt/PRS"))
    lines = [json.loads(x) for x in capsys.readouterr().out.splitlines() if x.startswith("{")]
    assert [(d["variant"], d["batch"]) for d in lines] == \
        [(v, b) for v in ("sv", "lt/PRS") for b in (10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7)]
    for d in lines:
        assert d["edges"] == 1 << 24 and d["inspected"] == 3 * d["edges"]
        assert d["inspected_per_edge"] == 3.0 and d["max_batch_inspections_per_edge"] == 3.0
        assert d["batches"] == -(-d["edges"] // d["batch"]) and d["ms"] == 2.0
