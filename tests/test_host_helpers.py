"""Host-only helpers of the package, on the CPU: the autotune cache (key,
hit, miss, persistence; the GPU calls replaced by fakes) and the degree
sweep's choice of scales at a fixed edge count."""
import json

import numpy as np
import pytest

import paper_1104_4518_gb300 as bfs
from paper_1104_4518_gb300 import sweep


class FakeGraph:
    def __init__(self, n, nnz):
        self.n, self.nnz = n, nnz

    def info(self):
        return self.n, self.nnz, 1


def test_graph_class_is_size_and_degree():
    assert bfs.graph_class(FakeGraph(1 << 22, 32 << 22)) == "n2^22-deg32"
    assert bfs.graph_class(FakeGraph(3 << 20, 3 << 23)) == "n2^22-deg8"  # log2(3 * 2^20) rounds to 22
    assert bfs.graph_class(FakeGraph(1, 0)) == "n2^0-deg0"


def test_autotune_cache_miss_then_hit(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FAKE GB300")
    calls = {"tune": 0, "set": []}

    def fake_autotune(g, roots, stream=None):
        calls["tune"] += 1
        t = bfs.bfs_tuning()
        t.alpha, t.beta, t.batch_width = 30.0, 24.0, 64
        return t

    current = bfs.bfs_tuning()

    def fake_set(g, **knobs):
        calls["set"].append(knobs)
        for k, v in knobs.items():
            setattr(current, k, v)

    monkeypatch.setattr(bfs, "bfs_autotune", fake_autotune)
    monkeypatch.setattr(bfs, "bfs_set_tuning", fake_set)
    monkeypatch.setattr(bfs, "bfs_get_tuning", lambda g: current)
    path = str(tmp_path / "tuning.json")
    g = FakeGraph(1 << 20, 16 << 20)
    t1 = bfs.bfs_autotune_cached(g, [0, 1], path)
    assert calls["tune"] == 1 and t1.alpha == 30.0
    cache = json.load(open(path))
    assert list(cache) == ["n2^20-deg16|FAKE GB300"] and cache["n2^20-deg16|FAKE GB300"]["alpha"] == 30.0
    t2 = bfs.bfs_autotune_cached(FakeGraph(1 << 20, 16 << 20), [5], path)  # same class: no timing
    assert calls["tune"] == 1 and calls["set"] and t2.alpha == 30.0
    bfs.bfs_autotune_cached(FakeGraph(1 << 21, 16 << 21), [0], path)  # another class: tuned and added
    assert calls["tune"] == 2 and len(json.load(open(path))) == 2


def test_sweep_keeps_the_edge_count_fixed():
    for ef in (4, 8, 16, 32, 64):
        scale = sweep.LOG2_EDGES - int(np.log2(ef))
        assert (1 << scale) * ef == 1 << sweep.LOG2_EDGES
    assert sweep._hmean([1e9, 1e9], [1000.0, 500.0]) == pytest.approx(4.0 / 3.0)  # times in ms
    assert sweep._hmean([], []) == 0.0
