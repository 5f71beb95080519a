"""Host-side parts of the selector's training pipeline, on the CPU: the R-MAT
parameter rule for the training graphs, the training and held-out graph sets
(the ranges of the learned-selector workload: R-MAT scales 18-24, edgefactor
8-32, A in 0.45-0.65; grids 64^3-192^3; Erdos-Renyi degree 4-32; held out:
R-MAT scale 25 edgefactor 16 and grid 256^3), the thinning of long
traversals' rows, and the seeded He-uniform start."""
import re

import numpy as np
import pytest

from paper_1104_4518_gb300 import selector


def test_rmat_parameters_sum_to_one():
    for a in (0.45, 0.5, 0.57, 0.6, 0.65):
        b = selector.rmat_bc(a)
        assert a + 2 * b + 0.05 == pytest.approx(1.0)
        assert b > 0.05  # D stays the smallest quadrant


def test_training_set_spans_the_workload_ranges():
    specs = selector.training_graphs()
    rmat = [re.match(r"rmat-s(\d+)-ef(\d+)-a([\d.]+)$", n) for n, *_ in specs]
    rmat = [(int(m[1]), int(m[2]), float(m[3])) for m in rmat if m]
    assert {s for s, _, _ in rmat} == set(range(18, 25))
    assert {e for _, e, _ in rmat} == {8, 16, 32}
    assert min(a for *_, a in rmat) == 0.45 and max(a for *_, a in rmat) == 0.65
    grids = sorted(int(n[4:]) for n, *_ in specs if n.startswith("grid"))
    assert grids[0] == 64 and grids[-1] == 192
    er = [re.match(r"er-(\d+)-d(\d+)$", n) for n, *_ in specs]
    degs = sorted(int(m[2]) for m in er if m)
    assert degs[0] == 4 and degs[-1] == 32
    names = [n for n, *_ in specs]
    assert len(names) == len(set(names))
    held = dict((n, (rs, k)) for n, _, rs, k in selector.heldout_graphs())
    assert set(held) == {"rmat-s25-ef16", "grid256"} and held["rmat-s25-ef16"][1] == 8
    assert not set(held) & set(names)  # held out means not trained on


def test_thin_rows_keeps_ends_and_order():
    X = np.arange(500 * 12, dtype=np.float32).reshape(500, 12)
    T = np.arange(500 * 4, dtype=np.float32).reshape(500, 4)
    Xs, Ts = selector.thin_rows(X, T)
    assert Xs.shape[0] <= 64 and Xs.shape[0] == Ts.shape[0]
    rows = Xs[:, 0] / 12
    assert np.all(np.diff(rows) > 0)  # order kept, no repeats
    assert set(range(8)) <= set(rows.astype(int)) and set(range(492, 500)) <= set(rows.astype(int))
    assert np.array_equal(Ts[:, 0] / 4, rows)  # X and T rows stay paired
    small_X, small_T = X[:40], T[:40]
    a, b = selector.thin_rows(small_X, small_T)
    assert a is small_X and b is small_T


def test_he_uniform_start():
    p = selector.init_params(3)
    assert p.dtype == np.float32 and p.shape == (5252,)
    assert np.array_equal(p, selector.init_params(3)) and not np.array_equal(p, selector.init_params(4))
    off = 0
    for fan_in, fan_out in ((12, 64), (64, 64), (64, 4)):
        w = p[off:off + fan_in * fan_out]
        bound = np.sqrt(6.0 / fan_in)
        assert np.all(np.abs(w) <= bound) and np.abs(w).max() > 0.9 * bound
        off += fan_in * fan_out
        assert np.all(p[off:off + fan_out] == 0)  # biases start at zero
        off += fan_out
    assert off == 5252
