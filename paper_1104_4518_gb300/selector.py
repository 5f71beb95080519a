"""Training and held-out evaluation of the per-level variant selector.

The selector network (12 -> 64 -> 64 -> 4, float32, see include/bfs.h) predicts
log2 level times of the four expansion variants from frontier statistics; the
traversal takes the argmin at every level.  Training data come from the
library's own traversals (`bfs_selector_collect`: every variant forced at
every level, median of repeated runs), training runs on the GPU through the
library's forward / backward / Adam kernels (`bfs_selector_train`).  This
module only orchestrates those calls and writes the weights file.

Training graphs (seeded): R-MAT scales 18-24 with edgefactor 8-32 and
A in 0.45-0.65 (B = C = (0.95 - A) / 2, D = 0.05), 3D grids 64^3-192^3 and
Erdos-Renyi graphs of average degree 4-32.  Held-out: R-MAT scale 25
edgefactor 16 and the 256^3 grid.

    python -m paper_1104_4518_gb300.selector train   [--out weights.bin] [--report report.json]
    python -m paper_1104_4518_gb300.selector evaluate [--weights weights.bin]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "selector_weights.bin")


def rmat_bc(a: float):
    """B = C = (0.95 - A) / 2 with D = 0.05 when A varies."""
    return (0.95 - a) / 2


def training_graphs():
    """(name, factory, roots seed, number of roots) of the training set."""
    specs = []
    rm = [(18, 8, .45), (18, 16, .57), (18, 32, .65), (19, 8, .60), (19, 16, .55), (19, 32, .50),
          (20, 8, .65), (20, 16, .45), (20, 32, .45), (21, 8, .55), (21, 16, .60), (21, 32, .65),
          (22, 8, .50), (22, 16, .57), (22, 32, .57), (23, 8, .62), (23, 16, .45), (23, 32, .52),
          (24, 8, .57), (24, 16, .65), (24, 32, .48)]
    for i, (sc, ef, a) in enumerate(rm):
        b = rmat_bc(a)
        specs.append((f"rmat-s{sc}-ef{ef}-a{a}", (lambda sc=sc, ef=ef, a=a, b=b, i=i:
                                                   inputs.rmat(sc, ef, a, b, b, seed=600 + i)), 700 + i, 6))
    for N in (64, 96, 128, 160, 192):
        specs.append((f"grid{N}", (lambda N=N: inputs.grid3d(N)), None, 1))
    for i, (lg, d) in enumerate([(20, 4), (20, 16), (21, 8), (21, 16), (22, 4), (22, 32)]):
        specs.append((f"er-{lg}-d{d}", (lambda lg=lg, d=d, i=i: inputs.erdos_renyi(1 << lg, d, seed=650 + i)),
                      750 + i, 3))
    return specs


def thin_rows(X, T, levels_per_run: int = 64):
    """Keeps at most about `levels_per_run` rows of a long traversal (grids have hundreds of
    near-identical levels), always keeping the first and last eight levels."""
    n = X.shape[0]
    if n <= levels_per_run:
        return X, T
    keep = np.zeros(n, dtype=bool)
    keep[:8] = True
    keep[-8:] = True
    keep[np.linspace(0, n - 1, levels_per_run - 16).astype(int)] = True
    return X[keep], T[keep]


def heldout_graphs():
    return [("rmat-s25-ef16", lambda: inputs.rmat(25, 16, seed=7), 107, 8),
            ("grid256", lambda: inputs.grid3d(256), None, 1)]


def _device_graph(el):
    import torch

    import paper_1104_4518_gb300 as bfs
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n)
    torch.cuda.synchronize()
    return g


def _roots(el, seed, k):
    if seed is None:
        return np.zeros(1, np.int32)  # grids: the corner
    return inputs.roots(el, k, seed)


def collect(specs, reps: int = 3, log=print):
    import paper_1104_4518_gb300 as bfs

    Xs, Ts = [], []
    for name, make, rseed, k in specs:
        t0 = time.time()
        el = make()
        g = _device_graph(el)
        xs, ts = [], []
        for r in _roots(el, rseed, k):
            x, t = bfs.bfs_selector_collect(g, [int(r)], reps=reps)
            x, t = thin_rows(x, t)
            xs.append(x)
            ts.append(t)
        X, T = np.concatenate(xs), np.concatenate(ts)
        g.destroy()
        Xs.append(X)
        Ts.append(T)
        log(f"collect {name}: {X.shape[0]} rows in {time.time() - t0:.1f} s")
    return np.concatenate(Xs), np.concatenate(Ts)


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights from seeded uniforms, zero biases (same rule as the oracle)."""
    rng = np.random.default_rng(seed)
    u = rng.random(5252)
    w = np.zeros(5252, dtype=np.float64)
    off = 0
    for fan_in, fan_out in ((12, 64), (64, 64), (64, 4)):
        size = fan_in * fan_out
        w[off:off + size] = (2 * u[off:off + size] - 1) * np.sqrt(6.0 / fan_in)
        off += size + fan_out
    return w.astype(np.float32)


def train(X, T, steps: int = 4000, lr: float = 3e-3, seed: int = 1):
    import torch

    import paper_1104_4518_gb300 as bfs

    p = torch.from_numpy(init_params(seed)).cuda()
    hist = torch.empty(steps, dtype=torch.float32, device="cuda")
    bfs.bfs_selector_train(p, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), steps, lr=lr,
                           loss_history=hist)
    return p.cpu().numpy(), hist.cpu().numpy()


def _time_run(g, s, opts, reps=3):
    import torch

    import paper_1104_4518_gb300 as bfs
    n = g.n
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    bfs.bfs_run(g, s, parent, level, opts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        bfs.bfs_run(g, s, parent, level, opts)
    e1.record()
    torch.cuda.synchronize()
    bfs.bfs_sync(g)
    return e0.elapsed_time(e1) / reps


def evaluate_graph(g, roots, weights, reps: int = 3):
    """Per-root times (ms) of heuristic, learned, exhaustive-best schedule and fixed variants,
    plus the learned selector's regret against the per-level best (from forced-run level times)."""
    import paper_1104_4518_gb300 as bfs

    out = []
    for s in roots:
        s = int(s)
        X, T = bfs.bfs_selector_collect(g, [s], reps=reps)
        best_sched = [int(v) for v in np.argmin(T, axis=1)]
        row = {"root": s, "levels": int(X.shape[0])}
        for v in range(bfs.BFS_NUM_VARIANTS):
            row[f"forced_{bfs.VARIANT_NAMES[v]}_ms"] = _time_run(
                g, s, bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v), reps)
        row["heuristic_ms"] = _time_run(g, s, bfs.RunOptions(selector=bfs.BFS_SELECT_HEURISTIC), reps)
        row["best_schedule_ms"] = _time_run(
            g, s, bfs.RunOptions(selector=bfs.BFS_SELECT_SCHEDULE, schedule=best_sched), reps)
        bfs.bfs_selector_set_params(weights)
        o = bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED, stats_levels=8192)
        bfs.run(g, s, o)
        learned_sched = [st["variant"] for st in o.stats()]
        row["learned_ms"] = _time_run(g, s, bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED), reps)
        bfs.bfs_selector_set_params(None)
        lt = np.exp2(T) / 1e3  # per-level ms of each variant
        k = min(len(learned_sched), lt.shape[0])
        row["learned_level_sum_ms"] = float(sum(lt[i, learned_sched[i]] for i in range(k)))
        row["best_level_sum_ms"] = float(lt[:k].min(axis=1).sum())
        row["regret_ms"] = row["learned_level_sum_ms"] - row["best_level_sum_ms"]
        row["learned_matches_best_levels"] = int(sum(learned_sched[i] == best_sched[i] for i in range(k)))
        if k <= 16:
            row["best_schedule"] = best_sched
            row["learned_schedule"] = learned_sched[:k]
            row["level_ms"] = [[round(float(x), 4) for x in lt[i]] for i in range(k)]
        out.append(row)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="train / evaluate the per-level variant selector")
    ap.add_argument("cmd", choices=["train", "evaluate"])
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--weights", default=DEFAULT_WEIGHTS)
    ap.add_argument("--report", default=None)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
    import paper_1104_4518_gb300 as bfs

    report = {}
    if args.cmd == "train":
        X, T = collect(training_graphs(), reps=args.reps)
        w, hist = train(X, T, steps=args.steps, lr=args.lr)
        w.astype("<f4").tofile(args.out)
        report = {"rows": int(X.shape[0]), "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
                  "steps": args.steps, "lr": args.lr, "weights": os.path.basename(args.out)}
        print(json.dumps(report))
    else:
        w = np.fromfile(args.weights, dtype="<f4")
        assert w.shape == (bfs.BFS_MLP_PARAMS,)
        for name, make, rseed, k in heldout_graphs():
            el = make()
            g = _device_graph(el)
            rows = evaluate_graph(g, _roots(el, rseed, k), w, reps=args.reps)
            g.destroy()
            report[name] = rows
            for r in rows:
                print(name, json.dumps(r), flush=True)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
