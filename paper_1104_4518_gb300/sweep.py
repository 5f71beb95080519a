"""GTEPS against average degree at a fixed number of edges (the paper's
edgefactor study, Sec. 6), on one GPU.

R-MAT graphs (A, B, C, D = .57, .19, .19, .05, relabelled) with edgefactor
4, 8, 16, 32 and 64 and the scale that keeps 2^27 generated undirected edges
(scale 25 down to scale 21); for each graph, 16 seeded roots of degree >= 1
and the harmonic-mean GTEPS of: the heuristic selector, every variant forced
at every level, the learned selector (when weights are shipped), and the
batched traversal of the 16 roots.  Edges per root are the undirected edges
of the root's component, as in bench.py.

    python -m paper_1104_4518_gb300.sweep [--report sweep.json] [--roots 16]
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LOG2_EDGES = 27


def _hmean(edges, ms):
    rates = [e / (t / 1e3) / 1e9 for e, t in zip(edges, ms) if t > 0]
    return len(rates) / sum(1.0 / r for r in rates) if rates else 0.0


def measure(ef: int, nroots: int = 16, seed: int = 40, reps: int = 2) -> dict:
    import torch

    import paper_1104_4518_gb300 as bfs

    scale = LOG2_EDGES - int(np.log2(ef))
    el = inputs.rmat(scale, ef, seed=seed + ef)
    roots = [int(r) for r in inputs.roots(el, nroots, seed + 100 + ef)]
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n)
    del el
    n = g.n
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    edges = []
    for s in roots:  # component edges of every root
        o = bfs.RunOptions(want_counts=True)
        bfs.bfs_run(g, s, parent, level, o)
        bfs.bfs_sync(g)
        edges.append(o.edges)

    def timed(make_opts):
        for s in roots:
            bfs.bfs_run(g, s, parent, level, make_opts())
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in roots]
            for (a, b), s in zip(ev, roots):
                a.record()
                bfs.bfs_run(g, s, parent, level, make_opts())
                b.record()
            torch.cuda.synchronize()
            ms = [a.elapsed_time(b) for a, b in ev]
            best = ms if best is None else [min(x, y) for x, y in zip(best, ms)]
        return round(_hmean(edges, best), 3)

    row = {"edgefactor": ef, "scale": scale, "n": n, "nnz": g.nnz, "roots": nroots,
           "mean_component_edges": float(np.mean(edges))}
    row["heuristic_gteps"] = timed(lambda: bfs.RunOptions(selector=bfs.BFS_SELECT_HEURISTIC))
    for v in range(bfs.BFS_NUM_VARIANTS):
        row[f"forced_{bfs.VARIANT_NAMES[v]}_gteps"] = timed(
            lambda v=v: bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=v))
    wpath = os.path.join(HERE, "selector_weights.bin")
    if os.path.exists(wpath):
        bfs.bfs_selector_load(wpath)
        row["learned_gteps"] = timed(lambda: bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED))
        bfs.bfs_selector_set_params(None)
    pb = torch.empty((nroots, n), dtype=torch.int32, device="cuda")
    lb = torch.empty_like(pb)
    bfs.bfs_run_batch(g, roots, pb, lb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        bfs.bfs_run_batch(g, roots, pb, lb)
    e1.record()
    torch.cuda.synchronize()
    bms = e0.elapsed_time(e1) / reps
    row["batched_gteps"] = round(sum(edges) / (bms / 1e3) / 1e9, 3)
    g.destroy()
    return row


def main(argv=None):
    ap = argparse.ArgumentParser(description="GTEPS against average degree at fixed edges")
    ap.add_argument("--report", default=None)
    ap.add_argument("--roots", type=int, default=16)
    ap.add_argument("--edgefactors", default="4,8,16,32,64")
    args = ap.parse_args(argv)
    rows = []
    for ef in [int(x) for x in args.edgefactors.split(",")]:
        row = measure(ef, args.roots)
        rows.append(row)
        print(json.dumps(row), flush=True)
    if args.report:
        with open(args.report, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
