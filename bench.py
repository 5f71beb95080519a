#!/usr/bin/env python3
"""Benchmark of the GB300 BFS library: GTEPS on the paper-shaped synthetic workloads.

Default workload (no flags): R-MAT scale 26, edgefactor 16, (A,B,C,D) =
(.57,.19,.19,.05), seeded relabelling, 64 seeded roots of degree >= 1 (graph seed
3, root seed 103): the largest plain single-root configuration that fits one
GPU.  One step = one single-root traversal (bfs_run, heuristic selector) from
each of the 64 roots.  TEPS follows Sec. 6 of the paper: the edges counted for
a root are the undirected edges of its component, and only roots in the large
component enter the mean (the harmonic mean of per-root GTEPS).  Inputs (CSR
adjacency, 8.6 GB) are far larger than the 129 MB L2, so no flush is done
between roots.

Printed (rank 0): one JSON line with value, roofline of the level-loop kernel,
the oracle CPU baseline, the end-to-end figure (host outputs), clocks sampled
during the timed region and side comparisons (batched, learned selector).

`--impl reference` times the CPU oracle on the same workload instead.
Multi-GPU (torchrun, N > 1): independent replicas, each rank with its own 64
seeded roots; no collective on the data path (the traversal does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1104_4518_gb300 import inputs  # noqa: E402

WORKLOADS = {
    "rmat22": dict(kind="rmat", scale=22, ef=16, graph_seed=2, root_seed=102, roots=64),
    "rmat16": dict(kind="rmat", scale=16, ef=16, graph_seed=1, root_seed=101, roots=16),
    "rmat23": dict(kind="rmat", scale=23, ef=16, graph_seed=8, root_seed=108, roots=64),
    "rmat24": dict(kind="rmat", scale=24, ef=16, graph_seed=4, root_seed=104, roots=64),
    "rmat26": dict(kind="rmat", scale=26, ef=16, graph_seed=3, root_seed=103, roots=64),
    "grid128": dict(kind="grid", N=128, roots=1),
    "grid256": dict(kind="grid", N=256, roots=1),
}
METRIC = "GTEPS (harmonic mean, 64 roots) & % HBM roofline; batched/learned vs plain"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def workload_name(wl: dict) -> str:
    if wl["kind"] == "rmat":
        return (f"R-MAT scale {wl['scale']} edgefactor {wl['ef']} (A,B,C,D=.57,.19,.19,.05, relabelled), "
                f"{wl['roots']} seeded roots, single-root BFS per root")
    return f"3D 7-point grid {wl['N']}^3 rooted at the corner"


def make_workload(wl: dict, rank: int = 0):
    if wl["kind"] == "rmat":
        el = inputs.rmat(wl["scale"], wl["ef"], seed=wl["graph_seed"])
        roots = inputs.roots(el, wl["roots"], wl["root_seed"] + 1000 * rank)
    else:
        el = inputs.grid3d(wl["N"])
        roots = np.zeros(1, np.int32)
    return el, roots


# ---------------- replicas (host logic, tested with gloo on CPU) ----------------

def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def aggregate(local_time_s: float, local_edges: int, group=None):
    """Max of the ranks' timed-region lengths and sum of their traversed edges."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return local_time_s, local_edges
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([local_time_s], dtype=torch.float64, device=dev)
    e = torch.tensor([float(local_edges)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(e, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), int(e.item())


def barrier():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------- measurement helpers ----------------

class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        time.sleep(0.05)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_hbm_peak():
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal


def profile_summary(name: str):
    """The `- key: value` lines of a committed ncu summary under profiles/, or None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        text = open(path).read()
    except OSError:
        return None
    kv = {}
    for line in text.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    return kv


def profile_traffic(name: str):
    """Per-launch DRAM traffic from a committed ncu summary, if it matches the current kernel source."""
    kv = profile_summary(name)
    if kv is None or kv.get("source_sha256") != kernel_source_hash():
        return None
    try:
        return float(kv["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ncu captures stay on small cases; larger R-MAT workloads scale this one.
SCALED_CAPTURE = "level_loop_rmat23.md"


def traffic_estimate(workload: str, algo_bytes: float):
    """(DRAM bytes per level-loop launch, how it was obtained) for `workload`.

    A capture of the same workload counts as it is.  Otherwise an R-MAT
    workload takes the scale-23 capture scaled by the ratio of algorithmic bytes
    per launch: a traversal's traffic grows with the rows, offsets and outputs
    it touches, which is what the algorithmic bytes count.  Captures whose
    kernel source hash differs from the current source count as missing."""
    own = profile_traffic(f"level_loop_{workload}.md")
    if own is not None:
        return own, f"ncu capture of this workload (profiles/level_loop_{workload}.md)"
    kv = profile_summary(SCALED_CAPTURE)
    if workload.startswith("rmat") and kv is not None and kv.get("source_sha256") == kernel_source_hash():
        try:
            t, a = float(kv["traffic_bytes_per_launch"]), float(kv["algorithmic_bytes_per_launch"])
        except (KeyError, ValueError):
            return None, "scaled capture lacks its byte counts"
        return t * algo_bytes / a, (f"profiles/{SCALED_CAPTURE} (R-MAT scale 23, one launch) scaled by the "
                                    f"ratio of algorithmic bytes per launch, {algo_bytes / a:.3f}")
    return None, "no ncu capture of the current kernel source"


def kernel_source_hash() -> str:
    import hashlib

    src = os.path.join(ROOT, "paper_1104_4518_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("level_loop.cu", "claims.cuh", "device_common.cuh", "internal.h", "mlp_device.cuh"):
        h.update(open(os.path.join(src, f), "rb").read())
    return h.hexdigest()[:16]


def harmonic_gteps(edges, times_s):
    rates = [e / t / 1e9 for e, t in zip(edges, times_s) if t > 0]
    return len(rates) / sum(1.0 / r for r in rates) if rates else 0.0


def bench_config(wl: dict, n: int, nnz: int, roots: int, n_large: int, teps_edges: int, world: int) -> dict:
    """The `config` object of the JSON line; both arms print the same one."""
    return {"workload": workload_name(wl), "n": int(n), "nnz": int(nnz), "roots": int(roots),
            "roots_in_large_component": int(n_large), "teps_edges_per_root": int(teps_edges),
            "selector": "heuristic", "l2": "not flushed: the CSR adjacency is larger than the 129 MB L2",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def oracle_census(og, roots):
    """(roots in the large component, that component's TEPS edges), found by the oracle.

    A BFS from the first root (of the first four) whose component holds more than 2/3 of the
    graph's edges settles it: every other component then has fewer than half
    as many edges, so the large-component rule (at least half the largest
    root component's edges) keeps exactly the roots that BFS reached.  If no
    root's component is that large, every root is traversed."""
    import oracle

    total = og.nnz // 2
    for s in roots[:4]:
        lv, _, _ = oracle.bfs(og, int(s))
        e = oracle.component_edges(og, lv)
        if 3 * e > 2 * total:
            return [int(r) for r in roots if lv[int(r)] >= 0], e
    res = oracle.bfs_many(og, [int(r) for r in roots])
    edges = [oracle.component_edges(og, lv) for lv, _, _ in res]
    emax = max(edges)
    large = [int(r) for r, e in zip(roots, edges) if e >= 0.5 * emax]
    return large, emax


def host_threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def timed_oracle_steps(og, step_roots, threads):
    """Wall time of one serial oracle BFS per entry of step_roots, `threads` at a time."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda s: oracle.bfs(og, s), step_roots))
    return time.perf_counter() - t0


def cpu_oracle_sample(el, roots_large, teps_edges):
    """The oracle (serial FIFO BFS + max-id parent pass) on the host cores: one
    large-component root per thread, all threads at once."""
    import oracle

    og = oracle.csr_of(el)
    threads = max(1, min(host_threads(), len(roots_large)))
    sample = [int(r) for r in roots_large[:threads]]
    wall = timed_oracle_steps(og, sample, threads)
    return {"value": teps_edges * len(sample) / wall / 1e9, "threads": threads,
            "sample": f"{len(sample)} large-component roots of the same graph, one serial oracle BFS per "
                      f"thread on {threads} threads at once ({wall:.1f} s wall); oracle CSR build not timed"}


def event_pair():
    import torch

    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def timed_roots(run_one, roots, steps, warmup, stream):
    """Per-root device times (ms, [steps][roots]) of run_one(root) after `warmup` untimed passes."""
    import torch

    for _ in range(warmup):
        for s in roots:
            run_one(int(s))
    torch.cuda.synchronize()
    ev = [[event_pair() for _ in roots] for _ in range(steps)]
    for k in range(steps):
        for i, s in enumerate(roots):
            ev[k][i][0].record(stream)
            run_one(int(s))
            ev[k][i][1].record(stream)
    torch.cuda.synchronize()
    return np.array([[a.elapsed_time(b) for a, b in row] for row in ev])


def batched_config_comparison(bfs, stream):
    """Batched against plain on R-MAT scale 24 (the batched configuration): GTEPS of one
    64-root batched traversal and of the 64 single-root traversals of the same roots."""
    import torch

    wl = WORKLOADS["rmat24"]
    el, roots = make_workload(wl)
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n)
    del el
    n, _, _ = g.info()
    rl = [int(s) for s in roots]
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    edges = []
    for s in rl:
        o = bfs.RunOptions(want_counts=True)
        bfs.bfs_run(g, s, parent, level, o)
        edges.append(o.edges)
    pt = timed_roots(lambda s: bfs.bfs_run(g, s, parent, level), rl, 3, 3, stream)
    plain_ms = float(pt.sum(axis=1).mean())
    pb = torch.empty((len(rl), n), dtype=torch.int32, device="cuda")
    lb = torch.empty((len(rl), n), dtype=torch.int32, device="cuda")
    for _ in range(3):
        bfs.bfs_run_batch(g, rl, pb, lb)
    e0, e1 = event_pair()
    e0.record(stream)
    for _ in range(3):
        bfs.bfs_run_batch(g, rl, pb, lb)
    e1.record(stream)
    torch.cuda.synchronize()
    bms = e0.elapsed_time(e1) / 3
    g.destroy()
    return {"workload": workload_name(wl), "batched_ms_per_64_roots": round(bms, 3),
            "plain_ms_per_64_roots": round(plain_ms, 3),
            "batched_gteps": round(sum(edges) / (bms / 1e3) / 1e9, 3),
            "plain_gteps": round(sum(edges) / (plain_ms / 1e3) / 1e9, 3)}


def ragged_comparison(bfs, stream):
    """32 independent R-MAT graphs (scales U{12..20}, one root each) traversed in one launch
    over their union (bfs_run_ragged) against 32 separate traversals of the same graphs."""
    import torch

    graphs, rts = inputs.ragged_rmat(32, 5)
    parts = [bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n)
             for el in graphs]
    u = bfs.bfs_graph_union(parts)
    levels = [torch.empty(el.n, dtype=torch.int32, device="cuda") for el in graphs]
    parents = [torch.empty(el.n, dtype=torch.int32, device="cuda") for el in graphs]
    edges = 0
    for gp, s, lv, pa in zip(parts, rts, levels, parents):
        o = bfs.RunOptions(want_counts=True)
        bfs.bfs_run(gp, s, pa, lv, o)
        edges += o.edges

    def union_run():
        bfs.bfs_run_ragged(u, rts, parents, levels)

    def separate_runs():
        for gp, s, lv, pa in zip(parts, rts, levels, parents):
            bfs.bfs_run(gp, s, pa, lv)

    out = {}
    for name, fn in (("one_launch", union_run), ("separate", separate_runs)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = event_pair()
        e0.record(stream)
        for _ in range(5):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        out[f"{name}_ms"] = round(ms, 3)
        out[f"{name}_gteps"] = round(edges / (ms / 1e3) / 1e9, 3)
    bfs.bfs_sync(u)
    u.destroy()
    for gp in parts:
        gp.destroy()
    out["teps_edges"] = int(edges)
    return out


# ---------------- the GPU arm ----------------

def run_gpu(args, wl):
    import torch
    import torch.distributed as dist

    import paper_1104_4518_gb300 as bfs

    rank, world, local_rank = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    el, roots = make_workload(wl, rank)
    g = bfs.bfs_graph_create_from_edges(torch.from_numpy(el.src).cuda(), torch.from_numpy(el.dst).cuda(), el.n)
    n, nnz, _ = g.info()
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    sel = bfs.BFS_SELECT_HEURISTIC
    base_opts = None

    # census (untimed): per-root component edges and reached vertices -> TEPS edges and compulsory bytes
    edges, reached = [], []
    for s in roots:
        o = bfs.RunOptions(selector=sel, want_counts=True)
        bfs.bfs_run(g, int(s), parent, level, o)
        edges.append(o.edges)
        reached.append(int((level >= 0).sum().item()))
    emax = max(edges)
    large = [i for i, e in enumerate(edges) if e >= 0.5 * emax]
    comp_bytes = [4 * 2 * e + 16 * r + 8 * n for e, r in zip(edges, reached)]

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        for s in roots:
            bfs.bfs_run(g, int(s), parent, level, base_opts)
    bfs.bfs_sync(g)

    R = len(roots)
    ev = [[event_pair() for _ in range(R)] for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t_start, t_end = event_pair()
    t_start.record(stream)
    for k in range(args.steps):
        for i, s in enumerate(roots):
            ev[k][i][0].record(stream)
            bfs.bfs_run(g, int(s), parent, level, base_opts)
            ev[k][i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    bfs.bfs_sync(g)
    total_ms = t_start.elapsed_time(t_end)
    root_ms = np.array([[ev[k][i][0].elapsed_time(ev[k][i][1]) for i in range(R)] for k in range(args.steps)])

    t_large = [root_ms[k, i] / 1e3 for k in range(args.steps) for i in large]
    e_large = [edges[i] for _ in range(args.steps) for i in large]
    hmean = harmonic_gteps(e_large, t_large)
    agg_time, agg_edges = aggregate(total_ms / 1e3, sum(edges[i] for i in large) * args.steps)
    value = hmean if world == 1 else agg_edges / agg_time / 1e9

    # roofline of the level-loop kernel (one launch per traversal)
    peak, peak_kind = measured_hbm_peak()
    algo_bytes = float(np.mean(comp_bytes))
    mean_launch_s = float(root_ms.mean()) / 1e3
    achieved = algo_bytes / mean_launch_s / 1e9
    traffic, traffic_how = traffic_estimate(args.workload, algo_bytes)
    roof = {"bound": "hbm", "kernel": "level_loop_kernel", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4),
            "peak_kind": f"{peak_kind} (copy bandwidth, burst: each launch timed alone)",
            "frac_of_nominal_8tbs": round(achieved / NOMINAL_HBM_GBS, 4),
            "algorithmic_bytes_per_launch": round(algo_bytes),
            "bytes_model": "4*sum deg(reached) + 16*n_reached + 8*n per root",
            "traffic": round(traffic) if traffic is not None else None, "traffic_source": traffic_how}
    if traffic is not None:
        dram = traffic / mean_launch_s / 1e9
        roof["dram_achieved"] = round(dram, 1)
        roof["dram_frac"] = round(dram / peak, 4)
        roof["traffic_over_algorithmic"] = round(traffic / algo_bytes, 3)

    cfg = bench_config(wl, n, nnz, R, len(large), edges[large[0]], world)
    result = {
        "metric": METRIC, "value": round(value, 3), "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded generators)",
        "config": cfg, "roofline": roof,
        "gpu_launches": args.steps * R * world,  # one level-loop launch per root, every rank
        "clocks": clk,
        "aggregate_gteps": round(agg_edges / agg_time / 1e9, 3),
        "root_ms": {"median": round(float(np.median(root_ms)), 4), "min": round(float(root_ms.min()), 4),
                    "max": round(float(root_ms.max()), 4)},
    }

    # end to end: host output buffers, device->host copies inside the timed region.  The
    # traversals are enqueued back to back with asynchronous host outputs (BFS_HOST_ASYNC),
    # alternating two pinned host buffer pairs, so that the copies of one root overlap the
    # next traversal; the wall clock runs from the first call to bfs_sync after the last.
    if not args.no_e2e:
        hbufs = [(torch.empty(n, dtype=torch.int32, pin_memory=True),
                  torch.empty(n, dtype=torch.int32, pin_memory=True)) for _ in range(2)]
        eo = bfs.RunOptions(selector=sel, host_outputs=True, host_async=True)
        e2e_steps = max(1, min(args.steps, 5))
        for j, s in enumerate(roots[:4]):
            bfs.bfs_run(g, int(s), *hbufs[j % 2], eo)
        bfs.bfs_sync(g)
        torch.cuda.synchronize()
        j = 0
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for i in large:
                bfs.bfs_run(g, int(roots[i]), *hbufs[j % 2], eo)
                j += 1
        bfs.bfs_sync(g)
        t_e2e = time.perf_counter() - t0
        e_e2e = sum(edges[i] for i in large) * e2e_steps
        t_all, e_all = aggregate(t_e2e, e_e2e)
        e2e = e_all / t_all / 1e9
        # the same calls one at a time (each waits for its copies): context for the overlap
        so = bfs.RunOptions(selector=sel, host_outputs=True)
        tt = []
        for i in large:
            t1 = time.perf_counter()
            bfs.bfs_run(g, int(roots[i]), *hbufs[0], so)
            tt.append(time.perf_counter() - t1)
        result["e2e"] = {"value": round(e2e, 3), "unit": "GTEPS", "h2d_bytes_per_step": 4 * R * world,
                         "d2h_bytes_per_step": 2 * 4 * n * R * world,
                         "synchronous_gteps": round(harmonic_gteps([edges[i] for i in large], tt), 3),
                         "how": "bfs_run with BFS_HOST_PTRS | BFS_HOST_ASYNC into pinned host buffers, the "
                                f"{len(large)} large-component roots x {e2e_steps} passes enqueued back to back "
                                "(the library copies parent and level out on its copy stream while the next "
                                "traversal runs), wall clock to bfs_sync after the last; synchronous_gteps: "
                                "the same calls waiting for their copies, harmonic mean per root"}

    # side comparisons (rank 0, once): batched, autotuned, learned selector and
    # every single variant forced at every level, on the same graph and roots
    if rank == 0 and not args.no_compare:
        comp = {}
        large_roots = [int(roots[i]) for i in large]
        e_one = [edges[i] for i in large]
        k = min(64, R)
        pb = torch.empty((k, n), dtype=torch.int32, device="cuda")
        lb = torch.empty((k, n), dtype=torch.int32, device="cuda")
        for _ in range(2):
            bfs.bfs_run_batch(g, [int(s) for s in roots[:k]], pb, lb)
        bfs.bfs_sync(g)
        e0, e1 = event_pair()
        reps = 3
        e0.record()
        for _ in range(reps):
            bfs.bfs_run_batch(g, [int(s) for s in roots[:k]], pb, lb)
        e1.record()
        torch.cuda.synchronize()
        del pb, lb
        bms = e0.elapsed_time(e1) / reps
        comp["batched_gteps"] = round(sum(edges[:k]) / (bms / 1e3) / 1e9, 3)
        comp["batched_ms_per_64_roots"] = round(bms, 3)
        comp["plain_ms_per_64_roots"] = round(float(root_ms[:, :k].sum(axis=1).mean()), 3)
        # learned selector: same roots, same steps and warm-up as the plain figure
        wpath = os.path.join(ROOT, "paper_1104_4518_gb300", "selector_weights.bin")
        if os.path.exists(wpath):
            bfs.bfs_selector_load(wpath)
            lo = bfs.RunOptions(selector=bfs.BFS_SELECT_LEARNED)
            lt = timed_roots(lambda s: bfs.bfs_run(g, s, parent, level, lo), large_roots, args.steps,
                             args.warmup, stream)
            bfs.bfs_sync(g)
            comp["learned_gteps"] = round(harmonic_gteps(e_one * args.steps, list(lt.flatten() / 1e3)), 3)
            bfs.bfs_selector_set_params(None)
        # one variant at every level (Sec. 5.2's comparison of expansion schemes): 4 roots each
        few = large_roots[:4]
        var = {}
        for vi, name in enumerate(bfs.VARIANT_NAMES):
            fo = bfs.RunOptions(selector=bfs.BFS_SELECT_FORCED, forced_variant=vi)
            ft = timed_roots(lambda s: bfs.bfs_run(g, s, parent, level, fo), few, 1, 1, stream)
            var[name] = round(harmonic_gteps(e_one[:len(few)], list(ft.flatten() / 1e3)), 3)
        bfs.bfs_sync(g)
        comp["forced_variant_gteps_4_roots"] = var
        # degree-binned expansion with the dense-frontier levels walked untiled (the heuristic's
        # schedule) against the same schedule with those levels on the 2D DCSC tiles
        sched = {}
        for s in few:
            so = bfs.RunOptions(stats_levels=256)
            bfs.bfs_run(g, s, parent, level, so)
            bfs.bfs_sync(g)
            sched[s] = [bfs.BFS_VARIANT_TILED if x["variant"] == bfs.BFS_VARIANT_PULL else x["variant"]
                        for x in so.stats()]
        tt = timed_roots(lambda s: bfs.bfs_run(g, s, parent, level, bfs.RunOptions(
            selector=bfs.BFS_SELECT_SCHEDULE, schedule=sched[s])), few, 1, 1, stream)
        ht = timed_roots(lambda s: bfs.bfs_run(g, s, parent, level), few, 1, 1, stream)
        comp["binned_with_pull_vs_tiled_4_roots"] = {
            "untiled_gteps": round(harmonic_gteps(e_one[:len(few)], list(ht.flatten() / 1e3)), 3),
            "tiled_gteps": round(harmonic_gteps(e_one[:len(few)], list(tt.flatten() / 1e3)), 3),
            "how": "the heuristic's per-level schedule (degree-binned / warp top-down levels, dense-frontier "
                   "levels) replayed with the dense-frontier levels on the 2D DCSC tiles"}
        # Sec. 4.2's sorted-output SpMSV: a BFS of expand-sort-compress steps, 2 roots
        try:
            srt = timed_roots(lambda s: bfs.bfs_run_sorted(g, s, parent, level, stream), large_roots[:2], 1, 1,
                              stream)
            comp["sorted_spmsv_bfs_2_roots"] = {
                "gteps": round(harmonic_gteps(e_one[:2], list(srt.flatten() / 1e3)), 3),
                "ms_per_root": round(float(srt.mean()), 3),
                "how": "bfs_run_sorted: every level one SpMSV with sorted output (the frontier's column entries "
                       "as 64-bit keys, radix-sorted, the last key of each row kept), a host loop over levels"}
        except bfs.BfsError as e:  # the keys of a level need about 28 bytes per frontier edge
            comp["sorted_spmsv_bfs_2_roots"] = {"error": str(e)}
        # symmetric half storage: a BFS that reads only the entries above the diagonal, 2 roots
        if not wl.get("directed"):
            try:
                hinfo = bfs.bfs_graph_half(g, host_copy=False)
                hrt = timed_roots(lambda s: bfs.bfs_run_half(g, s, parent, level, stream), large_roots[:2], 1, 1,
                                  stream)
                comp["half_storage_bfs_2_roots"] = {
                    "gteps": round(harmonic_gteps(e_one[:2], list(hrt.flatten() / 1e3)), 3),
                    "ms_per_root": round(float(hrt.mean()), 3),
                    "adjacency_bytes": 4 * int(hinfo["nnz"]), "full_adjacency_bytes": 4 * int(nnz),
                    "how": "bfs_run_half: per level a pull over the unvisited half rows (largest frontier "
                           "neighbour above) and a push from the frontier's half rows (atomicMax from below)"}
            except bfs.BfsError as e:
                comp["half_storage_bfs_2_roots"] = {"error": str(e)}
        # autotuned: tuning picked on 8 other seeded roots (a grid: on the opposite corner, which
        # its symmetry makes an equivalent root), then all timed roots (a grid's one root: every step)
        tune_roots = inputs.roots(el, 8, wl["root_seed"] + 7777) if wl["kind"] == "rmat" else [n - 1]
        tuned = bfs.bfs_autotune(g, tune_roots)
        at_steps = 1 if wl["kind"] == "rmat" else args.steps
        at = timed_roots(lambda s: bfs.bfs_run(g, s, parent, level), large_roots, at_steps, 1, stream)
        comp["autotuned_gteps"] = round(harmonic_gteps(e_one * at_steps, list(at.flatten() / 1e3)), 3)
        comp["autotuned_ms_per_step"] = round(float(at.sum(axis=1).mean()), 3)
        comp["autotuned"] = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in tuned.as_dict().items()}
        bfs.bfs_set_tuning(g, **{f: 0 for f in ("warp_degree", "cta_degree", "pull_thread_degree",
                                                 "chunk_degree", "batch_topdown_limit", "small_frontier",
                                                 "batch_width", "narrow_edges", "ctas_per_sm")}, alpha=0.0, beta=0.0)
        # the batched configuration's own graph (R-MAT scale 24, graph seed 4 / roots 104): 64 roots in
        # one batched traversal against 64 single-root traversals of the same roots
        if wl["kind"] == "rmat" and wl["scale"] != 24 and not args.no_batched_config:
            comp["batched_rmat24"] = batched_config_comparison(bfs, stream)
        if wl["kind"] == "rmat" and not args.no_batched_config:
            comp["ragged_32_graphs"] = ragged_comparison(bfs, stream)
        result["comparisons"] = comp

    g.destroy()
    del parent, level
    # CPU baseline: the oracle on a bounded sample (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cs = cpu_oracle_sample(el, [roots[i] for i in large], edges[large[0]])
        result["cpu_baseline"] = {"value": round(cs["value"], 5), "unit": "GTEPS", "cores": cs["threads"],
                                  "host_cpus": os.cpu_count(), "kind": "oracle", "sample": cs["sample"]}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------- the reference arm: the CPU oracle ----------------

def run_reference(args, wl):
    """The oracle timed on the host cores on the GPU arm's workload.  One step is
    one serial oracle BFS from a large-component root (the roots taken in turn);
    the W warm-up steps and then the K timed steps run `threads` at a time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    el, roots = make_workload(wl, 0)
    og = oracle.csr_of(el)
    del el
    large, e_comp = oracle_census(og, roots)
    threads = host_threads()
    seq = [large[i % len(large)] for i in range(args.warmup + args.steps)]
    timed_oracle_steps(og, seq[:args.warmup], threads)
    wall = timed_oracle_steps(og, seq[args.warmup:], threads)
    value = e_comp * args.steps / wall / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded generators)",
            "config": bench_config(wl, og.n, og.nnz, len(roots), len(large), e_comp, world),
            "cpu_baseline": {"value": round(value, 5), "unit": "GTEPS", "cores": min(threads, args.steps),
                             "host_cpus": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step: one serial oracle BFS (FIFO queue + max-id parent pass) from "
                                       f"a large-component root, the roots taken in turn; the {args.steps} timed "
                                       f"steps run {threads} at a time on the host threads; oracle CSR build "
                                       f"not timed"},
            "e2e": {"value": round(value, 5), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat26")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched-config", action="store_true")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)  # the timing rules ask for at least three untimed steps
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_gpu(args, wl)


if __name__ == "__main__":
    main()
