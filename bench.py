"""Benchmark of the fixpoint relaxation sweep on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload rmat22|grid4096|er16k]

One step is one pass of the whole hot path over the workload, all resident in
HBM when the timed region starts: build the graph (CSR, COO, symmetrised copy,
degree buckets) from the device-resident edge list, then SSSP and BFS from 8
seeded sources plus CC, each in all four modes (vertex/edge x sync/async),
every result copied out in bulk, then free the graph.  The value is GTEPS
(Graph500 convention: input edges whose source is reached, per query; all
edges for CC) over the whole step.  ``e2e`` is the same step through the same
C ABI with pinned host buffers (graph upload and result downloads inside the
timed region).  Under torchrun, every rank runs an independent replica
(the method shards by independent queries; no data-path collective).

Besides the step, the JSON line carries (kept short, so that a record of the
line's last few KB holds all of it): the roofline of the dominant kernel by
the measurement plan's byte formula, with the all-active sweep roofline test
nested in it (``roofline.sweep``); the multi-source sweep against the
separate queries of the step (``fused``); the batched workload (``batched``);
and the serving comparison on the stated ~64 GB resident set (``serving``:
per rate, [server, one-at-a-time] p50/p99 ms and completed/s).  ``--detail
PATH`` writes everything measured -- per kernel, the pull and bucket modes
(``extra_modes``), the bucketed SSSP on the 4096^2 grid (``grid_bucket``),
every serving row -- to a JSON file.  Each part can be skipped with its
``--no-...`` flag.

``--impl reference`` times the CPU oracle (single thread) on a bounded sample
of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

METRIC = "SSSP/BFS GTEPS & HBM-roofline %; served p50/p99 latency vs one-at-a-time"
MODE_NAMES = {0: "vertex_sync", 1: "vertex_async", 2: "edge_sync", 3: "edge_async", 5: "pull", 6: "bucket"}
ALGO_NAMES = ["sssp", "bfs", "cc"]

# DRAM bytes per launch from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by kernel; valid only while the device source
# is unchanged (sha256 over fg_internal.cuh, fg_device.cuh and fg_fixpoint.cu
# at capture time).
NCU_TRAFFIC: dict = {
    # profiles/sssp_rmat22_traffic.md: one launch each, first seeded source, R-MAT 22 (renumbered)
    "fixpoint_kernel<sssp,vertex_sync>": {"bytes_per_launch": 3255336960 + 123581184, "src_sha": "0c29859e2a74ef96"},
    "fixpoint_kernel<sssp,edge_sync>": {"bytes_per_launch": 4797810944 + 75623168, "src_sha": "0c29859e2a74ef96"},
    "fixpoint_kernel<sssp,vertex_async>": {"bytes_per_launch": 2316889344 + 134529536, "src_sha": "f5263d1212ab3d76"},
    "fixpoint_kernel<sssp,edge_async>": {"bytes_per_launch": 3582338048 + 167827712, "src_sha": "f5263d1212ab3d76"},
}


# DRAM bytes of one all-active sweep launch (R-MAT 22, the sweep roofline
# state), same validity rule
NCU_SWEEP_DRAM: dict = {
    # profiles/sweep_rmat22.md: the sweep roofline state on R-MAT 22 (renumbered), one launch each
    "vertex_sync": {"bytes": 584944128 + 3304960, "src_sha": "0c29859e2a74ef96"},
    "edge_sync": {"bytes": 829428224 + 3476736, "src_sha": "0c29859e2a74ef96"},
}

KERNEL_SOURCES = ("fg_internal.cuh", "fg_device.cuh", "fg_fixpoint.cu")


def fixpoint_source_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1903_01665_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# ---------------------------------------------------------------- workloads
def make_workload(name: str):
    if name == "rmat22":
        g = gg.rmat(22)
        desc = ("rmat-22 (4,194,304 V, 67,108,864 E, a,b,c=.57,.19,.19, w U[1,1000]): SSSP+BFS from 8 "
                "seeded sources + CC, each in 4 modes, graph build included")
    elif name == "grid4096":
        g = gg.grid(4096)
        desc = ("grid-4096 (16,777,216 V, ~65.8M E, 2% deleted, 0.1% shortcuts, w U[1,10000]): SSSP+BFS "
                "from 8 seeded sources + CC, each in 4 modes, graph build included")
    elif name == "er16k":
        g = gg.er()
        desc = "er-16384-131072 (w U[1,100]): SSSP from vertex 0, vertex-sync"
    else:
        raise SystemExit(f"unknown workload {name}")
    srcs = [0] if name == "er16k" else [int(s) for s in gg.sources(g, 8)]
    return g, srcs, desc


def queries_for(workload: str, srcs):
    """(algo, mode, source) triples of one step."""
    if workload == "er16k":
        return [(0, 0, 0)]
    q = []
    for mode in range(4):
        for s in srcs:
            q.append((0, mode, s))
            q.append((1, mode, s))
        q.append((2, mode, 0))
    return q


# ---------------------------------------------------------------- algorithmic bytes
def algorithmic_bytes(algo: int, mode: int, st: dict, info: dict) -> float:
    """Bytes the variant must move for one query, from its device counters.

    S activity words scanned (sync modes: vertex stamps or levels; edge-sync
    and the dense generations of edge-async: the edge sources streamed), Va
    expanded vertices (edge-async: worklist items expanded), Ea relaxed
    edges, U accepted candidates, P worklist appends, n vertices.  Ids,
    values and offsets are 4 bytes; per edge: col (+ w for SSSP) + the
    target's value.
    """
    S, Va, Ea, U, P = (st["scanned"], st["vertices_processed"], st["edges_relaxed"], st["updates"],
                       st["pushes"])
    n = info["n"]
    per_edge = {0: 12, 1: 8, 2: 8}[algo]
    if mode in (0, 2):           # sync: scans + expansion (2 offsets, value, carry) + MIN and stamp
        if algo == 1:
            b = 4 * S + Va * 8 + Ea * per_edge + U * 4
        else:
            b = 4 * S + Va * 16 + Ea * per_edge + U * 12
    else:                        # async: per item (item, offsets, value), per edge, per update, per push
        item = 12 if algo == 1 else 16
        if mode == 3:
            item += 16           # degree prefix: item, offsets, prefix write
        upd = 8 if algo == 1 else 12
        b = Va * item + Ea * per_edge + U * upd + P * 8
        if mode == 3:
            b += 4 * S           # dense generations: the streamed edge sources
    if algo == 2:
        b += st["jump_passes"] * n * 8
    return float(b)


def plan_bytes(algo: int, mode: int, st: dict, info: dict) -> float:
    """Algorithmic bytes of one query by the measurement plan's per-round
    formulas (4-byte offsets o, ids and values), summed over the rounds run:

      vertex-sync (and pull): V*(o + 4 cur + 8 next init/copy) per round + E_a*(4 col + 4 w + 4 next[dst])
                              + 4*U
      edge-sync:              V*8 per round + E_a*(12 src,dst,w + 4 dist[src] + 4 dist[dst]) + 4*U
      async (vertex, edge, bucket): per processed vertex 2o + 4 dist[u] + 4 worklist read, per edge 12
                              (col, w, target), 4 per worklist push, 4 per update
      CC:                     the same on the symmetrised graph, + 8*V per pointer-jumping pass

    with V vertices, R rounds, E_a relaxed edges, U successful updates.
    Weights are counted for SSSP only: BFS and CC read none (4 bytes less
    per edge)."""
    R, Va, Ea, U, P = (st["rounds"], st["vertices_processed"], st["edges_relaxed"], st["updates"],
                       st["pushes"])
    V = info["n"]
    wb = 4 if algo == 0 else 0
    if mode in (0, 5):
        b = 16 * V * R + (8 + wb) * Ea + 4 * U
    elif mode == 2:
        b = 8 * V * R + (16 + wb) * Ea + 4 * U
    else:
        b = 16 * Va + (8 + wb) * Ea + 4 * P + 4 * U
    if algo == 2:
        b += 8 * V * st["jump_passes"]
    return float(b)


def host_info() -> dict:
    """The host the CPU baseline runs on: logical CPUs (nproc) and model name."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return {"host_cores": int(cores or 0), "cpu_model": model or platform.processor() or platform.machine(),
            "arch": platform.machine()}


# ---------------------------------------------------------------- clocks
REASONS = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.idx),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def pump():
            for line in self.proc.stdout:
                self.lines.append(line.strip())
        self.thread = threading.Thread(target=pump, daemon=True)
        self.thread.start()

    def stop(self) -> dict:
        if self.proc is None:
            return {"error": "nvidia-smi unavailable"}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, power, seen = [], [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(REASONS[1:], parts[4:8]):
                if val.lower().startswith("active"):
                    seen.add(name)
        if not sm:
            return {"error": "no clock samples"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(seen)}


# ---------------------------------------------------------------- our arm
class Runner:
    def __init__(self, workload: str, device):
        import torch
        import paper_1903_01665_gb300 as fg
        self.fg, self.torch = fg, torch
        self.workload = workload
        self.g, self.srcs, self.desc = make_workload(workload)
        g = self.g
        self.d_src = torch.from_numpy(g.src).to(device)
        self.d_dst = torch.from_numpy(g.dst).to(device)
        self.d_w = torch.from_numpy(g.w).to(device)
        self.h_src = torch.from_numpy(g.src).pin_memory()
        self.h_dst = torch.from_numpy(g.dst).pin_memory()
        self.h_w = torch.from_numpy(g.w).pin_memory()
        self.queries = queries_for(workload, self.srcs)
        self.outs = [torch.empty(g.n, dtype=torch.int32, device=device) for _ in range(2)]
        self.h_out = torch.empty(g.n, dtype=torch.int32).pin_memory()
        self.deg = np.bincount(g.src, minlength=g.n).astype(np.int64)
        self.teps_edges = self._teps_edges()
        self.info = None

    def _teps_edges(self):
        """Graph500 edge count per query: edges whose source is reached (all edges for CC)."""
        fg, torch, g = self.fg, self.torch, self.g
        st, h = fg.fg_graph_create_coo(g.n, self.d_src, self.d_dst, self.d_w)
        fg.check(st)
        st, info = fg.fg_graph_info(h)
        self.info_base = info.as_dict()
        reach = {}
        for s in set(self.srcs):
            fg.check(fg.fg_bfs(h, s, self.outs[0], fg.FG_EDGE_ASYNC))
            lv = self.outs[0].cpu().numpy()
            reach[s] = int(self.deg[lv != fg.FG_INF].sum())
        fg.check(fg.fg_graph_destroy(h))
        return {(a, s): (reach[s] if a != 2 else g.m) for (a, _m, s) in self.queries}

    def step(self, e2e: bool = False, record=None):
        """One pass of the hot path; returns (units, stats list)."""
        fg, g = self.fg, self.g
        if e2e:
            st, h = fg.fg_graph_create_coo(g.n, self.h_src, self.h_dst, self.h_w)
        else:
            st, h = fg.fg_graph_create_coo(g.n, self.d_src, self.d_dst, self.d_w)
        fg.check(st)
        if self.info is None:
            st2, info = fg.fg_graph_info(h)
            self.info = info.as_dict()
        units = 0
        for i, (algo, mode, s) in enumerate(self.queries):
            out = self.h_out if e2e else self.outs[i & 1]
            st, stats = fg.fg_run(h, algo, s, out, mode)
            fg.check(st)
            units += self.teps_edges[(algo, s)]
            if record is not None:
                record.append((algo, mode, stats.as_dict()))
        fg.check(fg.fg_graph_destroy(h))
        return units


def run_extra_modes(r, per_kernel: dict, modes, reps: int = 2) -> dict:
    """The modes beyond the paper's four (FG_PULL; the bucketed SSSP), on the
    step's workload graph and queries: device time per query against the
    fastest of the four paper modes measured in the timed step."""
    fg, g = r.fg, r.g
    st, h = fg.fg_graph_create_coo(g.n, r.d_src, r.d_dst, r.d_w)
    fg.check(st)
    out = {}
    try:
        for mode in modes:
            name = fg.MODE_NAMES[mode]
            res = {}
            for algo in sorted({a for a, _m, _s in r.queries}):
                srcs = [s_ for a, _m, s_ in r.queries if a == algo and _m == 0]
                ms, pulls = [], []
                for rep in range(reps + 1):
                    for s_ in srcs:
                        st, stats = fg.fg_run(h, algo, s_, r.outs[0], mode)
                        fg.check(st)
                        if rep:
                            ms.append(stats.kernel_ms)
                            pulls.append(stats.pull_rounds)
                best = min((k for k in per_kernel if k[0] == algo), key=lambda k: per_kernel[k]["ms"] / per_kernel[k]["launches"])
                bms = per_kernel[best]["ms"] / per_kernel[best]["launches"]
                res[ALGO_NAMES[algo]] = {"avg_ms": round(float(np.mean(ms)), 4),
                                         "best_paper_mode": MODE_NAMES[best[1]], "best_paper_mode_ms": round(bms, 4),
                                         "speedup": round(bms / float(np.mean(ms)), 3),
                                         "pull_rounds": round(float(np.mean(pulls)), 2)}
            out[name] = res
    finally:
        fg.check(fg.fg_graph_destroy(h))
    return out


def run_fused_compare(r, per_kernel: dict, reps: int = 3) -> dict:
    """The multi-source sweep on the step's workload: the 8 seeded sources of
    SSSP (and of BFS) in one fg_run_multi sweep against the 8 queries of the
    fastest paper mode measured in the timed step (device time), with every
    fused output compared to a plain query's."""
    fg, torch, g = r.fg, r.torch, r.g
    st, h = fg.fg_graph_create_coo(g.n, r.d_src, r.d_dst, r.d_w)
    fg.check(st)
    out = {}
    try:
        srcs = list(r.srcs)
        outs = [torch.empty(g.n, dtype=torch.int32, device=r.d_src.device) for _ in srcs]
        for algo in (0, 1):
            ms = []
            for rep in range(reps + 1):
                st, sts, stats = fg.fg_run_multi(h, algo, srcs, outs)
                fg.check(st)
                if rep:
                    ms.append(stats.kernel_ms)
            exact = True
            for s_, o in zip(srcs, outs):
                fg.check(fg.fg_run(h, algo, s_, r.outs[0], fg.FG_VERTEX_SYNC)[0])
                exact &= bool(torch.equal(o, r.outs[0]))
            cand = [k for k in per_kernel if k[0] == algo]
            if not cand:
                continue
            best = min(cand, key=lambda k: per_kernel[k]["ms"] / per_kernel[k]["launches"])
            sep = per_kernel[best]["ms"] / per_kernel[best]["launches"] * len(srcs)
            fused = float(np.median(ms))
            out[ALGO_NAMES[algo]] = {"fused_ms": round(fused, 3), "separate_ms": round(sep, 3),
                                     "separate_mode": MODE_NAMES[best[1]], "speedup": round(sep / fused, 3),
                                     "rounds": stats.rounds, "bit_exact": exact}
        out["sources"] = len(srcs)
    finally:
        fg.check(fg.fg_graph_destroy(h))
    return out


def run_grid_bucket(device, reps: int = 2) -> dict:
    """The bucketed SSSP (near-far) where it is meant to help: the 4096^2
    road-like grid, SSSP from two seeded sources, against the paper's
    vertex-sync and vertex-async modes (device time, edges relaxed, exact
    agreement of the three results)."""
    import torch
    import paper_1903_01665_gb300 as fg
    g = gg.grid(4096)
    srcs = [int(x) for x in gg.sources(g, 2)]
    st, h = fg.fg_graph_create_coo(g.n, torch.from_numpy(g.src).to(device), torch.from_numpy(g.dst).to(device),
                                   torch.from_numpy(g.w).to(device))
    fg.check(st)
    outs = [torch.empty(g.n, dtype=torch.int32, device=device) for _ in range(3)]
    res = {}
    exact = True
    try:
        for k, (name, mode) in enumerate((("vertex_sync", fg.FG_VERTEX_SYNC), ("vertex_async", fg.FG_VERTEX_ASYNC),
                                          ("bucket", fg.FG_BUCKET))):
            ms, edges, gens = [], [], []
            for s_ in srcs:
                for rep in range(reps + 1):
                    st, stats = fg.fg_run(h, 0, s_, outs[k], mode)
                    fg.check(st)
                    if rep:
                        ms.append(stats.kernel_ms)
                        edges.append(stats.edges_relaxed)
                        gens.append(stats.rounds)
                if mode == fg.FG_BUCKET:
                    fg.check(fg.fg_run(h, 0, s_, outs[0], fg.FG_VERTEX_SYNC)[0])
                    fg.check(fg.fg_run(h, 0, s_, outs[1], fg.FG_VERTEX_ASYNC)[0])
                    exact &= bool(torch.equal(outs[0], outs[2]) and torch.equal(outs[1], outs[2]))
            res[name] = {"avg_ms": round(float(np.mean(ms)), 3), "edges_relaxed": int(np.mean(edges)),
                         "generations": int(np.mean(gens))}
    finally:
        fg.check(fg.fg_graph_destroy(h))
    res["bit_exact"] = exact
    res["workload"] = "grid-4096 (16,777,216 V, ~65.8 M E, w U[1,10000]), SSSP from 2 seeded sources"
    return res


def run_batched(device, reps: int = 3) -> dict:
    """The batched workload: 512 SSSP/BFS queries (8 seeded sources per
    graph, alternating) over 64 resident graphs of uneven size (R-MAT scales
    10-20, grids 256^2-2048^2, weights U[1,1000]), FG_AUTO (the selection
    model's plan per graph), run one query at a time with the plain per-query
    kernels and as one batched CUDA-graph launch, fused and unfused; every
    output compared bit for bit.  Then the model is checked against the
    autotuner: per (graph, algorithm), the device time of the model's plan
    against the fastest (mode, CTAs per SM) fg_autotune measured."""
    import torch
    import paper_1903_01665_gb300 as fg
    graphs = gg.batched_graphs()
    queries = gg.batched_queries(graphs)
    handles, degs = [], []
    try:
        for g in graphs:
            st, h = fg.fg_graph_create_coo(g.n, torch.from_numpy(g.src).to(device),
                                           torch.from_numpy(g.dst).to(device), torch.from_numpy(g.w).to(device))
            fg.check(st)
            handles.append(h)
            degs.append(torch.from_numpy(np.bincount(g.src, minlength=g.n).astype(np.int64)).to(device))
        plans = {}
        for qi, (gi, algo, s) in enumerate(queries):
            if (gi, algo) not in plans:
                st, pl = fg.fg_select_plan(handles[gi], algo)
                fg.check(st)
                plans[(gi, algo)] = (pl.mode, pl.blocks_per_sm, s, qi)
        outs1 = [torch.empty(graphs[gi].n, dtype=torch.int32, device=device) for gi, _, _ in queries]
        outs2 = [torch.empty(graphs[gi].n, dtype=torch.int32, device=device) for gi, _, _ in queries]
        outs3 = [torch.empty(graphs[gi].n, dtype=torch.int32, device=device) for gi, _, _ in queries]
        batch = [(handles[gi], algo, s, outs2[i], fg.FG_AUTO) for i, (gi, algo, s) in enumerate(queries)]
        fused = [(handles[gi], algo, s, outs3[i], fg.FG_AUTO) for i, (gi, algo, s) in enumerate(queries)]
        t_one, t_batch, t_fused = [], [], []
        for _ in range(reps + 1):          # the first repetition is a warm-up
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            for i, (gi, algo, s) in enumerate(queries):
                st, _ = fg.fg_run(handles[gi], algo, s, outs1[i], fg.FG_AUTO)
                fg.check(st)
            torch.cuda.synchronize(device)
            t_one.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            st, sts, _, bst = fg.fg_run_batch(batch, use_cuda_graph=True)
            fg.check(st)
            torch.cuda.synchronize(device)
            t_batch.append(time.perf_counter() - t0)
            t0 = time.perf_counter()
            st, sts, _, fbst = fg.fg_run_batch(fused, use_cuda_graph=True, fuse_same_graph=True)
            fg.check(st)
            torch.cuda.synchronize(device)
            t_fused.append(time.perf_counter() - t0)
        exact = all(torch.equal(a, b) for a, b in zip(outs1, outs2))
        exact_fused = all(torch.equal(a, b) for a, b in zip(outs1, outs3))
        edges = 0
        for i, (gi, algo, s) in enumerate(queries):
            edges += int(degs[gi][outs1[i] != fg.FG_INF].sum().item())
        one = statistics.median(t_one[1:])
        bat = statistics.median(t_batch[1:])
        fus = statistics.median(t_fused[1:])
        modes = {}
        for (gi, algo), (m, bps, _s, _q) in plans.items():
            key = f"{ALGO_NAMES[algo]}/{MODE_NAMES[m]}" + ("/2cta" if bps else "")
            modes[key] = modes.get(key, 0) + 1
        # the model against the autotuner's measurement (median of 3 each)
        ratios = []
        for (gi, algo), (m, bps, s, qi) in plans.items():
            ts = []
            for _ in range(3):
                st, stt = fg.fg_run(handles[gi], algo, s, outs1[qi], m, blocks_per_sm=bps)
                fg.check(st)
                ts.append(stt.kernel_ms)
            st, best, times = fg.fg_autotune(handles[gi], algo, s)
            fg.check(st)
            ratios.append(statistics.median(ts) / min(t for t in times if t > 0))
        model_check = {"pairs": len(ratios), "within_10pct": int(sum(r <= 1.1 for r in ratios)),
                       "worst_ratio": round(max(ratios), 3), "median_ratio": round(statistics.median(ratios), 3)}
        return {"queries": len(queries), "graphs": len(graphs),
                "one_at_a_time_qps": round(len(queries) / one, 1), "batched_qps": round(len(queries) / fus, 1),
                "speedup": round(one / fus, 3), "bit_exact": exact and exact_fused,
                "unfused_qps": round(len(queries) / bat, 1), "unfused_speedup": round(one / bat, 3),
                "one_at_a_time_gteps": round(edges / one / 1e9, 3), "batched_gteps": round(edges / fus / 1e9, 3),
                "batch_kernel_ms": round(fbst.kernel_ms, 3), "launches": fbst.launches, "teams": fbst.teams,
                "ctas": fbst.ctas, "unfused_launches": bst.launches, "model_modes": modes,
                "model_check": model_check,
                "fusion": "queries on one graph share work: SSSP/BFS as multi-source sweeps of up to 8 "
                          "sources, CC once (fuse_same_graph); unfused = one fixpoint per query",
                "timing": "wall clock around each run, median of %d, after one warm-up" % reps}
    finally:
        for h in handles:
            fg.fg_graph_destroy(h)


def run_serving(device, full: bool = False, rates=(100, 300, 1000, 3000, 10000), n_req: int = 2000,
                seed: int = 0x5E57) -> dict:
    """Poisson arrivals of SSSP/BFS/CC requests (40/40/20, uniform over the
    resident graphs, seeded sources) served (a) by the continuous-batching
    server and (b) one request at a time with the plain kernels; p50/p99
    latency (submission to completion) and completed requests per second."""
    import torch
    import paper_1903_01665_gb300 as fg
    if full:
        graphs = [gg.rmat(24), gg.rmat(25), gg.rmat(26), gg.grid(8192, whi=1000)]
    else:
        graphs = [gg.rmat(20), gg.rmat(21), gg.rmat(22), gg.grid(2048, whi=1000)]
    handles = []
    try:
        device_bytes = 0
        for g in graphs:
            st, h = fg.fg_graph_create_coo(g.n, torch.from_numpy(g.src).to(device),
                                           torch.from_numpy(g.dst).to(device), torch.from_numpy(g.w).to(device))
            fg.check(st)
            handles.append(h)
            device_bytes += fg.fg_graph_info(h)[1].device_bytes
        srcs = [gg.sources(g, 64, seed=seed + i) for i, g in enumerate(graphs)]
        for h in handles:   # the selection model's plans (and their depth estimates) before the clock starts
            for algo in (0, 1, 2):
                fg.check(fg.fg_select_plan(h, algo)[0])
        # output buffers: one per request (recycled round-robin on the large set,
        # 32 per graph: 24 GB in all)
        ring = 32 if full else n_req
        outs = [[torch.empty(g.n, dtype=torch.int32, device=device) for _ in range(min(ring, n_req))]
                for g in graphs]
        result = {"resident_graphs": [f"{g.name} ({g.n} V, {g.m} E)" for g in graphs],
                  "resident_device_gb": round(device_bytes / 1e9, 2), "requests_per_rate": n_req,
                  "mix": "40% SSSP / 40% BFS / 20% CC, uniform over graphs, FG_AUTO (the selection model's plan)",
                  "rates": []}
        for rate in rates:
            rng = np.random.Generator(np.random.PCG64(seed + int(rate)))
            gaps = rng.exponential(1.0 / rate, n_req)
            arrive = np.cumsum(gaps) - gaps[0]
            gis = rng.integers(0, len(graphs), n_req)
            u = rng.random(n_req)
            algos = np.where(u < 0.4, 0, np.where(u < 0.8, 1, 2))
            pick = rng.integers(0, 64, n_req)
            row = {"rate_per_s": rate}
            for kind in ("batched", "one_at_a_time"):
                if kind == "batched":
                    st, srv = fg.fg_server_create(hbm_budget_bytes=16 << 30, max_inflight=2, max_wave=64)
                else:
                    st, srv = fg.fg_server_create(one_at_a_time=True)
                fg.check(st)
                counters = [0] * len(graphs)
                torch.cuda.synchronize(device)
                t0 = time.perf_counter()
                for i in range(n_req):
                    while time.perf_counter() - t0 < arrive[i]:
                        pass
                    gi = int(gis[i])
                    out = outs[gi][counters[gi] % len(outs[gi])]
                    counters[gi] += 1
                    st, _ = fg.fg_server_submit(srv, handles[gi], int(algos[i]), int(srcs[gi][pick[i]]), out,
                                                fg.FG_AUTO)
                    fg.check(st)
                fg.check(fg.fg_server_drain(srv, 0))
                span = time.perf_counter() - t0
                comps = fg.fg_server_poll(srv, cap=n_req + 16)
                fg.check(fg.fg_server_destroy(srv))
                lat = np.array([c[3] for c in comps])
                ok = all(c[1] == fg.FG_OK for c in comps)
                row[kind] = {"p50_ms": round(float(np.percentile(lat, 50)), 3),
                             "p99_ms": round(float(np.percentile(lat, 99)), 3),
                             "mean_ms": round(float(lat.mean()), 3),
                             "completed_per_s": round(len(comps) / span, 1), "all_ok": ok,
                             "mean_wave": round(float(np.mean([c[2] for c in comps])), 2)}
            result["rates"].append(row)
        return result
    finally:
        for h in handles:
            fg.fg_graph_destroy(h)


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(units_local: int, seconds_local: float, pg=None, device=None):
    """Whole-job throughput of independent replicas: total units over all ranks
    divided by the slowest rank's time (max over ranks).  Returns (units, seconds)."""
    if pg is None:
        return units_local, seconds_local
    import torch
    t = torch.tensor([seconds_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    pg.all_reduce(u, op=pg.ReduceOp.SUM)
    return int(u.item()), float(t.item())


def run_sweep_roofline(r, peak_gbps: float, reps: int = 10, warm: int = 3) -> dict:
    """The headline roofline test: one all-active relaxation round (fg_sweep)
    over the workload graph, vertex variant (Alg. 1) and edge variant
    (Alg. 2), from a fixed mid-run state: three synchronous rounds from the
    first seeded source, then every vertex still unreached set to 2^30 so that
    every vertex and edge is active.  Device time of each launch by CUDA
    events inside the library; median of `reps` after `warm` warm-ups, next
    reset to cur before every launch (outside the timed kernel).
    Algorithmic bytes per round (4-byte offsets and values):
      vertex: V*(4 row_off + 4 cur + 8 next init/copy) + E*(4 dst + 4 w + 4 next[dst]) + 4*lowered
      edge:   V*8 + E*(12 src,dst,w + 4 cur[src] + 4 next[dst]) + 4*lowered"""
    fg, torch, g = r.fg, r.torch, r.g
    st, h = fg.fg_graph_create_coo(g.n, r.d_src, r.d_dst, r.d_w)
    fg.check(st)
    try:
        inf = fg.FG_INF
        cur = torch.full((g.n,), inf, dtype=torch.int32, device=r.d_src.device)
        cur[int(r.srcs[0])] = 0
        for _ in range(3):
            nxt = cur.clone()
            fg.check(fg.fg_sweep(h, fg.FG_VERTEX_SYNC, cur, nxt)[0])
            cur = nxt
        reached_after_3 = int((cur != inf).sum().item())
        cur[cur == inf] = 1 << 30
        nxt = torch.empty_like(cur)
        out = {"state": "3 rounds from the first seeded source, unreached vertices set to 2^30 "
                        "(every vertex and edge active)",
               "reached_after_3_rounds": reached_after_3, "timing": f"median of {reps} launches"}
        for mode, name in ((fg.FG_VERTEX_SYNC, "vertex_sync"), (fg.FG_EDGE_SYNC, "edge_sync")):
            times = []
            for i in range(warm + reps):
                nxt.copy_(cur)
                st, upd, ms = fg.fg_sweep(h, mode, cur, nxt)
                fg.check(st)
                if i >= warm:
                    times.append(ms)
            lowered = int((nxt < cur).sum().item())
            v, e = g.n, g.m
            nbytes = (16 * v + 12 * e if mode == fg.FG_VERTEX_SYNC else 8 * v + 20 * e) + 4 * lowered
            med = float(np.median(times))
            gbps = nbytes / (med * 1e-3) / 1e9
            out[name] = {"us": round(med * 1e3, 1), "algorithmic_bytes": nbytes, "gbps": round(gbps, 1),
                         "frac": round(gbps / peak_gbps, 4), "lowered": lowered, "writes": int(upd)}
        return out
    finally:
        fg.check(fg.fg_graph_destroy(h))


def run_ours(args):
    import torch
    import paper_1903_01665_gb300 as fg
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
        pg = dist
    fg.load(build_if_missing=False)
    r = Runner(args.workload, device)
    stream = torch.cuda.current_stream(device)

    def barrier():
        torch.cuda.synchronize(device)
        if pg:
            pg.barrier()
        torch.cuda.synchronize(device)

    for _ in range(args.warmup):
        r.step()
    # ---- timed region: device-resident inputs
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_idx = vis.split(",")[local] if vis and not vis.startswith("GPU-") else str(local)
    clocks = ClockSampler(int(smi_idx) if smi_idx.isdigit() else local)
    clocks.start()
    record = []
    barrier()
    l0 = fg.fg_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    units = 0
    for _ in range(args.steps):
        units += r.step(record=record)
    ev1.record(stream)
    barrier()
    launches = fg.fg_kernel_launches() - l0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    units_all, sec = aggregate(units, ms * 1e-3, pg, device)
    ms = sec * 1e3
    value = units_all / sec / 1e9
    # raw relaxations per second: edges whose source was active, every query
    relax_all, _ = aggregate(sum(int(st["edges_relaxed"]) for _a, _m, st in record), sec, pg, device)

    # ---- roofline of the dominant kernel (largest share of device time)
    per_kernel = {}
    for algo, mode, st in record:
        k = (algo, mode)
        d = per_kernel.setdefault(k, {"ms": 0.0, "bytes": 0.0, "model_bytes": 0.0, "launches": 0})
        d["ms"] += st["kernel_ms"]
        d["bytes"] += plan_bytes(algo, mode, st, r.info)
        d["model_bytes"] += algorithmic_bytes(algo, mode, st, r.info)
        d["launches"] += 1
    total_kernel_ms = sum(d["ms"] for d in per_kernel.values())
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    dk = per_kernel[dom]
    peaks = load_peaks()
    launch_s = dk["ms"] / dk["launches"] * 1e-3
    achieved = (dk["bytes"] / dk["launches"]) / launch_s / 1e9
    achieved_model = (dk["model_bytes"] / dk["launches"]) / launch_s / 1e9
    kname = f"fixpoint_kernel<{ALGO_NAMES[dom[0]]},{MODE_NAMES[dom[1]]}>"
    traffic = None
    rec = NCU_TRAFFIC.get(kname)
    if rec and rec.get("src_sha") == fixpoint_source_sha():
        traffic = rec["bytes_per_launch"]
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peaks[0],
                "unit": "GB/s", "frac": round(achieved / peaks[0], 4), "peak_source": peaks[1],
                "bytes": "measurement-plan formula, per launch", "traffic": traffic,
                "algorithmic_bytes_per_launch": round(dk["bytes"] / dk["launches"]),
                "frac_model": round(achieved_model / peaks[0], 4),
                "dram_frac": None if traffic is None else round(traffic / launch_s / 1e9 / peaks[0], 4),
                "avg_launch_ms": round(dk["ms"] / dk["launches"], 4),
                "share_of_kernel_time": round(dk["ms"] / total_kernel_ms, 4)}
    per_mode = {}
    for (algo, mode), d in sorted(per_kernel.items()):
        per_mode[f"{ALGO_NAMES[algo]}/{MODE_NAMES[mode]}"] = {
            "avg_ms": round(d["ms"] / d["launches"], 4),
            "gbps": round(d["bytes"] / (d["ms"] * 1e-3) / 1e9, 1),
            "gbps_model": round(d["model_bytes"] / (d["ms"] * 1e-3) / 1e9, 1)}

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        # one untimed step first (first use of the host-input path), then as
        # many timed steps as the device-resident leg, by the host clock
        k2 = max(1, args.steps)
        r.step(e2e=True)
        barrier()
        t0 = time.perf_counter()
        u2 = 0
        for _ in range(k2):
            u2 += r.step(e2e=True)
        barrier()
        dt = time.perf_counter() - t0
        u2, dt = aggregate(u2, dt, pg, device)
        e2e = {"value": round(u2 / dt / 1e9, 4), "unit": "GTEPS",
               "h2d_bytes_per_step": 3 * 4 * r.g.m,
               "d2h_bytes_per_step": 4 * r.g.n * len(r.queries), "steps": k2, "warmup": 1}

    sweep = None if args.no_sweep else run_sweep_roofline(r, peaks[0])
    fused = None if args.no_fused or len(r.srcs) < 2 else run_fused_compare(r, per_kernel)
    extra = None if args.no_extra else run_extra_modes(r, per_kernel, [fg.FG_PULL, fg.FG_BUCKET])

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(r.g, r.srcs, r.deg, args.workload)
    desc, nqueries = r.desc, len(r.queries)
    gbytes = int(r.info["device_bytes"]) if r.info else 0
    l2_note = (f"inputs larger than L2 (graph {gbytes / 1e9:.2f} GB built per step)" if gbytes > 129 << 20 else
               f"inputs smaller than L2 ({gbytes / 1e6:.1f} MB graph), not flushed: a parity-size case")
    batched = serving = None
    del r
    torch.cuda.empty_cache()
    grid_bucket = None if args.no_grid_bucket else run_grid_bucket(device)
    if not args.no_batched:
        batched = run_batched(device)
    if not args.no_serving:
        rates = tuple(int(x) for x in args.serving_rates.split(","))
        n_req = args.serving_requests
        if args.serving_full:   # the full sweep: five rates, 2000 requests each
            rates, n_req = (100, 300, 1000, 3000, 10000), max(n_req, 2000)
        serving = run_serving(device, full=args.serving_set == "stated" or args.serving_full, rates=rates,
                              n_req=n_req)

    if rank == 0:
        if sweep is not None:
            # the headline all-active round, in the roofline object the record keeps whole
            roofline["sweep"] = {k: {"us": v["us"], "gbps": v["gbps"], "frac": v["frac"]}
                                 for k, v in sweep.items() if isinstance(v, dict)}
            sweep_dram = {k: v for k, v in NCU_SWEEP_DRAM.items()
                          if v.get("src_sha") == fixpoint_source_sha()}
            for k, v in sweep_dram.items():
                if k in roofline["sweep"]:
                    us = roofline["sweep"][k]["us"]
                    roofline["sweep"][k]["dram_frac"] = round(v["bytes"] / (us * 1e-6) / 1e9 / peaks[0], 4)
        line = {"metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic (seeded generators in graphgen/)",
                "config": {"workload": desc, "queries_per_step": nqueries,
                           "teps_edges_per_step": units // max(args.steps, 1),
                           "l2": l2_note,
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk,
                "relaxations_gps": round(relax_all / sec / 1e9, 3)}
        if fused is not None:
            line["fused"] = {k: ({kk: v[kk] for kk in ("fused_ms", "separate_ms", "speedup", "bit_exact")}
                                 if isinstance(v, dict) else v) for k, v in fused.items()}
        if batched is not None:
            line["batched"] = {k: batched[k] for k in ("batched_qps", "one_at_a_time_qps", "speedup", "bit_exact",
                                                       "launches", "unfused_speedup", "model_check") if k in batched}
        if serving is not None:
            line["serving"] = compact_serving(serving)
        detail = {"per_kernel": per_mode, "sweep_roofline": sweep, "fused": fused, "extra_modes": extra,
                  "grid_bucket": grid_bucket,
                  "batched": batched, "serving": serving,
                  "relaxations_per_step": relax_all // max(args.steps * ws, 1)}
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump({"line": line, "detail": detail}, f, indent=1)
        print(json.dumps(line, separators=(",", ":")), flush=True)
    if pg:
        pg.destroy_process_group()


def compact_serving(serving: dict) -> dict:
    """Per arrival rate: p50/p99 latency (ms) and completed requests/s of the
    server (continuous batching) and of the one-at-a-time baseline."""
    out = {"graphs": len(serving.get("resident_graphs", [])), "device_gb": serving.get("resident_device_gb"),
           "requests": serving.get("requests_per_rate"), "rates": {}}
    for row in serving.get("rates", []):
        b, o = row["batched"], row["one_at_a_time"]
        out["rates"][str(row["rate_per_s"])] = {
            "p50": [round(b["p50_ms"], 1), round(o["p50_ms"], 1)],
            "p99": [round(b["p99_ms"], 1), round(o["p99_ms"], 1)],
            "qps": [b["completed_per_s"], o["completed_per_s"]],
            "ok": bool(b["all_ok"] and o["all_ok"])}
    out["order"] = "[server, one-at-a-time]"
    return out


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- oracle timing
def cpu_baseline_sample(g, srcs, deg, workload):
    """The oracle, untuned, single thread: SSSP + BFS from one source and CC."""
    import oracle
    s = srcs[0]
    t0 = time.perf_counter()
    rc1, d = oracle.sssp(g.n, g.src, g.dst, g.w, s)
    rc2, lv = oracle.bfs(g.n, g.src, g.dst, s)
    units = 2 * int(deg[lv != oracle.UNREACHED].sum())
    if workload != "er16k":
        oracle.cc(g.n, g.src, g.dst)
        units += g.m
    dt = time.perf_counter() - t0
    out = {"value": round(units / dt / 1e9, 5), "unit": "GTEPS", "cores": 1, "kind": "oracle",
           "sample": f"1 SSSP + 1 BFS from source {s}" + (" + 1 CC" if workload != "er16k" else "")
                     + f" on {workload}, sequential C, {dt:.1f} s"}
    out.update(host_info())
    out["omp"] = omp_baseline_sample(g, srcs, deg, workload)
    return out


def omp_baseline_sample(g, srcs, deg, workload):
    """The multi-core CPU baseline (OpenMP frontier SSSP/BFS, union-find CC,
    all host cores), context only: one adjacency build, then SSSP and BFS
    from each seeded source and one CC, like the GPU step's build and
    queries.  Its results are checked against the oracle by the CPU tests."""
    from oracle import omp
    if omp.build() is None:
        return {"unavailable": "no OpenMP in the host compiler"}
    t0 = time.perf_counter()
    units = 0
    with omp.Graph(g.n, g.src, g.dst, g.w) as h:
        if h.status != omp.OK:
            return {"unavailable": f"build status {h.status}"}
        for s in srcs:
            rc1, _ = h.sssp(int(s))
            rc2, lv = h.bfs(int(s))
            if rc1 != omp.OK or rc2 != omp.OK:
                return {"unavailable": f"query status {rc1}/{rc2}"}
            units += 2 * int(deg[lv != np.iinfo(np.int32).max].sum())
    n_cc = 0
    if workload != "er16k":
        omp.cc(g.n, g.src, g.dst)
        units += g.m
        n_cc = 1
    dt = time.perf_counter() - t0
    return {"value": round(units / dt / 1e9, 5), "cores": omp.threads(),
            "sample": f"1 build + {len(srcs)} SSSP + {len(srcs)} BFS + {n_cc} CC, {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import oracle
    g, srcs, desc = make_workload(args.workload)
    deg = np.bincount(g.src, minlength=g.n).astype(np.int64)
    oracle.build()

    def one(i):
        s = srcs[i % len(srcs)]
        _, lv = oracle.bfs(g.n, g.src, g.dst, s)
        oracle.sssp(g.n, g.src, g.dst, g.w, s)
        units = 2 * int(deg[lv != oracle.UNREACHED].sum())
        if args.workload != "er16k":
            oracle.cc(g.n, g.src, g.dst)
            units += g.m
        return units

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    units = 0
    for i in range(args.steps):
        units += one(args.warmup + i)
    dt = time.perf_counter() - t0
    value = units / dt / 1e9
    sample = (f"each step: 1 SSSP + 1 BFS from one of the 8 sources" +
              (" + 1 CC" if args.workload != "er16k" else "") + f" on {args.workload}, sequential C oracle")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "GTEPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (seeded generators in graphgen/)", "config": {"workload": desc},
            "cpu_baseline": {"value": round(value, 5), "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": sample, **host_info()},
            "e2e": {"value": round(value, 5), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_case(args):
    """Profiling driver: one query type on one seeded graph, run twice (the
    second run is the one to capture), stats printed; no benchmark line."""
    import torch
    import paper_1903_01665_gb300 as fg
    algo_name, mode_name = args.case.split(":")
    mode = {v: k for k, v in MODE_NAMES.items()}.get(mode_name, -1)
    if args.case_graph == "rmat":
        g = gg.rmat(args.case_scale)
    else:
        g = gg.grid(args.case_scale)
    s = int(gg.sources(g, 1)[0])
    st, h = fg.fg_graph_create_coo(g.n, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(),
                                   torch.from_numpy(g.w).cuda())
    fg.check(st)
    if algo_name == "sweep":
        # the all-active round of the sweep roofline test, from its state
        cur = torch.full((g.n,), fg.FG_INF, dtype=torch.int32, device="cuda")
        cur[s] = 0
        for _ in range(3):
            nxt = cur.clone()
            fg.check(fg.fg_sweep(h, fg.FG_VERTEX_SYNC, cur, nxt)[0])
            cur = nxt
        cur[cur == fg.FG_INF] = 1 << 30
        nxt = torch.empty_like(cur)
        for i in range(2):
            nxt.copy_(cur)
            st, upd, ms = fg.fg_sweep(h, mode, cur, nxt)
            fg.check(st)
            print(i, json.dumps({"writes": upd, "kernel_ms": ms}), flush=True)
        fg.check(fg.fg_graph_destroy(h))
        return
    if mode_name == "multi":
        # the multi-source sweep of the 8 seeded sources
        algo = ALGO_NAMES.index(algo_name)
        srcs = [int(x) for x in gg.sources(g, 8)]
        outs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in srcs]
        for i in range(2):
            st, sts, stats = fg.fg_run_multi(h, algo, srcs, outs)
            fg.check(st)
            print(i, json.dumps(stats.as_dict()), flush=True)
        fg.check(fg.fg_graph_destroy(h))
        return
    algo = ALGO_NAMES.index(algo_name)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for i in range(2):
        st, stats = fg.fg_run(h, algo, s, out, mode)
        fg.check(st)
        print(i, json.dumps(stats.as_dict()), flush=True)
    fg.check(fg.fg_graph_destroy(h))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default=None,
                    help="profiling driver, e.g. sssp:edge_sync, sweep:edge_sync or sssp:multi (8-source sweep)")
    ap.add_argument("--case-graph", default="rmat", choices=["rmat", "grid"])
    ap.add_argument("--case-scale", type=int, default=20, help="R-MAT scale or grid side")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22", choices=["rmat22", "grid4096", "er16k"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the all-active sweep roofline test")
    ap.add_argument("--no-extra", action="store_true", help="skip the pull/bucket comparison on the workload")
    ap.add_argument("--no-fused", action="store_true", help="skip the multi-source sweep comparison")
    ap.add_argument("--no-grid-bucket", action="store_true", help="skip the bucketed-SSSP grid comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-workload comparison")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving comparison")
    ap.add_argument("--serving-set", default="stated", choices=["stated", "reduced"],
                    help="resident set served: R-MAT 24-26 + 8192^2 grid (~64 GB, the stated serving "
                         "configuration) or R-MAT 20-22 + 2048^2 grid (~4 GB)")
    ap.add_argument("--serving-rates", default="100,1000,10000", help="Poisson arrival rates, requests/s")
    ap.add_argument("--serving-requests", type=int, default=1000, help="requests per rate")
    ap.add_argument("--serving-full", action="store_true",
                    help="the stated set at rates 100,300,1000,3000,10000 with at least 2000 requests each")
    ap.add_argument("--detail", default=None, help="also write every measurement (per kernel, extra modes, "
                                                   "serving rows) as JSON to this path")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
