#!/usr/bin/env python3
"""Benchmark: D-iteration edge pushes/s to L1 residual 1e-8 on one GB300, vs the same GPU's power iteration.

Workload (default): the Zipf graph at scale -- N = 2^24 nodes, exactly 12% dangling,
other out-degrees Zipf(2.1) clipped to [1, 50000], targets drawn proportional to
rank^-0.9 over permuted ids, int32 CSR, d = 0.85, V = 1/N, FP64, stop when the
Theorem 2 bound |F|_1/(1-d) <= 1e-8.  Synthetic and seeded (graphgen, seed 1).

One step = one full solve on the device-resident graph: initialization, threshold
sweeps (scan/exchange, push, finalize) in one CUDA-graph while-loop, the exact
|F|_1 confirmation and the copy of H to a device buffer.  value = edges pushed
by all ranks / max over ranks of the device time of K steps.

Besides the headline the JSON line reports: the power iteration (MAT-ITER, pull
SpMV) to the paper's stop rule at the same tolerance on the same GPU; the
per-kernel roofline of a profiled solve (same kernels, launched one by one with
CUDA events around each); an end-to-end number through the C ABI with pinned
host buffers (create from host CSR + solve + H to host, every step); SM clocks
sampled during the timed region; and the oracle (sequential FP64 CPU snapshot
sweeps) timed on a bounded sample on the host cores.

--impl reference times the oracle alone, as it stands, on the host cores.
Multi-GPU: replicas only (each rank solves its own copy; no collective on the
data path), launched with torchrun; rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge pushes/s to L1 resid 1e-8 vs GPU power iter; PPR queries/s, p50/p99 ms"
UNIT = "edge pushes/s"
WORKLOADS = {
    "zipf24": dict(kind="zipf", n=1 << 24, alpha=2.1, kmax=50000, dangling=0.12, target_exp=0.9, d=0.85, tol=1e-8,
                   label="Zipf N=2^24, outdeg Zipf(2.1) clipped [1,50000] + 12% dangling, targets ~ rank^-0.9, "
                         "d=0.85, V=1/N, FP64, L1 bound 1e-8"),
    "zipf20": dict(kind="zipf", n=1 << 20, alpha=2.1, kmax=50000, dangling=0.12, target_exp=0.9, d=0.85, tol=1e-8,
                   label="Zipf N=2^20 (reduced size for quick runs), d=0.85, V=1/N, FP64, L1 bound 1e-8"),
    "uniform1e4": dict(kind="uniform", n=10000, dmax=20, d=0.85, tol=1e-10 / 0.15,
                       label="uniform outdeg U{0..20}, N=10^4, d=0.85, V=1/N, FP64, |F|_1 < 1e-10"),
    "rmat23": dict(kind="rmat", scale=23, d=0.85, tol=1e-7,
                   label="R-MAT scale 23, edge factor 16, (a,b,c)=(.57,.19,.19), duplicates removed, d=0.85, V=1/N, "
                         "FP64, L1 bound 1e-7 (the precision workload's graph)"),
    "rmat22": dict(kind="rmat", scale=22, d=0.85, tol=1e-8,
                   label="R-MAT scale 22, edge factor 16, (a,b,c)=(.57,.19,.19), duplicates removed, d=0.85, V=1/N, "
                         "FP64, L1 bound 1e-8 (profiling case for dense sweeps)"),
}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def make_graph(w, seed=1):
    import graphgen as gg
    if w["kind"] == "zipf":
        return gg.zipf_graph(w["n"], alpha=w["alpha"], kmax=w["kmax"], dangling_frac=w["dangling"],
                             target_exp=w["target_exp"], seed=seed)
    if w["kind"] == "rmat":
        return gg.rmat_graph(w["scale"], 16, seed=seed)
    return gg.uniform_graph(w["n"], w["dmax"], seed=seed)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"diter_clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["no samples"]}
        loaded = sorted(sm)[len(sm) // 2:] if len(sm) > 2 else sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def push_sources_digest():
    """sha256 over the sources the push kernel is compiled from (push.cu and its headers)."""
    import hashlib
    h = hashlib.sha256()
    for name in ("push.cu", "device_common.cuh", "internal.h", "dbg.cuh"):
        with open(os.path.join(ROOT, "paper_1202_6158_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def push_traffic():
    """DRAM bytes per push launch from the committed ncu summary of the push kernel on this
    workload (under profiles/), if the push sources are unchanged since it was taken.

    The summary records the digest of the push kernel's sources it was taken with; a
    different digest means the kernel changed and the counters no longer apply.
    """
    summ = os.path.join(ROOT, "profiles", "push_sweep_zipf24.md")
    if not os.path.exists(summ):
        return None
    vals = {}
    for line in open(summ):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("push sources sha256") != push_sources_digest():
        return None
    try:
        return float(vals["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_ranks(dist, dev, sums, maxes):
    """Whole-job figures of a replicas run: the work of all ranks adds up (sums) and the time
    is the slowest rank's (maxes).  dist is torch.distributed with a process group, or None for
    one process; dev is the device the reduction tensors live on (cuda for NCCL, cpu for gloo)."""
    if dist is None:
        return [float(x) for x in sums], [float(x) for x in maxes]
    import torch
    t = torch.tensor([float(x) for x in sums], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    m = torch.tensor([float(x) for x in maxes], dtype=torch.float64, device=dev)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()], [float(x) for x in m.tolist()]


def cpu_baseline(g, w, max_pushes, cores=1):
    """The oracle (sequential FP64 snapshot sweeps, as it stands) on a bounded sample of the same solve."""
    import graphgen as gg
    import oracle
    V = gg.uniform_v(g.n)
    t0 = time.perf_counter()
    r = oracle.diter(g.n, g.row_ptr, g.col_idx, w["d"], V, w["tol"], mode="sweep", beta=0.5, max_pushes=max_pushes)
    dt = time.perf_counter() - t0
    return {"value": r.edges / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "_H": r.H,
            "sample": f"oracle snapshot sweeps (beta=0.5) from F_0 on the same graph, cut at {max_pushes} diffusions: "
                      f"{r.sweeps} sweeps, {r.edges} edge pushes in {dt:.1f} s on 1 host core "
                      f"({'converged' if r.converged else 'not converged'})",
            "seconds": dt, "edges": int(r.edges), "sweeps": int(r.sweeps), "converged": bool(r.converged)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_power_baselines(g, w, sample_products=6):
    """MAT-ITER on the host: the oracle's power iteration on one core over a bounded sample of
    products (the rate per product is the same at every product), and the OpenMP pull version
    on all host cores to the paper's stop rule at the workload's tolerance."""
    import graphgen as gg
    import oracle
    V = gg.uniform_v(g.n)
    out = {}
    t0 = time.perf_counter()
    _, it, _, _ = oracle.power(g.n, g.row_ptr, g.col_idx, w["d"], V, w["tol"], max_iter=sample_products)
    dt = time.perf_counter() - t0
    out["power_cpu"] = {"value": it * g.nnz / dt, "unit": UNIT, "cores": 1, "kind": "oracle MAT-ITER",
                        "ms_per_product": 1e3 * dt / it,
                        "sample": f"the oracle's power iteration from X_0 = 0, cut at {it} products, {dt:.1f} s"}
    try:
        in_ptr, in_src = oracle.transpose(g.n, g.row_ptr, g.col_idx)
        deg = oracle.outdeg(g.n, g.row_ptr)
        t0 = time.perf_counter()
        _, it, _, ok, used = oracle.power_omp(g.n, in_ptr, in_src, deg, w["d"], V, w["tol"], threads=0)
        dt = time.perf_counter() - t0
        out["power_cpu_omp"] = {"value": it * g.nnz / dt, "unit": UNIT, "cores": used, "kind": "OpenMP MAT-ITER",
                                "time_to_residual_ms": 1e3 * dt, "products": it, "converged": bool(ok),
                                "sample": f"the full power iteration to the stop rule at tol {w['tol']:g} on "
                                          f"{used} threads (in-link lists built beforehand, not timed)"}
    except (OSError, subprocess.SubprocessError) as e:
        out["power_cpu_omp"] = {"unavailable": f"OpenMP build failed: {e}"}
    return out


def _oracle_rmat_worker(scale, d, tol, path):
    """Spawned process: the oracle's snapshot-sweep solve of R-MAT `scale` (edge factor 16,
    seed 1, V = 1/N) to bound `tol`; H goes to `path` (.npy)."""
    import graphgen as gg
    import oracle
    g = gg.rmat_graph(scale, 16, seed=1)
    t0 = time.perf_counter()
    r = oracle.diter(g.n, g.row_ptr, g.col_idx, d, gg.uniform_v(g.n), tol, mode="sweep", beta=0.5)
    np.save(path, r.H)
    with open(path + ".json", "w") as f:
        json.dump({"seconds": time.perf_counter() - t0, "sweeps": int(r.sweeps), "edges": int(r.edges),
                   "bound": r.l1F / (1 - d), "converged": bool(r.converged)}, f)


class OracleInBackground:
    """The oracle's config-3 solve (R-MAT scale 23, d = 0.85, bound 1e-7) in a spawned process,
    started before the first GPU call and joined before the timed CPU baselines run."""

    def __init__(self, scale=23, d=0.85, tol=1e-7):
        import multiprocessing as mp
        self.path = os.path.join(tempfile.gettempdir(), f"diter_oracle_rmat{scale}_{os.getpid()}.npy")
        self.proc = mp.get_context("spawn").Process(target=_oracle_rmat_worker, args=(scale, d, tol, self.path))
        self.proc.start()

    def result(self, timeout=900):
        """(H, info) once the solve has finished, or (None, reason)."""
        self.proc.join(timeout)
        if self.proc.is_alive():
            self.proc.terminate()
            self.proc.join(5)
            return None, "oracle solve did not finish in %d s" % timeout
        if self.proc.exitcode != 0 or not os.path.exists(self.path):
            return None, "oracle process exited with code %s" % self.proc.exitcode
        H = np.load(self.path)
        with open(self.path + ".json") as f:
            info = json.load(f)
        for q in (self.path, self.path + ".json"):
            os.remove(q)
        return H, info


def bench_ppr(di, torch, dev, nbatches=3):
    """Batched personalized queries: R-MAT scale 20 (edge factor 16, a,b,c = .57,.19,.19, duplicates removed),
    d = 0.85, 64 queries with 1..32 uniform seeds, per-query bound 1e-6; one batch vs 64 single queries."""
    import graphgen as gg
    g = gg.rmat_graph(20, 16, seed=1)
    seeds = gg.seed_sets(g.n, 64, 1, 32, seed=7)
    G = di.DiGraph(g.n, torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col_idx).to(dev), 0.85)
    H = torch.empty((64, g.n), dtype=torch.float64, device=dev)
    for _ in range(2):
        G.query_batch(seeds, 1e-6, H_out=H)
    torch.cuda.synchronize()
    lat = []
    for _ in range(nbatches):
        t0 = time.perf_counter()
        _, stq, sta = G.query_batch(seeds, 1e-6, H_out=H)
        torch.cuda.synchronize()
        lat.append(time.perf_counter() - t0)
    h1 = torch.empty(g.n, dtype=torch.float64, device=dev)
    single = {}
    for name, prec in (("fp64", di.DI_FP64), ("fp32_mixed", di.DI_FP32_MIXED)):
        for q in range(2):
            G.query(seeds[q], 1e-6, H_out=h1, prec=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in range(64):
            G.query(seeds[q], 1e-6, H_out=h1, prec=prec)
        torch.cuda.synchronize()
        single[name] = time.perf_counter() - t0
    # one more batch with the sweep kernels launched from the host between events: the split of device
    # time over scan, push-or-pull and finalize (the captured loop above runs the same kernels)
    _, _, stp = G.query_batch(seeds, 1e-6, H_out=H, profile=1)
    # the autotuner for this width, then the same batches with its settings
    t0 = time.perf_counter()
    best, tried = G.autotune_batch(seeds, 1e-6)
    tune_s = time.perf_counter() - t0
    G.query_batch(seeds, 1e-6, H_out=H)
    torch.cuda.synchronize()
    tlat = []
    for _ in range(nbatches):
        t0 = time.perf_counter()
        _, stq_t, sta_t = G.query_batch(seeds, 1e-6, H_out=H)
        torch.cuda.synchronize()
        tlat.append(time.perf_counter() - t0)
    G.close()
    med, tmed = float(np.median(lat)), float(np.median(tlat))
    return {"workload": "R-MAT scale 20 (n=%d, L=%d), 64 queries x 1-32 seeds, d=0.85, per-query bound 1e-6" % (g.n, g.nnz),
            "batched_queries_per_s": 64 / med, "batch_ms": 1e3 * med, "sweeps": sta["sweeps"],
            "max_bound": max(s["bound"] for s in stq), "single_fp64_queries_per_s": 64 / single["fp64"],
            "single_fp32_mixed_queries_per_s": 64 / single["fp32_mixed"],
            "speedup": (64 / med) / (64 / single["fp64"]),
            "speedup_same_precision": (64 / med) / (64 / single["fp32_mixed"]),
            "lane_dtype": "f32 fluid rows, f64 histories",
            "kernel_ms": {k: round(v, 3) if isinstance(v, float) else v for k, v in stp["profile"].items()},
            "tuned": {"queries_per_s": 64 / tmed, "batch_ms": 1e3 * tmed, "vs_default": med / tmed,
                      "max_bound": max(s["bound"] for s in stq_t), "converged": bool(sta_t["converged"]),
                      "best": best, "candidates": len(tried), "tuning_s": tune_s}}


def bench_update(di, torch, G, g, d, tol, fracs=(1e-4, 1e-3, 1e-2)):
    """Graph update (Section 3.2) on the headline graph: P' keeps each edge with probability 1-f and gains
    f*L uniform random edges.  A converged solve on P (bound tol) continues on P' from
    F_0' = F + d(P'-P)H, against a solve of P' from F_0 = (1-d)V.  Device times include the injection."""
    import graphgen as gg
    dev = torch.device("cuda")
    H = torch.empty(g.n, dtype=torch.float64, device=dev)
    out = {"what": "edit f of the edges of the headline graph; continue its converged solve (bound %g) on the "
                   "edited graph vs solving the edited graph from scratch" % tol, "runs": []}
    for k, f in enumerate(fracs):
        g2 = gg.modify(g, f, int(f * g.nnz), seed=40 + k)
        G2 = di.DiGraph(g2.n, g2.row_ptr, g2.col_idx, d)
        G2.solve(tol, H_out=H)
        _, sc = G2.solve(tol, H_out=H)
        G.solve(tol, H_out=H)
        G2.update_from(G, tol, H_out=H)
        G.solve(tol, H_out=H)
        _, su = G2.update_from(G, tol, H_out=H)
        out["runs"].append({"f": f, "scratch_ms": 1e3 * sc["seconds"], "scratch_edges": sc["edges_pushed"],
                            "scratch_sweeps": sc["sweeps"], "update_ms": 1e3 * su["seconds"],
                            "update_edges": su["edges_pushed"], "update_sweeps": su["sweeps"],
                            "update_bound": su["bound"], "speedup": sc["seconds"] / su["seconds"]})
        log(f"update f={f}: {out['runs'][-1]}")
        G2.close()
    return out


def bench_selection(di, torch, graphs, tol):
    """ALGO-OP / ALGO-OP2 (Section 4.3) as weighted threshold sweeps vs the plain threshold, FP64, bound tol."""
    dev = torch.device("cuda")
    out = {}
    for name, (G, n) in graphs.items():
        H = torch.empty(n, dtype=torch.float64, device=dev)
        row = {}
        for sel in ("ref", "op", "op2"):
            G.solve(tol, H_out=H, select=sel)
            _, st = G.solve(tol, H_out=H, select=sel)
            row[sel] = {"ms": 1e3 * st["seconds"], "sweeps": st["sweeps"], "edges": st["edges_pushed"],
                        "bound": st["bound"]}
        out[name] = row
        log(f"selection {name}: {row}")
    return out


def bench_mixed(di, torch, zipf=None, scale=23, ds=(0.85, 0.99), tol=1e-7, ref_tol=1e-10):
    """FP32-mixed against FP64 D-iteration.  R-MAT (scale 23, edge factor 16, a,b,c = .57,.19,.19,
    duplicates removed), V = 1/N, bound 1e-7, d = 0.85 and 0.99, push only and with pull sweeps;
    and the headline Zipf graph (`zipf` = (DiGraph, graph, workload)) at its bound.  The FP64
    solve to bound 1e-10 is the reference H_ref (|X - H_ref|_1 <= 1e-10); the error of each
    result is |H - H_ref|_1 + 1e-10.  The d = 0.85 R-MAT results are kept on the host in
    `keep` so that the caller can add their distance to the oracle's solve."""
    import graphgen as gg
    g = gg.rmat_graph(scale, 16, seed=1)
    out = {"workload": "R-MAT scale %d (n=%d, L=%d), V=1/N, L1 bound %g, FP32-mixed vs FP64" % (scale, g.n, g.nnz, tol),
           "reference": "FP64 D-iteration to bound %g" % ref_tol, "runs": []}
    keep = {}
    dev = torch.device("cuda")
    for d in ds:
        G = di.DiGraph(g.n, g.row_ptr, g.col_idx, d)
        Href = torch.empty(g.n, dtype=torch.float64, device=dev)
        H = torch.empty(g.n, dtype=torch.float64, device=dev)
        for direction in (0, 1):                    # warm-up: graph capture, buffers, in-link CSR
            G.solve(tol, H_out=H, direction=direction)
            G.solve(tol, H_out=H, prec=di.DI_FP32_MIXED, direction=direction)
        _, sref = G.solve(ref_tol, H_out=Href)
        run = {"d": d}
        # push only, and with the pull direction on dense sweeps (di_solve_opts.direction = 1)
        for suffix, direction in (("", 0), ("_pull", 1)):
            for name, prec in (("fp64", di.DI_FP64), ("fp32_mixed", di.DI_FP32_MIXED)):
                _, st = G.solve(tol, H_out=H, prec=prec, direction=direction)
                torch.cuda.synchronize()
                err = float((H - Href).abs().sum().item()) + ref_tol
                run[name + suffix] = {"ms": 1e3 * st["seconds"], "edge_pushes_per_s": st["edges_pushed"] / st["seconds"],
                                      "sweeps": st["sweeps"], "edges": st["edges_pushed"], "bound": st["bound"],
                                      "l1_error_vs_reference": err}
                if d == 0.85:
                    keep[name + suffix] = H.cpu().numpy()
        run["fp32_speedup"] = run["fp64"]["ms"] / run["fp32_mixed"]["ms"]
        run["fp32_speedup_pull"] = run["fp64_pull"]["ms"] / run["fp32_mixed_pull"]["ms"]
        out["runs"].append(run)
        log(f"mixed precision d={d}: {run}")
        G.close()
    if zipf is not None:
        Gz, gz, wz = zipf
        Href = torch.empty(gz.n, dtype=torch.float64, device=dev)
        H = torch.empty(gz.n, dtype=torch.float64, device=dev)
        Gz.solve(wz["tol"], H_out=H, prec=di.DI_FP32_MIXED)
        Gz.solve(ref_tol, H_out=Href)
        zr = {"workload": "the headline Zipf graph (n=%d, L=%d), d=%g, bound %g" % (gz.n, gz.nnz, wz["d"], wz["tol"])}
        for name, prec in (("fp64", di.DI_FP64), ("fp32_mixed", di.DI_FP32_MIXED)):
            ms = []
            for _ in range(5):
                _, st = Gz.solve(wz["tol"], H_out=H, prec=prec)
                ms.append(1e3 * st["seconds"])
            torch.cuda.synchronize()
            zr[name] = {"ms": float(np.median(ms)), "edge_pushes_per_s": st["edges_pushed"] / (1e-3 * float(np.median(ms))),
                        "sweeps": st["sweeps"], "edges": st["edges_pushed"], "bound": st["bound"],
                        "l1_error_vs_reference": float((H - Href).abs().sum().item()) + ref_tol}
            keep["zipf24_" + name] = H.cpu().numpy()
        zr["fp32_speedup"] = zr["fp64"]["ms"] / zr["fp32_mixed"]["ms"]
        out["zipf24"] = zr
        log(f"mixed precision zipf: {zr}")
    return out, keep


def serve_trace(gs, rate, duration, seed):
    """Poisson arrivals at `rate` for `duration` s, graph uniform, seed sets of 1..16 distinct uniform nodes."""
    import graphgen as gg
    rng = np.random.default_rng(seed)
    nreq = int(rng.poisson(rate * duration))
    arr = np.sort(rng.uniform(0.0, duration, nreq))
    gof = rng.integers(0, len(gs), nreq)
    seeds = [gg.seed_set(gs[k].n, 1, 16, 500 + int(k), i) for i, k in enumerate(gof)]
    return arr, gof, seeds


def serve_run(di, srv, gs, ring, trace, tol, warm):
    """Open-loop replay through the server; latency = result in host memory - scheduled arrival."""
    arr, gof, seeds = trace
    arrival = {}
    lat, arr_counted = [], []
    t_end = 0.0
    per_g = [[] for _ in gs]
    t0 = di.di_clock() + 0.02
    i, n = 0, len(arr)
    t_first = t_last = None
    while True:
        now = di.di_clock()
        while i < n and t0 + arr[i] <= now:
            k = int(gof[i])
            tk = srv.submit(k, seeds[i], tol, ring[k][i % len(ring[k])])
            arrival[tk] = (t0 + arr[i], k, arr[i] >= warm)
            i += 1
        for c in srv.poll(0.0 if i < n else 0.01):
            a, k, counted = arrival.pop(c["ticket"])
            t_end = max(t_end, c["t_done"])
            if counted:
                lat.append(c["t_done"] - a)
                arr_counted.append(a)
                per_g[k].append(c["t_done"] - a)
                t_first = a if t_first is None else min(t_first, a)
                t_last = c["t_done"] if t_last is None else max(t_last, c["t_done"])
        if i >= n and not arrival:
            break
        if now - t0 > 300:
            raise RuntimeError("serving trace did not drain in 300 s")
    lat = np.array(lat) * 1e3
    dur = max(1e-9, t_last - t_first) if len(lat) else 1.0
    h = len(lat) // 2  # completions in arrival order of the counted queries: first and second half
    order = np.argsort(np.array(arr_counted)) if arr_counted else np.zeros(0, int)
    lat_o = lat[order] if len(order) == len(lat) else lat
    return {"offered_per_s": float(n / arr[-1]) if n else 0.0, "queries": int(len(lat)),
            "drain_s": float(t_end - (t0 + arr[-1])) if n else 0.0,
            "queries_per_s": float(len(lat) / dur) if len(lat) else 0.0,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p99_ms_halves": [float(np.percentile(lat_o[:h], 99)) if h else None,
                              float(np.percentile(lat_o[h:], 99)) if h else None],
            "p50_ms_halves": [float(np.percentile(lat_o[:h], 50)) if h else None,
                              float(np.percentile(lat_o[h:], 50)) if h else None],
            "p50_ms_per_graph": [round(float(np.percentile(np.array(v) * 1e3, 50)), 2) if v else None
                                 for v in per_g],
            "served_per_s_per_graph": [round(float(len(v) / dur), 1) for v in per_g]}


def stable(r, drain_s=1.5):
    """An open-loop run kept up with its arrivals: the last query finished within drain_s seconds
    of the last arrival (a server that falls behind builds a backlog that takes longer to drain),
    and its latency did not grow over the stream (the p50 and the p99 of the queries arriving in
    the second half within 1.5x those of the first half, + 50 ms)."""
    (a, b), (c, e) = r["p99_ms_halves"], r["p50_ms_halves"]
    return (a is not None and r["drain_s"] <= drain_s and b <= 1.5 * a + 50.0 and e <= 1.5 * c + 50.0)


def serve_one_at_a_time(di, Gs, gs, ring, trace, tol, count, prec=None):
    """The same arrival stream's first `count` queries, one at a time (di_query, FP64 unless prec
    says otherwise) in arrival order."""
    arr, gof, seeds = trace
    lat, t_first, t_end = [], None, None
    t0 = di.di_clock() + 0.02
    for i in range(min(count, len(arr))):
        a = t0 + arr[i]
        while di.di_clock() < a:
            pass
        k = int(gof[i])
        Gs[k].query(seeds[i], tol, H_out=ring[k][0], prec=di.DI_FP64 if prec is None else prec)
        t_end = di.di_clock()
        lat.append(t_end - a)
        t_first = a if t_first is None else t_first
    lat = np.array(lat) * 1e3
    return {"queries": int(len(lat)), "queries_per_s": len(lat) / (t_end - t_first),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}


def bench_serve(di, torch, scales=(16, 18, 20, 21, 22, 23), tol=1e-6, budget=120e9,
                runs=((2000.0, 2.0), (100.0, 4.0)), warm=0.5, base_count=100,
                ladder_rates=(100.0, 150.0, 200.0, 250.0, 300.0, 400.0), ladder_s=4.0):
    """Continuous batching over six R-MAT graphs (edge factor 16, d = 0.85), Poisson arrivals, graph uniform,
    seed sets U{1..16}, per-query bound 1e-6, lane pools under a 120 GB budget; every H copied to pinned host
    memory.  Queries arriving in the first `warm` seconds of a trace are not counted."""
    import graphgen as gg
    t = time.time()
    gs = [gg.rmat_graph(s, 16, seed=100 + s) for s in scales]
    Gs = [di.DiGraph(g.n, g.row_ptr, g.col_idx, 0.85) for g in gs]
    ring = [[torch.empty(g.n, dtype=torch.float64).pin_memory() for _ in range(4)] for g in gs]
    torch.cuda.synchronize()
    log(f"serving graphs ready in {time.time() - t:.1f}s")
    out = {"workload": "6 R-MAT graphs, scales %s, edge factor 16, d=0.85; Poisson arrivals, graph uniform, "
                       "1-16 uniform seeds, per-query bound 1e-6, H to pinned host memory" % (list(scales),),
           "nnz": [g.nnz for g in gs], "budget_bytes": int(budget)}
    with di.DiServer(Gs, mem_budget=int(budget), round_sweeps=8) as srv:
        out["lanes"] = srv.lanes()
        serve_run(di, srv, gs, ring, serve_trace(gs, 50.0, 0.5, 7), tol, 0.0)   # warm-up
        for rate, dur in runs:
            trace = serve_trace(gs, rate, dur, int(rate))
            out["poisson_%d" % int(rate)] = serve_run(di, srv, gs, ring, trace, tol, warm)
            log(f"serving at {rate} q/s: {out['poisson_%d' % int(rate)]}")
        # the highest offered rate the server keeps up with (a ladder of short streams)
        ladder = []
        for rate in ladder_rates:
            r = serve_run(di, srv, gs, ring, serve_trace(gs, rate, ladder_s, 1000 + int(rate)), tol, warm)
            ok = bool(stable(r))
            ladder.append({"offered_per_s": round(float(r["offered_per_s"]), 1),
                           "queries_per_s": round(float(r["queries_per_s"]), 1),
                           "p50_ms": round(r["p50_ms"], 2), "p99_ms": round(r["p99_ms"], 2),
                           "drain_s": round(r["drain_s"], 3),
                           "p50_ms_halves": [round(x, 2) for x in r["p50_ms_halves"]],
                           "p99_ms_halves": [round(x, 2) for x in r["p99_ms_halves"]], "stable": ok})
            log(f"serving ladder {rate} q/s: {ladder[-1]}")
            if not ok:
                break
        good = [x for x in ladder if x["stable"]]
        out["sustainable"] = {"queries_per_s": good[-1]["queries_per_s"] if good else None,
                              "p99_ms": good[-1]["p99_ms"] if good else None,
                              "offered_per_s": good[-1]["offered_per_s"] if good else None,
                              "rule": "highest offered rate of the ladder whose %g-s stream kept up: the last query done "
                                      "within 1.5 s of the last arrival, and the p50 and p99 of the second half's "
                                      "arrivals within 1.5x the first half's + 50 ms" % ladder_s,
                              "ladder": ladder}
        out["device_ms_per_graph"] = [round(srv.stats(k)["device_ms"], 1) for k in range(len(gs))]
    trace = serve_trace(gs, runs[0][0], runs[0][1], int(runs[0][0]))
    out["one_at_a_time"] = serve_one_at_a_time(di, Gs, gs, ring, trace, tol, base_count)
    out["one_at_a_time"]["what"] = "first %d queries of the %d q/s trace, di_query FP64 one by one" % (
        base_count, int(runs[0][0]))
    out["one_at_a_time_fp32_mixed"] = serve_one_at_a_time(di, Gs, gs, ring, trace, tol, base_count,
                                                          prec=di.DI_FP32_MIXED)
    out["one_at_a_time_fp32_mixed"]["what"] = "the same queries, di_query FP32-mixed (the lanes' precision)"
    for G in Gs:
        G.close()
    return out


def run_config(args, w, g, world):
    """The `config` object of both arms' JSON lines: the workload and the solve's settings."""
    return {"workload": w["label"], "n": g.n, "nnz": g.nnz, "d": w["d"], "tol": w["tol"], "beta": args.beta,
            "precision": "FP64" if args.prec == "fp64" else "FP32-mixed",
            "direction": "push, pull on dense sweeps" if args.direction else "push",
            "parallelism": "replicas" if world > 1 else "single-gpu",
            "l2": "inputs larger than L2 (CSR + F + H of the solve exceed 129 MB)"}


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    g = make_graph(w)
    # each step is the oracle's whole solve (about 4N diffusions; 8N bounds it): the first
    # sweep alone selects every node and is the fastest part, so a shorter cut overstates the
    # rate.  One solve takes a few seconds on one host core.
    cap = args.cpu_pushes if args.cpu_pushes > 0 else 8 * g.n
    vals, secs = [], []
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(g, w, cap)
        cb.pop("_H")
        if k >= args.warmup:
            vals.append(cb["value"])
            secs.append(cb["seconds"])
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": run_config(args, w, g, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="zipf24", choices=sorted(WORKLOADS))
    ap.add_argument("--beta", type=float, default=0.5)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"],
                    help="fluid precision of the timed and profiled solves (fp32: FP32-mixed)")
    ap.add_argument("--direction", type=int, default=0, choices=[0, 1],
                    help="1: dense sweeps pull along the in-links (di_solve_opts.direction)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-pushes", type=int, default=0,
                    help="diffusions in the oracle sample (0: 8N, which covers the full solve)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ppr", action="store_true", help="skip the batched personalized-query measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the continuous-batching serving measurement")
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP32-mixed vs FP64 measurement")
    ap.add_argument("--no-update", action="store_true", help="skip the graph-update and selection measurements")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warm-up below 3 is not allowed; using 3")
        args.warmup = 3
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)
    rank0 = dist_env()[0] == 0
    # the oracle's config-3 solve runs on a host core while the GPU measurements run
    orc_bg = OracleInBackground() if rank0 and not args.no_mixed and not args.no_cpu else None

    import torch
    import paper_1202_6158_gb300 as di

    prec = di.DI_FP64 if args.prec == "fp64" else di.DI_FP32_MIXED
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    t0 = time.perf_counter()
    g = make_graph(w)
    gen_s = time.perf_counter() - t0
    log(f"[rank {rank}] graph n={g.n} nnz={g.nnz} generated in {gen_s:.1f}s")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    ci_d = torch.from_numpy(g.col_idx).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G = di.DiGraph(g.n, rp_d, ci_d, w["d"])
    torch.cuda.synchronize()
    create_ms = 1e3 * (time.perf_counter() - t0)
    H = torch.empty(g.n, dtype=torch.float64, device=dev)
    X = torch.empty(g.n, dtype=torch.float64, device=dev)
    tol = w["tol"]

    # ---- warm-up, then K timed solves on device-resident inputs
    for _ in range(args.warmup):
        G.solve(tol, H_out=H, beta=args.beta, direction=args.direction, prec=prec)
    torch.cuda.synchronize()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    edges = 0
    launches = 0
    sweeps = []
    with ClockSampler(local) as clocks:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            _, st = G.solve(tol, H_out=H, beta=args.beta, direction=args.direction, prec=prec)
            edges += st["edges_pushed"]
            launches += st["kernel_launches"]
            sweeps.append(st["sweeps"])
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    bound = st["bound"]
    clk = clocks.summary()

    # ---- power iteration to the paper's stop rule at the same tolerance, same GPU and graph
    for _ in range(2):
        G.power(tol, X_out=X)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        _, pst = G.power(tol, X_out=X)
    p1.record(stream)
    torch.cuda.synchronize()
    pms = p0.elapsed_time(p1) / args.steps
    p_edges = pst["edges_pushed"]
    agree = float((H - X).abs().sum().item())

    # ---- profiled power iteration: pull kernel CUDA-event time
    _, ppst = G.power(tol, X_out=X, profile=1)
    # per in-link: source, target, z gather; per node: Y read + reset, x read + write, z write, d/outdeg
    pull_bytes_iter = g.nnz * (4 + 4 + 8) + g.n * (2 * 8 + 2 * 8 + 8 + 8)

    # ---- profiled solve: per-kernel CUDA-event times and algorithmic bytes from the trace
    G.solve(tol, H_out=H, beta=args.beta, profile=1, trace=1, direction=args.direction, prec=prec)
    prof = G.profile()
    trace = G.trace()
    s_f = 8 if prec == di.DI_FP64 else 4
    push_bytes = sum((4 + 2 * s_f) * t["edges"] + 16 * t["pushed"] for t in trace)
    scan_bytes = sum(g.n * s_f + t["sources"] * (s_f + 16 + 8) + 16 * t["pushed"] for t in trace)
    hbm_peak, peak_kind = load_peaks()
    kernels = {
        "push": {"ms": prof["push_ms"], "launches": prof["sweeps"], "alg_bytes": push_bytes},
        "scan": {"ms": prof["scan_ms"], "launches": prof["sweeps"], "alg_bytes": scan_bytes},
    }
    pull = {"ms": ppst["pull_ms"], "launches": ppst["sweeps"], "alg_bytes": pull_bytes_iter * ppst["sweeps"]}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    kd = kernels[dom]
    achieved = kd["alg_bytes"] / (kd["ms"] * 1e-3) / 1e9 if kd["ms"] > 0 else None
    # the committed DRAM summary is for the FP64 headline workload's push
    traffic = push_traffic() if dom == "push" and args.workload == "zipf24" and prec == di.DI_FP64 else None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": (achieved / hbm_peak) if achieved else None, "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else
                "fallback 6800 GB/s",
                "alg_bytes_per_launch": kd["alg_bytes"] / max(1, kd["launches"]),
                "avg_launch_us": 1e3 * kd["ms"] / max(1, kd["launches"]),
                "per_kernel": {k: {"ms_total": v["ms"], "launches": v["launches"],
                                   "GBps": v["alg_bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] > 0 else None}
                               for k, v in list(kernels.items()) + [("power iteration product", pull)]},
                "finalize_ms_total": prof["finalize_ms"]}

    # ---- end to end through the C ABI with pinned host buffers
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    ci_h = torch.from_numpy(g.col_idx).pin_memory()
    H_h = torch.empty(g.n, dtype=torch.float64).pin_memory()
    e2e_edges = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    split = np.zeros(3)  # host wall clock: create (copies in, ingest), solve (H out), free
    for _ in range(args.e2e_steps):
        ta = time.perf_counter()
        Ge = di.DiGraph(g.n, rp_h, ci_h, w["d"])
        torch.cuda.synchronize()
        tb = time.perf_counter()
        _, est = Ge.solve(tol, H_out=H_h, beta=args.beta, direction=args.direction)
        tc = time.perf_counter()
        Ge.close()
        torch.cuda.synchronize()
        split += [tb - ta, tc - tb, time.perf_counter() - tc]
        e2e_edges += est["edges_pushed"]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = 4 * (g.n + 1) + 4 * g.nnz
    d2h = 8 * g.n

    # ---- aggregate over ranks: sum of work, max of time
    (tot_edges, tot_e2e_edges), (max_ms, max_e2e) = aggregate_ranks(dist, dev, [edges, e2e_edges], [ms, e2e_s])

    ppr = None
    if rank == 0 and not args.no_ppr:
        ppr = bench_ppr(di, torch, dev)

    update = selection = None
    if rank == 0 and not args.no_update:
        update = bench_update(di, torch, G, g, w["d"], tol)
        import graphgen as gg
        gr = gg.rmat_graph(22, 16, seed=1)
        Gr = di.DiGraph(gr.n, gr.row_ptr, gr.col_idx, 0.85)
        selection = bench_selection(di, torch, {"zipf24": (G, g.n), "rmat22": (Gr, gr.n)}, tol)
        Gr.close()

    mixed, keep = None, {}
    if rank == 0 and not args.no_mixed:
        mixed, keep = bench_mixed(di, torch, zipf=(G, g, w))
        if orc_bg is not None:
            Ho, info = orc_bg.result()
            run = mixed["runs"][0]
            if Ho is None:
                run["oracle"] = {"unavailable": info}
            else:
                run["oracle"] = dict(info, what="the oracle's snapshot-sweep solve on one host core, same graph, "
                                               "d=0.85, bound 1e-7")
                for key in [k for k in keep if k in run]:
                    run[key]["l1_error_vs_oracle"] = float(np.abs(keep.pop(key) - Ho).sum())
            log(f"mixed precision vs oracle: {run.get('oracle')}")
            orc_bg = None

    serve = None
    if rank == 0 and not args.no_serve:
        serve = bench_serve(di, torch)

    if orc_bg is not None:
        orc_bg.result()  # nothing may run on the host cores while the CPU baselines are timed
    cpu = None
    if rank == 0 and not args.no_cpu:
        cap = args.cpu_pushes if args.cpu_pushes > 0 else 8 * g.n
        cpu = cpu_baseline(g, w, cap)
        cpu.pop("seconds", None)
        Ho = cpu.pop("_H")
        if cpu["converged"]:
            # the headline device solve (the last timed step's H) against the oracle's full solve,
            # and the FP64 and FP32-mixed solves of the mixed-precision measurement
            cpu["headline_l1_error_vs_oracle"] = float(np.abs(H.cpu().numpy() - Ho).sum())
            if mixed is not None and "zipf24" in mixed:
                for name in ("fp64", "fp32_mixed"):
                    Hk = keep.pop("zipf24_" + name, None)
                    if Hk is not None:
                        mixed["zipf24"][name]["l1_error_vs_oracle"] = float(np.abs(Hk - Ho).sum())
        cpu.update(cpu_power_baselines(g, w))
        cpu["cpu_model"] = cpu_model()
        cpu["nproc"] = os.cpu_count()

    if rank == 0:
        value = tot_edges / (max_ms * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == di.DI_FP64 else "f32 fluid, f64 history",
            "data": "synthetic",
            "config": run_config(args, w, g, world),
            "time_to_residual_ms": {"diter": max_ms / args.steps, "power": pms,
                                    "speedup_vs_power": pms / (max_ms / args.steps)},
            "diter": {"edges_per_solve": edges // args.steps, "sweeps": sweeps[-1], "bound": bound,
                      "edges_over_L": edges / args.steps / g.nnz},
            "power_iteration": {"iters": pst["sweeps"], "edges": p_edges, "value": p_edges / (pms * 1e-3),
                                "unit": UNIT, "bound": pst["bound"], "l1_diff_vs_diter": agree},
            "create_ms": create_ms,
            "roofline": roofline,
            "e2e": {"value": tot_e2e_edges / max_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "what": "pinned host CSR -> di_graph_create (copy, validation, ingest) -> di_solve to host H -> "
                            "di_free, host wall clock",
                    "split_ms": {k: round(1e3 * v / args.e2e_steps, 3)
                                 for k, v in zip(("create", "solve_to_host", "free"), split)}},
            "cpu_baseline": cpu,
            "ppr_batch": ppr,
            "serving": serve,
            "mixed_precision": mixed,
            "graph_update": update,
            "selection": selection,
            "clocks": clk,
            "gpu_launches": launches,
            "host": {"nproc": os.cpu_count()},
        }
        print(json.dumps(line), flush=True)
    G.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
