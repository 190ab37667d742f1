#!/usr/bin/env python3
"""Throughput benchmark of the semi-Lagrangian foot -> locate -> P1 path.

One benchmark step is one run of the whole hot path over the workload: the
S-step time loop of Algorithm 2 (foot, clip, walk from the previous foot
triangle, P1) replayed as one CUDA graph, starting from the initial start
triangles (so the first step's long strategy-(a) walk is included).

Default workload: the 4096 x 4096 graded, jittered mesh (16 785 409 nodes,
33 554 432 triangles), solid rotation, Gaussian data, dt = 0.02, 50 steps,
FP64, Hilbert-renumbered.  Metric: node-updates/s = N * S / time.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores instead, on bounded samples of the same workload.
Launch on N GPUs with torchrun: every rank runs its own copy of the workload
(independent problems, no collective on the data path), timing is the max
over ranks, value counts every rank's node-updates.
"""
import argparse
import gc
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

import sl_inputs as si  # noqa: E402

BYTES_PER_NODE = {"fp64": 64, "fp32": 48}   # algorithmic bytes per node-update


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="C3", choices=["C1", "C2", "C3", "C4", "C5"])
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32"],
                    help="precision of the batch workload C5 (default fp64)")
    ap.add_argument("--cells", type=int, default=None, help="override cells per side (smaller test runs)")
    ap.add_argument("--kernel", type=int, default=0, help="SL_OPT_KERNEL (0 auto, 1 plain FP64, 2 tiled)")
    ap.add_argument("--curve", default="auto", choices=["auto", "none", "hilbert", "morton"],
                    help="node / triangle numbering: auto = chosen by sl_autotune_layout (as given, Hilbert, "
                         "Morton), else that curve")
    ap.add_argument("--config-id", type=int, default=None, help="SL_OPT_CONFIG launch configuration (0..5); "
                    "default: chosen by sl_autotune")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 kernel comparison")
    ap.add_argument("--split", type=int, choices=[0, 1], default=None,
                    help="SL_OPT_SPLIT for the later steps (default: chosen by sl_autotune)")
    ap.add_argument("--study", choices=["courant", "structured"], default=None,
                    help="the paper's studies (Sec. 4), one JSON line: 'courant' = mean hops per "
                         "node-update and time per step against the Courant number for strategies (a) "
                         "and (b); 'structured' = walk (b) against the direct location on the "
                         "structured Courant grid at alpha = 5, N = 1e6..8e6")
    ap.add_argument("--study-cells", type=int, default=386,
                    help="cells per side of the study mesh (386: 1.5e5 nodes, the paper's size)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary workloads (C4 FP32, C5 FP64 and FP32) of the default line")
    ap.add_argument("--secondary-runs", type=int, default=5, help="timed runs of each secondary workload")
    ap.add_argument("--l2-window", type=int, choices=[0, 1], default=0,
                    help="SL_OPT_L2_WINDOW: walk records persisting in L2 during graph runs")
    ap.add_argument("--pdl", type=int, choices=[0, 1], default=1,
                    help="SL_OPT_PDL: step kernels launched with programmatic stream serialization")
    ap.add_argument("--records", type=int, choices=[0, 1], default=None,
                    help="SL_OPT_RECORDS for the double-float kernel (default: chosen by sl_autotune)")
    ap.add_argument("--precise", type=int, default=None,
                    help="SL_OPT_PRECISE: gradient bound G of the FP64 value path (default: the library's, 32; "
                         "0 = never)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(dist, seconds, device):
    """The slowest rank's timed region (every rank gets the same value)."""
    import torch
    if dist is None:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(nodes_per_rank, steps_per_run, runs, world, seconds):
    """node-updates/s of the whole job: every rank advances its own copy of
    the workload (replicas, weak scaling), timed by the slowest rank."""
    return nodes_per_rank * steps_per_run * runs * world / seconds


def launches_per_run(steps_per_run, double_float):
    """Kernels one timed run launches: the start-cache fill after the T^0
    reset, one step kernel per step and, for the double-float path, the value
    conversions to and from (hi, lo) pairs."""
    return steps_per_run + 1 + (2 if double_float else 0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


class Workload:
    """The meshes, fields, time steps and initial data of one benchmark run."""

    def __init__(self, name, probs, precision, n_steps, description):
        self.name = name
        self.probs = probs                      # list of sl_inputs.Problem
        self.precision = precision
        self.n_steps = n_steps
        self.description = description
        self.nodes = sum(p.mesh.n_nodes for p in probs)
        self.triangles = sum(p.mesh.n_tri for p in probs)


def build_workload(args):
    """The workload of a configuration (curve=auto until the layout is tuned)."""
    if args.config == "C5":
        prec = args.precision or "fp64"
        probs = si.batch_config(256, precision=prec)
        n = sum(p.mesh.n_nodes for p in probs)
        desc = (f"C5: 256 jittered meshes of {min(p.mesh.n_nodes for p in probs)}-"
                f"{max(p.mesh.n_nodes for p in probs)} nodes ({n} nodes in all), rotation / swirl / "
                f"Fourier-8 fields, Courant 5-30, 50 steps, {prec}, curve={args.curve}")
        return Workload("C5", probs, prec, 50, desc)
    prob = si.config(args.config, M=args.cells)
    m = prob.mesh
    desc = (f"{prob.name}: {m.M}x{m.M} {'graded ' if m.graded else ''}jittered mesh ({m.n_nodes} nodes, "
            f"{m.n_tri} triangles), field kind {prob.field.kind}, dt={prob.dt}, {prob.n_steps} steps, "
            f"{prob.precision}, curve={args.curve}")
    return Workload(prob.name, [prob], prob.precision, prob.n_steps, desc)


TRAFFIC_SOURCES = ("step_fast.cu", "step_fast_impl.cuh", "step_fast_c01.cu", "step_fast_c23.cu", "step_fast_c45.cu", "step_fast.cuh", "df.cuh", "predicates.cuh", "step_common.cuh", "step_kernels.cuh")


def committed_traffic(workload_key, split=0):
    """DRAM bytes per step of the dominant kernel (the fused step kernel, or
    the settle + finish passes of a split step) from the committed ncu
    summary (profiles/k_step_fast_df_c3_traffic.md), or None when the kernel
    sources changed since that capture, the workload differs or the form was
    not captured."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "profiles", "k_step_fast_df_c3_traffic.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and not line.startswith(("|", "#", " ", "`")):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(here, "paper_2104_09189_gb300", "csrc", f), "rb").read())
    if fields.get("source_sha256") != h.hexdigest() or fields.get("workload") != workload_key:
        return None
    key = "traffic_bytes_per_step_split" if split else "traffic_bytes_per_step_fused"
    return float(fields[key]) if key in fields else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def cpu_sample(wl, seconds, steps=2):
    """Time the oracle (as it stands) on a bounded sample of the workload:
    `steps` steps of a node range of the first problems, sized to about
    `seconds` of CPU work."""
    import oracle
    threads = oracle.default_threads()
    budget = seconds
    done_nodes, elapsed, parts = 0, 0.0, []
    for prob in wl.probs:
        om = oracle.OracleMesh(prob.mesh.xy, prob.mesh.tri)
        kind, par = prob.field.kind, prob.field.packed()
        n_cal = min(prob.mesh.n_nodes, 200_000)
        t0 = time.perf_counter()
        om.step(kind, par, prob.dt, 0, prob.v0, lo=0, hi=n_cal, nthreads=threads, want_feet=False)
        rate = n_cal / max(time.perf_counter() - t0, 1e-6)
        n_s = int(min(prob.mesh.n_nodes, max(1000, rate * budget / steps)))
        lo = (prob.mesh.n_nodes - n_s) // 2
        t0 = time.perf_counter()
        for st in range(steps):
            om.step(kind, par, prob.dt, st, prob.v0, lo=lo, hi=lo + n_s, nthreads=threads, want_feet=False)
        dt = time.perf_counter() - t0
        om.close()
        done_nodes += n_s * steps
        elapsed += dt
        parts.append(f"{prob.name} nodes [{lo}, {lo + n_s}) of {prob.mesh.n_nodes}")
        budget -= dt + n_s * steps / rate
        if budget <= 0:
            break
    # one thread on a smaller sample of the first problem (a few seconds)
    prob = wl.probs[0]
    om = oracle.OracleMesh(prob.mesh.xy, prob.mesh.tri)
    n1 = int(min(prob.mesh.n_nodes, max(1000, rate / threads * 3.0)))
    lo1 = (prob.mesh.n_nodes - n1) // 2
    t0 = time.perf_counter()
    om.step(prob.field.kind, prob.field.packed(), prob.dt, 0, prob.v0, lo=lo1, hi=lo1 + n1, nthreads=1, want_feet=False)
    one = n1 / (time.perf_counter() - t0)
    om.close()
    return {"value": done_nodes / elapsed, "unit": "node-updates/s", "cores": threads, "kind": "oracle",
            "sample": f"{steps} steps (n=0..{steps - 1}) of " + "; ".join(parts[:4]) +
                      (f" and {len(parts) - 4} more problems" if len(parts) > 4 else "") +
                      f"; bin grid build excluded; {threads} threads",
            "value_1_thread": one,
            "sample_1_thread": f"step n=0 of {prob.name} nodes [{lo1}, {lo1 + n1}), 1 thread"}


def oracle_reference(probs, n_steps):
    """V^{n_steps} of the FP64 oracle for every problem (original numbering),
    its threads over the machine's host cores."""
    import oracle
    out = []
    for p in probs:
        om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
        out.append(om.run(p.field.kind, p.field.packed(), p.dt, 0, n_steps, p.v0))
        om.close()
    return out


def error_vs_oracle(probs, got, want):
    """Errors of a GPU result against the FP64 oracle: max and L2 (RMS) of
    the absolute error, and the normwise relative error max|dV| / max|V^0|
    of the worst problem (P1 is a convex combination, so max|V^0| bounds
    every value of a run)."""
    off = np.cumsum([0] + [p.mesh.n_nodes for p in probs])
    err = np.abs(got - np.concatenate(want))
    rel = max(float(err[off[k]:off[k + 1]].max() / max(np.abs(p.v0).max(), 1e-300)) for k, p in enumerate(probs))
    return {"max_abs": float(err.max()), "l2_rms": float(np.sqrt((err ** 2).mean())), "max_rel_to_max_v0": rel,
            "reference": "CPU oracle (FP64), same problems and steps"}


class _Args:
    """The subset of the command-line arguments build_workload reads."""

    def __init__(self, config, precision, curve="auto"):
        self.config, self.precision, self.cells, self.curve = config, precision, None, curve


def secondary_workload(sl, torch, config, precision, runs, warmup, oracle_cache):
    """A further workload measured beside the headline one (C4: the FP32
    filtered-precision path on the 16.8M-node mesh; C5: the 256-problem
    batch, FP64 and FP32): the same timed path as the headline (autotuned,
    one CUDA graph per run, runs queued back to back, CUDA events), the
    result's error against the FP64 oracle, the exact-stage (fallback) test
    count and the speed-up over the plain FP64 GPU kernel on the same
    problems."""
    wl = build_workload(_Args(config, precision))
    S, N = wl.n_steps, wl.nodes
    prec = sl.SL_FP64 if precision == "fp64" else sl.SL_FP32
    no, to, xy, tri = sl.pack_meshes([(p.mesh.xy, p.mesh.tri) for p in wl.probs])
    probs = sl.problems([(p.field.kind, p.dt, p.field.packed()) for p in wl.probs])
    v0_all = np.concatenate([p.v0 for p in wl.probs])

    def handle(pr):
        h = sl.sl_mesh_create(no, to, xy, tri, precision=pr, seed=wl.probs[0].seed)
        lp, _ = sl.sl_mesh_reorder(h, sl.SL_CURVE_HILBERT)
        perm = lp.astype(np.int64) + np.repeat(no[:-1], np.diff(no))
        return h, perm

    h = sl.sl_mesh_create(no, to, xy, tri, precision=prec, seed=wl.probs[0].seed)
    vt = torch.float64 if prec == sl.SL_FP64 else torch.float32
    v, w = torch.tensor(v0_all, dtype=vt, device="cuda"), torch.empty(N, dtype=vt, device="cuda")
    lp, _, tune = sl.sl_autotune_layout(h, probs, 3, v, w)
    wl.description = wl.description.replace("curve=auto", f"curve={tune['curve']} (autotuned)")
    perm = lp.astype(np.int64) + np.repeat(no[:-1], np.diff(no))
    v0 = v.clone()
    sl.sl_mesh_set_option(h, sl.SL_OPT_STATS, 1)
    sl.sl_mesh_stats(h, reset=True)
    sl.sl_mesh_reset_t0(h)
    v.copy_(v0)
    sl.sl_run(h, probs, 0, S, v, w, use_graph=True)
    stats = sl.sl_mesh_stats(h, reset=True)
    got = np.empty(N)
    got[perm] = v.double().cpu().numpy()
    sl.sl_mesh_set_option(h, sl.SL_OPT_STATS, 0)
    for _ in range(warmup):
        sl.sl_mesh_reset_t0(h)
        sl.sl_run(h, probs, 0, S, v, w, use_graph=True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sl.sl_mesh_set_option(h, sl.SL_OPT_ASYNC, 1)
    e0.record(stream)
    for _ in range(runs):
        sl.sl_mesh_reset_t0(h)
        sl.sl_run(h, probs, 0, S, v, w, use_graph=True, stats=False)
    e1.record(stream)
    torch.cuda.synchronize()
    sl.sl_mesh_set_option(h, sl.SL_OPT_ASYNC, 0)
    sl.sl_mesh_status(h)
    ms = e0.elapsed_time(e1) / runs
    sl.sl_mesh_destroy(h)
    # the plain FP64 kernel on the same problems (FP64 mesh), one run
    hp, pp = handle(sl.SL_FP64)
    sl.sl_mesh_set_option(hp, sl.SL_OPT_KERNEL, 1)
    a64 = torch.tensor(v0_all[pp], dtype=torch.float64, device="cuda")
    b64 = torch.empty_like(a64)
    sl.sl_run(hp, probs, 0, S, a64, b64, use_graph=True)
    sl.sl_mesh_reset_t0(hp)
    a64.copy_(torch.tensor(v0_all[pp], dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    e0.record(stream)
    sl.sl_run(hp, probs, 0, S, a64, b64, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    sl.sl_mesh_destroy(hp)
    del v, w, v0, a64, b64
    torch.cuda.empty_cache()
    key = config
    if key not in oracle_cache:
        t0 = time.perf_counter()
        oracle_cache[key] = (oracle_reference(wl.probs, S), time.perf_counter() - t0)
    want, oracle_s = oracle_cache[key]
    err = error_vs_oracle(wl.probs, got, want)
    bpn = BYTES_PER_NODE[precision]
    peaks, peak_src = measured_peaks()
    value = N * S / (ms / 1e3)
    achieved = bpn * N * S / (ms / 1e3) / 1e9
    return {
        "workload": wl.description, "nodes": N, "steps_per_run": S, "precision": precision,
        "value": value, "unit": "node-updates/s", "ms_per_run": ms, "runs": runs,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks.get("hbm_gbs", 6800.0), "unit": "GB/s",
                     "frac": achieved / peaks.get("hbm_gbs", 6800.0), "algorithmic_bytes_per_node": bpn,
                     "peak_source": peak_src},
        "error_vs_fp64_oracle": err,
        "walk": {"mean_hops_per_node_update": stats["walk_moves"] / max(1, stats["node_updates"]),
                 "exact_tests": stats["exact_tests"], "filter2_tests": stats["filter2_tests"],
                 "fallback_tests": stats["exact_tests"] + stats["filter2_tests"], "clipped": stats["clipped"]},
        "plain_fp64": {"value": N * S / (plain_ms / 1e3), "ms_per_run": plain_ms},
        "speedup_vs_plain_fp64": plain_ms / ms,
        "autotune": tune, "oracle_seconds": oracle_s,
    }


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = build_workload(args)
    per_step = max(1.0, 120.0 / max(1, args.steps + args.warmup))
    import oracle
    threads = oracle.default_threads()
    prob = wl.probs[0]
    om = oracle.OracleMesh(prob.mesh.xy, prob.mesh.tri)
    kind, par = prob.field.kind, prob.field.packed()
    n_cal = min(prob.mesh.n_nodes, 100_000)
    t0 = time.perf_counter()
    om.step(kind, par, prob.dt, 0, prob.v0, lo=0, hi=n_cal, nthreads=threads, want_feet=False)
    rate = n_cal / max(time.perf_counter() - t0, 1e-6)
    n_s = int(min(prob.mesh.n_nodes, max(10_000, rate * per_step)))
    times = []
    v = prob.v0
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        om.step(kind, par, prob.dt, k % prob.n_steps, v, lo=0, hi=n_s, nthreads=threads, want_feet=False)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n_s * len(times) / total
    line = {
        "impl": "reference", "metric": "node-updates/s (foot+locate+P1)", "value": value,
        "unit": "node-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, wl),
        "cpu_baseline": {"value": value, "unit": "node-updates/s", "cores": threads, "kind": "oracle",
                         "sample": f"each step: one SL step of nodes [0, {n_s}) of {prob.name} "
                                   f"({prob.mesh.n_nodes} nodes), {threads} threads"},
        "e2e": {"value": value, "unit": "node-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args, wl):
    return {"workload": wl.description, "nodes": wl.nodes, "triangles": wl.triangles, "problems": len(wl.probs),
            "steps_per_run": wl.n_steps, "precision": wl.precision,
            "l2": "inputs larger than L2 (129 MB)" if wl.nodes * 64 > 2 * 129e6 else "inputs may fit in L2"}


STUDY_ALPHAS = (0.25, 0.5, 1, 2, 4, 6, 8, 10, 12, 14, 16, 18, 20)


def run_study(args):
    """Dependence on the Courant number (Sec. 4): the paper's rotating field
    f = (cos(C0 |x - c| + C1 t), sin(...)), |f| = 1, L_x = C0 = 2 pi and
    L_t = C1 in {2 pi, 8 pi}; dt = alpha dx, ceil(1/dt) steps over t in
    [0, 1]; nodes whose foot leaves the domain excluded; hops averaged over
    the located node-updates.  Strategy (a) starts every walk at the node's
    own incident triangle, (b) at the previous step's foot triangle, (c) at
    the triangle just located for the node's parent in a breadth-first
    spanning tree (one launch per tree level, no graph)."""
    import torch
    import paper_2104_09189_gb300 as sl
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    M = args.study_cells
    mesh = si.grid_mesh(M, 0.25, 7)
    no, to, xy, tri = sl.pack_meshes([(mesh.xy, mesh.tri)])
    h = sl.sl_mesh_create(no, to, xy, tri, precision=sl.SL_FP64, seed=7)
    node_perm, _ = sl.sl_mesh_reorder(h, sl.SL_CURVE_HILBERT)
    sl.sl_mesh_set_option(h, sl.SL_OPT_OUTSIDE, 1)
    sl.sl_mesh_set_option(h, sl.SL_OPT_STATS, 1)
    v0 = torch.tensor(si.cosine_bump(mesh.xy, 0.5, 0.75, 0.15)[node_perm], dtype=torch.float64, device="cuda")
    v = v0.clone()
    w = torch.empty_like(v)
    stream = torch.cuda.current_stream()
    rows = []
    for lt_name, lt in (("2pi", 2 * np.pi), ("8pi", 8 * np.pi)):
        f = si.paper_field(2 * np.pi, lt)
        for alpha in STUDY_ALPHAS:
            dt = alpha / M
            S = int(np.ceil(1.0 / dt))
            probs = sl.problems([(f.kind, dt, f.packed())])
            for strategy, name in ((1, "a"), (0, "b"), (3, "c")):
                sl.sl_mesh_set_option(h, sl.SL_OPT_STRATEGY, strategy)
                sl.sl_mesh_stats(h, reset=True)
                v.copy_(v0)
                sl.sl_run(h, probs, 0, S, v, w, use_graph=True)       # records the graph; statistics
                st = sl.sl_mesh_stats(h, reset=True)
                sl.sl_mesh_reset_t0(h)
                v.copy_(v0)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sl.sl_run(h, probs, 0, S, v, w, use_graph=True)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                located = st["node_updates"] - st["excluded"]
                rows.append({"Lt": lt_name, "alpha": alpha, "strategy": name, "steps": S,
                             "mean_hops": st["walk_moves"] / max(1, located),
                             "excluded_fraction": st["excluded"] / max(1, st["node_updates"]),
                             "ms_per_step": ms / S, "ns_per_located_node_update": 1e6 * ms / max(1, located)})
    sl.sl_mesh_destroy(h)
    print(json.dumps({"study": "courant", "source": "Sec. 4, dependence on the Courant number",
                      "mesh": {"cells": M, "nodes": mesh.n_nodes, "triangles": mesh.n_tri, "jitter": 0.25,
                               "dx": 1.0 / M, "curve": "hilbert"},
                      "field": "paper (cos(C0|x-c|+C1 t), sin(...)), C0 = 2 pi, c = (0.5, 0.5)",
                      "outside": "excluded", "precision": "fp64 (double-float kernel)", "rows": rows}), flush=True)


def _timed_run(sl, torch, h, probs, S, v, v0, w):
    """One S-step run (graph) for the statistics, then the same run timed
    with CUDA events.  Returns (ms, stats of the first run)."""
    stream = torch.cuda.current_stream()
    sl.sl_mesh_stats(h, reset=True)
    sl.sl_mesh_reset_t0(h)
    v.copy_(v0)
    sl.sl_run(h, probs, 0, S, v, w, use_graph=True)
    st = sl.sl_mesh_stats(h, reset=True)
    sl.sl_mesh_reset_t0(h)
    v.copy_(v0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sl.sl_run(h, probs, 0, S, v, w, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), st


def run_study_structured(args):
    """Comparison with a structured grid (Sec. 4): on the Courant grid of M x M
    cells the foot's triangle has a direct formula; the paper times it against
    the walk (b) at L_x = L_t = 2 pi, alpha = 5, N from 1e6 to 8e6, location
    plus barycentric coordinates included.  Here each arm is the full step
    (foot, location, P1) with feet outside excluded: walk (b) on a jittered
    mesh of the same size, walk (b) on the Courant grid, and the direct
    location on the Courant grid (strategy 2, a certified walk from the
    formula's triangle)."""
    import torch
    import paper_2104_09189_gb300 as sl
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    f = si.paper_field(2 * np.pi, 2 * np.pi)
    rows = []
    for M in (1000, 1414, 2000, 2828):
        dt = 5.0 / M
        S = int(np.ceil(1.0 / dt))
        probs = sl.problems([(f.kind, dt, f.packed())])
        for mesh_name, mesh in (("jittered", si.grid_mesh(M, 0.25, 17)), ("courant", si.courant_grid(M))):
            no, to, xy, tri = sl.pack_meshes([(mesh.xy, mesh.tri)])
            h = sl.sl_mesh_create(no, to, xy, tri, precision=sl.SL_FP64, seed=17)
            node_perm, _ = sl.sl_mesh_reorder(h, sl.SL_CURVE_HILBERT)
            sl.sl_mesh_set_option(h, sl.SL_OPT_OUTSIDE, 1)
            sl.sl_mesh_set_option(h, sl.SL_OPT_STATS, 1)
            v0 = torch.tensor(si.cosine_bump(mesh.xy, 0.5, 0.75, 0.15)[node_perm], dtype=torch.float64,
                              device="cuda")
            v = v0.clone()
            w = torch.empty_like(v)
            arms = [("walk_b", 0)] + ([("direct", 2)] if mesh_name == "courant" else [])
            for arm, strategy in arms:
                sl.sl_mesh_set_option(h, sl.SL_OPT_STRATEGY, strategy)
                ms, st = _timed_run(sl, torch, h, probs, S, v, v0, w)
                located = st["node_updates"] - st["excluded"]
                rows.append({"cells": M, "nodes": mesh.n_nodes, "mesh": mesh_name, "location": arm, "steps": S,
                             "mean_hops": st["walk_moves"] / max(1, located),
                             "excluded_fraction": st["excluded"] / max(1, st["node_updates"]),
                             "ms_per_step": ms / S, "ns_per_located_node_update": 1e6 * ms / max(1, located)})
            sl.sl_mesh_destroy(h)
            del v, w, v0
            torch.cuda.empty_cache()
    print(json.dumps({"study": "structured", "source": "Sec. 4, comparison with a structured grid",
                      "field": "paper (cos(C0|x-c|+C1 t), sin(...)), C0 = C1 = 2 pi, c = (0.5, 0.5)",
                      "alpha": 5, "outside": "excluded", "precision": "fp64 (double-float kernel)",
                      "rows": rows}), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.study == "structured":
        return run_study_structured(args)
    if args.study:
        return run_study(args)
    import torch
    import paper_2104_09189_gb300 as sl
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    wl = build_workload(args)
    S = wl.n_steps
    N = wl.nodes
    prec = sl.SL_FP64 if wl.precision == "fp64" else sl.SL_FP32
    t_setup = time.perf_counter()
    no, to, xy, tri = sl.pack_meshes([(p.mesh.xy, p.mesh.tri) for p in wl.probs])
    h = sl.sl_mesh_create(no, to, xy, tri, precision=prec, seed=wl.probs[0].seed)
    tuning = args.config_id is None and args.kernel != 1
    if args.kernel:
        sl.sl_mesh_set_option(h, sl.SL_OPT_KERNEL, args.kernel)
    if args.config_id is not None:
        sl.sl_mesh_set_option(h, sl.SL_OPT_CONFIG, args.config_id)
        sl.sl_mesh_set_option(h, sl.SL_OPT_CONFIG_FIRST, args.config_id)
    if args.precise is not None and prec == sl.SL_FP64:
        sl.sl_mesh_set_option(h, sl.SL_OPT_PRECISE, args.precise)
    probs = sl.problems([(p.field.kind, p.dt, p.field.packed()) for p in wl.probs])
    vt = torch.float64 if prec == sl.SL_FP64 else torch.float32
    v0_all = np.concatenate([p.v0 for p in wl.probs])
    tune = None
    if args.curve == "auto" and tuning:
        # numbering, then launch configurations, by measurement
        v = torch.tensor(v0_all, dtype=vt, device="cuda")
        w = torch.empty_like(v)
        lperm, _, tune = sl.sl_autotune_layout(h, probs, 3, v, w)
        wl.description = wl.description.replace("curve=auto", f"curve={tune['curve']} (autotuned)")
    else:
        curve = {"none": sl.SL_CURVE_NONE, "hilbert": sl.SL_CURVE_HILBERT, "morton": sl.SL_CURVE_MORTON}[
            "hilbert" if args.curve == "auto" else args.curve]
        lperm, _ = sl.sl_mesh_reorder(h, curve)
    perm = lperm.astype(np.int64) + np.repeat(no[:-1], np.diff(no))     # global new -> old
    v0 = torch.tensor(v0_all[perm], dtype=vt, device="cuda")
    v = v0.clone()
    w = torch.empty_like(v)
    stream = torch.cuda.current_stream()
    if tuning and tune is None:
        tune = sl.sl_autotune(h, probs, 3, v, w)
    if args.split is not None:
        sl.sl_mesh_set_option(h, sl.SL_OPT_SPLIT, args.split)
    if args.records is not None and prec == sl.SL_FP64:
        sl.sl_mesh_set_option(h, sl.SL_OPT_RECORDS, args.records)
    if args.l2_window:
        sl.sl_mesh_set_option(h, sl.SL_OPT_L2_WINDOW, 1)
    if not args.pdl:
        sl.sl_mesh_set_option(h, sl.SL_OPT_PDL, 0)
    split = (args.split if args.split is not None else (tune or {}).get("split", 0)) if prec == sl.SL_FP64 else 0
    setup_s = time.perf_counter() - t_setup

    def one_run():
        sl.sl_mesh_reset_t0(h)
        sl.sl_run(h, probs, 0, S, v, w, use_graph=True)

    # first run records the graph; collect walk statistics on a separate run
    sl.sl_mesh_set_option(h, sl.SL_OPT_STATS, 1)
    sl.sl_mesh_stats(h, reset=True)
    one_run()
    stats = sl.sl_mesh_stats(h, reset=True)
    sl.sl_mesh_set_option(h, sl.SL_OPT_STATS, 0)
    for _ in range(args.warmup):
        one_run()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # one event before each run and one after the last (the runs are timed
    # as a whole; the per-run spread shows host stalls between runs); the
    # collector is paused so that it cannot stall the launching thread
    # runs are queued back to back (SL_OPT_ASYNC): a host stall between two
    # launches then only eats into the queued work; the device status of all
    # runs is checked once after the region
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    sl.sl_mesh_set_option(h, sl.SL_OPT_ASYNC, 1)
    gc.disable()
    evs[0].record(stream)
    for k in range(args.steps):
        sl.sl_mesh_reset_t0(h)
        sl.sl_run(h, probs, 0, S, v, w, use_graph=True, stats=False)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    gc.enable()
    sl.sl_mesh_set_option(h, sl.SL_OPT_ASYNC, 0)
    sl.sl_mesh_status(h)
    if dist:
        dist.barrier()
    elapsed = evs[0].elapsed_time(evs[-1]) / 1e3
    per_run = [evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)]
    clocks = sampler.stop()
    elapsed = max_over_ranks(dist, elapsed, "cuda")

    # phases: the first step (walks start at the initial incident triangles)
    # and the remaining steps (walks start at the previous foot triangles)
    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    sl.sl_mesh_reset_t0(h)
    first_ms = timed(lambda: sl.sl_run(h, probs, 0, 1, v, w, use_graph=False))
    rest_ms = timed(lambda: sl.sl_run(h, probs, 1, S - 1, v, w, use_graph=False)) / max(1, S - 1)
    phases = {"first_step_ms": first_ms, "later_step_ms": rest_ms,
              "note": "eager launches, one run, after the timed region"}

    # the effective gather roofline of a later step: a kernel making exactly
    # its memory accesses (on the current start triangles) with no arithmetic
    gather = None
    if prec == sl.SL_FP64 and args.kernel != 1:
        probe_ms = sl.sl_probe_gather(h, v, w, reps=20)
        gather = {"probe_ms": probe_ms, "later_step_ms": rest_ms, "frac_of_gather_bound": probe_ms / rest_ms,
                  "kernel": "k_gather_probe (node pair and start state, three vertex pairs, three values, one write)"}

    # FP32 workloads: the error of the result against the FP64 oracle
    fp32_check = None
    if wl.precision == "fp32" and not args.no_cpu and rank == 0 and args.cells is None:
        sl.sl_mesh_reset_t0(h)
        vv = v0.clone()
        sl.sl_run(h, probs, 0, S, vv, w, use_graph=True)
        got = np.empty(N)
        got[perm] = vv.double().cpu().numpy()
        fp32_check = error_vs_oracle(wl.probs, got, oracle_reference(wl.probs, S))

    plain = None
    if wl.precision == "fp64" and not args.no_plain and args.kernel != 1:
        sl.sl_mesh_set_option(h, sl.SL_OPT_KERNEL, 1)
        one_run()
        k_plain = 2
        tp = timed(lambda: [one_run() for _ in range(k_plain)]) / 1e3
        plain = {"value": N * S * k_plain / tp, "unit": "node-updates/s", "ms_per_step": 1e3 * tp / k_plain,
                 "kernel": "plain FP64 step (one thread per node, all arithmetic in double)"}
        sl.sl_mesh_set_option(h, sl.SL_OPT_KERNEL, args.kernel)

    value = whole_job_value(N, S, args.steps, world, elapsed)
    launch_s = elapsed / (args.steps * S)
    bpn = BYTES_PER_NODE[wl.precision]
    peaks, peak_src = measured_peaks()
    achieved_gbs = bpn * N / launch_s / 1e9
    hbm = peaks.get("hbm_gbs", 6800.0)

    def phase(ms):
        a = bpn * N / (ms / 1e3) / 1e9
        return {"ms": ms, "achieved": a, "frac": a / hbm}

    phase_roofline = {"first_step": phase(first_ms), "later_steps": phase(rest_ms),
                      "note": "eager launches after the timed region; the first step walks from the initial "
                              "incident triangles, the later ones from the previous foot triangles"}

    # end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        host = torch.tensor(v0_all[perm], dtype=vt).pin_memory()
        hv = host.numpy()
        sl.sl_mesh_reset_t0(h)
        sl.sl_run_host(h, probs, 0, S, hv, use_graph=True)
        torch.cuda.synchronize()
        k_e2e = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            sl.sl_mesh_reset_t0(h)
            sl.sl_run_host(h, probs, 0, S, hv, use_graph=True)
        e2e_s = time.perf_counter() - t0
        esize = 8 if prec == sl.SL_FP64 else 4
        e2e = {"value": N * S * k_e2e * world / e2e_s, "unit": "node-updates/s",
               "h2d_bytes_per_step": N * esize, "d2h_bytes_per_step": N * esize,
               "api": "sl_run_host (pinned host V in/out, graph replay, status read)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_sample(wl, args.cpu_seconds)

    sl.sl_mesh_destroy(h)
    del v, w, v0
    torch.cuda.empty_cache()

    # the precision and batching patterns on their own workloads
    secondary = None
    if (rank == 0 and world == 1 and not args.no_secondary and args.config == "C3" and args.cells is None
            and args.kernel != 1):
        cache = {}
        secondary = [secondary_workload(sl, torch, c, p, args.secondary_runs, 2, cache)
                     for c, p in (("C4", "fp32"), ("C5", "fp64"), ("C5", "fp32"))]

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": "node-updates/s (foot+locate+P1)",
        "value": value,
        "unit": "node-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps,
        "step_definition": f"one benchmark step = one run of the whole path: {S} SL steps of the workload "
                           "(sl_run, one CUDA graph) from the initial start triangles",
        "ms_per_sl_step": 1e3 * elapsed / (args.steps * S),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f64" if args.kernel == 1 else "df64 (FP32 pairs, 48-bit significand; FP64-accuracy results)")
                 if prec == sl.SL_FP64 else "f32",
        "data": "synthetic",
        "config": workload_config(args, wl),
        "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks.get("hbm_gbs", 6800.0),
                     "unit": "GB/s", "frac": achieved_gbs / peaks.get("hbm_gbs", 6800.0),
                     "traffic": (committed_traffic(f"{args.config} {wl.precision}", split)
                                 if args.kernel != 1 and args.cells is None else None),
                     "peak_source": peak_src,
                     "algorithmic_bytes_per_node": bpn,
                     "kernel": ("k_step_plain_f64" if args.kernel == 1 else
                                ("k_step_fast_df" + (" (later steps split: k_settle_df + k_finish_df)" if split else "")
                                 if prec == sl.SL_FP64 else "k_step_fast_f32"))
                               + " (one step over all nodes; duration = timed region / steps)",
                     "launch_ms": launch_s * 1e3,
                     "phases": phase_roofline},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * (launches_per_run(S, prec == sl.SL_FP64 and args.kernel != 1)
                                      + (S - 1 if split else 0)),
        "clocks": clocks,
        "walk": {"first_run_mean_hops_per_node_update": stats["walk_moves"] / max(1, stats["node_updates"]),
                 "max_hops": stats["max_moves"], "exact_tests": stats["exact_tests"],
                 "filter2_tests": stats["filter2_tests"], "clipped": stats["clipped"],
                 "fallbacks": stats["fallbacks"]},
        "setup_s": setup_s,
        "phases": phases,
        "per_run_ms": {"min": min(per_run), "median": statistics.median(per_run), "max": max(per_run)},
        "gather_probe": gather,
        "autotune": tune,
        "plain_fp64": plain,
        "speedup_vs_plain_fp64": (value / world) / plain["value"] if plain else None,
        "fp32_error_vs_fp64_oracle": fp32_check,
        "secondary": secondary,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
