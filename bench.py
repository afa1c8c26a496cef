#!/usr/bin/env python
"""Benchmark of the CEM explicit step on GB300.

Workload: the 0.1 x 0.04 x 0.01 m notched block refined to 200 x 80 x 10
hexahedral cells split into six tetrahedra each (960,000 elements, 179,091
nodes), E = 32 GPa, nu = 0.2, rho = 2450 kg/m^3, Gc = 3 J/m^2, 1 MPa traction
on the top and bottom faces, element splitting on.  A "step" is one explicit
time step of the whole path: predictor, element strains, smoothed edge
stresses, element forces, node update, energy release rates of the crack-front
elements and the splits they trigger.

Metric: tet-steps/s = (input elements) x (timed steps) / (device time), max
over ranks, summed over ranks (independent replicas; the step is not sharded
across GPUs).  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cem|reference]

--impl reference times the CPU FP64 oracle (test infrastructure) on the same
workload on the host cores, single-threaded.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

if "reference" in sys.argv or "--cpu-baseline-worker" in sys.argv or "--cpu-allcore-worker" in sys.argv:
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        os.environ[_v] = "1"

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tet-steps/s"
CHUNK_STEPS = 500    # steps between host reads of the mesh counts in the timed region
PROFILE_EVERY = 16   # kernel timing sampled on every 16th step (events between kernels block launch overlap)
WORKLOAD = "notched_block_200x80x10"


def _workload(name="block"):
    if name == "ensemble":
        from cem_inputs import ensemble
        return ensemble()
    from cem_inputs import plate_medium
    return plate_medium()


KERNEL_UNITS = {"predict": "nodes", "strain": "tets", "edge_stress": "edges", "force": "tets", "node_update": "nodes"}

# DRAM bytes (read + write) per unit measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch, divided by the launch's units: 982,000 elements, 1,219,792 edges, 187,533 nodes after the notch)
# on the intact 960,000-element block, for the kernels as they are now.  Source:
# profiles/step_kernels_fp64_notched_block_200x80x10.md and profiles/step_kernels_mixed_notched_block_200x80x10.md.
DRAM_BYTES_PER_UNIT = {"fp64": {"strain": 107.1, "edge_stress": 103.8, "force": 216.3, "node_update": 837.3},
                       "mixed": {"strain": 63.0, "edge_stress": 70.5, "force": 129.1, "node_update": 556.1}}


def b_alg_per_tet_step(T, E, N, precision):
    """Algorithmic bytes per element-step of the whole step (the survey's model, section 8(d)).

    Each algorithmic array is streamed once per step; gathers hit in L2; the
    intermediates h (element strains), sigma (edge stresses) and the element forces
    are not algorithmic (a perfectly fused step keeps them on chip).  FP64:
      node state u r/w, v r/w, 1/m, f_ext   128 B per node
      connectivity (4 x i32)                 16 B per element
      geometry V grad N (9 x f64)            72 B per element
      edge fan CSR (6 i32 per element, one i32 offset per edge)  24 + 4 E/T
      edge 1/sum V (f64)                      8 B per edge
      node CSR (4 i32 per element, one i32 offset per node)       16 + 4 N/T
    Mixed: geometry (36 B) and 1/sum V (4 B) in FP32, and a Kahan compensation of u
    (80 B per node: the survey's +14 B per element-step at N/T = 0.1738).
    """
    n, e = N / T, E / T
    b = 128.0 * n + 16 + 72 + 24 + 4.0 * e + 8.0 * e + 16 + 4.0 * n
    if precision == "mixed":
        b += -36.0 - 4.0 * e + 80.0 * n
    return b


def flops_per_tet_step(T, E, N):
    """Algorithmic FP64 flops per element-step of the whole step (FMA = 2): the sum of
    kernel_costs' per-unit counts weighted by units per element."""
    fl, _, _ = kernel_costs(T, E, N, "fp64")
    return fl["predict"] * N / T + fl["strain"] + fl["edge_stress"] * E / T + fl["force"] + fl["node_update"] * N / T


def kernel_costs(T, E, N, precision):
    """Per unit of each hot kernel: (FP64 flops, algorithmic bytes, moved bytes).

    Flops (FMA = 2) are counted from the kernels' arithmetic.  Algorithmic bytes
    charge each array of b_alg_per_tet_step to the first kernel of the step that
    reads it (so they sum to the whole step's figure): the predictor the u read and
    write (the node update in mixed precision, which carries the predictor),
    strain the connectivity and geometry, edge stress the fan lists and 1/sum V,
    the node update v, 1/m, f_ext, the incidence lists and (mixed) the Kahan term;
    the force kernel reads only intermediates and the element-edge map.  Moved
    bytes are what the kernel as written reads and writes, each array once,
    intermediates included (gathered operands counted once per producer).
    f = mean fan size 6T/E, g = mean node incidence 4T/N.
    """
    f, g = 6.0 * T / E, 4.0 * T / N
    flops = {"predict": 12.0, "strain": 57.0, "edge_stress": 6.0 * f + 13.0, "force": 90.0,
             "node_update": 3.0 * g + 18.0}
    if precision == "fp64":
        alg = {"predict": 48.0, "strain": 16.0 + 72.0, "edge_stress": 4.0 * f + 4.0 + 8.0, "force": 0.0,
               "node_update": 48.0 + 8.0 + 24.0 + 4.0 * g + 4.0}
        moved = {"predict": 96.0,
                 "strain": 16 + 72 + 48 + 24.0 * N / T,
                 "edge_stress": 8 + 4.0 * f + 16 + 48 + 48.0 * T / E,
                 "force": 24 + 72 + 96 + 48.0 * E / T,
                 "node_update": 8 + 4.0 * g + 24 + 8 + 96 + 96.0 * T / N}
    else:
        alg = {"predict": 0.0, "strain": 16.0 + 36.0, "edge_stress": 4.0 * f + 4.0 + 4.0, "force": 0.0,
               "node_update": 48.0 + 48.0 + 8.0 + 24.0 + 4.0 * g + 4.0 + 80.0}
        moved = {"predict": 0.0,   # carried by the node update
                 "strain": 16 + 36 + 32 + 32.0 * N / T,
                 "edge_stress": 8 + 4.0 * f + 8 + 32 + 32.0 * T / E,
                 "force": 24 + 36 + 64 + 32.0 * E / T,
                 "node_update": 8 + 4.0 * g + 24 + 8 + 96 + 80 + 64.0 * T / N}
    return flops, alg, moved


def roofline_accounting(chunks, prof, precision, scale, t_ms, hbm, fp64_peak):
    """Per-kernel figures, the dominant step kernel's roofline and the whole step's.

    chunks: [(counts, steps, {kernel: (ms, launches)})] for consecutive windows of the
    timed region; counts holds the window's mean n_active_tets, n_edges and n_nodes,
    steps the window's step count and the dict the sampled launches' time and number in
    that window.  prof: {kernel: (total ms, launches)} over the whole region; scale =
    timed steps / sampled steps; t_ms the region's time; hbm the HBM peak in GB/s;
    fp64_peak the FP64 FMA rate in FLOP/s.  The flops and bytes of a sampled launch are
    the per-unit figures of kernel_costs for its window's sizes times its units, so a
    mesh that grows during the run is accounted window by window.

    The dominant kernel's roofline: FP64 path, bound "alu": its FP64 flops per launch /
    its mean launch time against fp64_peak (the FP64 step kernels do several FP64
    operations per algorithmic byte, far above GB300's FP64-to-HBM balance of about 0.19
    flop/B).  Mixed path, bound "hbm": its algorithmic bytes per launch / its mean launch
    time against hbm.  The whole step: algorithmic bytes (flops) of every element-step of
    the region / the region's time, against the same peaks.
    """
    acc = {k: dict(bytes=0.0, moved=0.0, flops=0.0, units=0.0, traffic=0.0) for k in KERNEL_UNITS}
    per_unit = DRAM_BYTES_PER_UNIT.get(precision, {})
    whole_bytes = whole_flops = elem_steps = 0.0
    for cnt, nsteps, dp in chunks:
        T, E, N = cnt["n_active_tets"], cnt["n_edges"], cnt["n_nodes"]
        fl, alg, mv = kernel_costs(T, E, N, precision)
        whole_bytes += b_alg_per_tet_step(T, E, N, precision) * T * nsteps
        whole_flops += flops_per_tet_step(T, E, N) * T * nsteps
        elem_steps += T * nsteps
        for k, (_, nl) in dp.items():
            units = {"tets": T, "edges": E, "nodes": N}[KERNEL_UNITS[k]]
            acc[k]["bytes"] += nl * alg[k] * units
            acc[k]["moved"] += nl * mv[k] * units
            acc[k]["flops"] += nl * fl[k] * units
            acc[k]["units"] += nl * units
            acc[k]["traffic"] += nl * (per_unit.get(k) or 0.0) * units
    kernels = {}
    for k, (ms_tot, nl) in prof.items():
        kernels[k] = {"ms": ms_tot * scale, "launches_timed": nl, "share": ms_tot * scale / max(t_ms, 1e-9)}
        if k in KERNEL_UNITS and nl:
            sec = ms_tot * 1e-3
            kernels[k].update(per_launch_us=sec / nl * 1e6, alg_gbs=acc[k]["bytes"] / sec / 1e9,
                              moved_gbs=acc[k]["moved"] / sec / 1e9, fp64_tflops=acc[k]["flops"] / sec / 1e12)
    hot = {k: prof[k] for k in KERNEL_UNITS}
    dom = max(hot, key=lambda k: hot[k][0])
    ms_tot, nl = hot[dom]
    nl = max(nl, 1)
    per_launch_s = ms_tot * 1e-3 / nl
    units = acc[dom]["units"] / nl
    flops, bytes_, moved = acc[dom]["flops"] / nl, acc[dom]["bytes"] / nl, acc[dom]["moved"] / nl
    if precision == "fp64":
        achieved, peak, unit, bound = flops / per_launch_s / 1e12, fp64_peak / 1e12, "TFLOP/s", "alu"
        src = "FP64 FMA rate measured live on this GPU (cem_probe_fp64_fma, FMA = 2 FLOP)"
    else:
        achieved, peak, unit, bound = bytes_ / per_launch_s / 1e9, hbm, "GB/s", "hbm"
        src = "HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    traffic = acc[dom]["traffic"] / nl if per_unit.get(dom) else None
    t_s = t_ms * 1e-3
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak if peak else None, "traffic": traffic, "peak_source": src,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per unit of the current "
                                   "kernel on the intact 960,000-element block, times the units per launch"
                                   if traffic else None),
                "per_launch_us": per_launch_s * 1e6, "algorithmic_flops_per_launch": flops,
                "algorithmic_bytes_per_launch": bytes_, "moved_bytes_per_launch": moved,
                "units_per_launch": units,
                "units_integrated_over": "%d windows of <= %d steps" % (len(chunks), CHUNK_STEPS),
                "whole_step": {
                    "b_alg_per_element_step": whole_bytes / max(elem_steps, 1.0),
                    "flops_per_element_step": whole_flops / max(elem_steps, 1.0),
                    "alg_gbs": whole_bytes / t_s / 1e9, "hbm_peak_gbs": hbm,
                    "hbm_frac": whole_bytes / t_s / 1e9 / hbm if hbm else None,
                    # the FP64 figures only for the FP64 path (mixed precision does its element and
                    # edge arithmetic in FP32)
                    "fp64_tflops": whole_flops / t_s / 1e12 if precision == "fp64" else None,
                    "fp64_peak_tflops": fp64_peak / 1e12,
                    "fp64_frac": whole_flops / t_s / fp64_peak if (fp64_peak and precision == "fp64") else None,
                    "active_element_steps_per_s": elem_steps / t_s}}
    return kernels, roofline


# --------------------------------------------------------------------------- helpers
def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=19995)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["cem", "reference"], default="cem")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                   help="precision of the headline run (default: plain FP64); the other runs as a sub-object")
    p.add_argument("--workload", choices=["block", "ensemble"], default="block",
                   help="block: the 960,000-element notched block; ensemble: 256 notched blocks of "
                        "5k-200k elements (about 2.6e7) advanced as one union mesh")
    p.add_argument("--adjoint-steps", type=int, default=5000,
                   help="steps of the gradient (adjoint) sub-run on the 102,000-element block; 0 skips it")
    p.add_argument("--ensemble-steps", type=int, default=200,
                   help="steps of the ensemble sub-run in the default (block) mode; 0 skips it")
    p.add_argument("--hex-steps", type=int, default=1000,
                   help="steps of the hexahedral (ES-H-FEM) sub-run on 200x80x10 hexahedra; 0 skips it")
    p.add_argument("--no-compare", action="store_true", help="skip the second-precision run and agreement check")
    p.add_argument("--no-graph", action="store_true", help="skip the graph-replay comparison")
    p.add_argument("--no-autotune", action="store_true", help="keep the default launch variants")
    p.add_argument("--reorder-growth", type=float, default=None,
                   help="renumber node storage after this fractional node growth (0: never; default: the "
                        "library's)")
    p.add_argument("--split-capacity", type=int, default=0,
                   help="max elements that may split (0: all); lower it to shrink device memory for profiling")
    p.add_argument("--state", help="checkpoint file for --save-at / --resume")
    p.add_argument("--save-at", type=int, default=0,
                   help="run the benchmark workload this many steps, write its state to --state and exit "
                        "(to profile a late window of the job without replaying it)")
    p.add_argument("--resume", action="store_true",
                   help="load --state into a fresh context and time --steps steps from there, then exit")
    p.add_argument("--cpu-baseline-worker", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--cpu-allcore-worker", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--cpu-steps", type=int, default=80, help=argparse.SUPPRESS)
    return p.parse_args()


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


HBM_FALLBACK_GBS = 6800.0   # the profiling recipe's fallback copy bandwidth, used only without MEASURED_PEAKS.json


def _hbm_peak(peaks):
    """(HBM GB/s, source): the measured copy bandwidth, else the recipe's fallback."""
    if peaks.get("hbm_gbs"):
        return float(peaks["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    return HBM_FALLBACK_GBS, "of fallback (no MEASURED_PEAKS.json: the recipe's 6.8 TB/s)"


def _leg(name, fn):
    """Run a secondary leg; a failure is recorded in the line instead of losing it."""
    try:
        return fn()
    except Exception as ex:   # reported, not hidden
        return {"error": "%s: %r" % (name, ex)}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 100 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "100"]
        if bus_id:
            cmd += ["-i", bus_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def wait_first(self, timeout=5.0):
        """Block until nvidia-smi has written its first sample (or timeout)."""
        t0 = time.time()
        while self.p is not None and time.time() - t0 < timeout:
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                return True
            time.sleep(0.05)
        return False

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _bus_id(dev):
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return None


def _oracle_rate(steps):
    """Time the CPU oracle on the benchmark workload: (tet-steps/s, steps, seconds)."""
    from oracle import CEMOracle
    w = _workload()
    o = CEMOracle.from_workload(w)
    o.step(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return w.n_tets * steps / dt, steps, dt


def _host_cpu():
    """The host's logical CPU count and model name (lscpu), for the baseline record."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def _single_thread_env():
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    return env


ALLCORE_BLOCK = (100, 40, 10, 0.05, 0.02, 0.01, 0.025)   # the benchmark's cell shape on a quarter of its block


def _allcore_workload():
    from cem_inputs import kuhn_block
    nx, ny, nz, lx, ly, lz, notch = ALLCORE_BLOCK
    return kuhn_block(nx, ny, nz, lx, ly, lz, notch_length=notch, traction=1e6)


def _allcore_worker(steps):
    """One single-threaded oracle process of the all-core baseline: set up, report ready,
    wait for the go line on stdin, time `steps` steps, report."""
    from oracle import CEMOracle
    w = _allcore_workload()
    o = CEMOracle.from_workload(w)
    o.step(1)
    print("ready", flush=True)
    sys.stdin.readline()
    t0 = time.time()
    o.step(steps)
    t1 = time.time()
    print(json.dumps({"tets": w.n_tets, "steps": steps, "t0": t0, "t1": t1}), flush=True)


def _cpu_baseline(steps, allcore_steps=20):
    """The oracle on the host cores; returns the cpu_baseline object.

    value: one single-threaded process on the benchmark workload (steps 2..steps+1).
    all_cores: one single-threaded process per logical CPU at once, each on a quarter-size
    block of the same cell shape (one benchmark-size oracle per core would not fit in host
    memory): every process sets up untimed, then all start together; the figure is the
    elements x steps of all processes over the span from the first start to the last end.
    """
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker", "--cpu-steps", str(steps)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=_single_thread_env(), timeout=1800)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    out = {"value": res["value"], "unit": METRIC, "cores": 1, "kind": "oracle",
           "sample": "%s, steps 2-%d of the run (%.1f s of CPU time; setup untimed), "
                     "single-threaded numpy/scipy FP64 oracle" % (WORKLOAD, res["steps"] + 1, res["seconds"]),
           "host": _host_cpu()}
    try:
        n = os.cpu_count() or 1
        wcmd = [sys.executable, os.path.abspath(__file__), "--cpu-allcore-worker", "--cpu-steps", str(allcore_steps)]
        procs = [subprocess.Popen(wcmd, stdin=subprocess.PIPE, stdout=subprocess.PIPE, text=True,
                                  env=_single_thread_env()) for _ in range(n)]
        for p in procs:
            if p.stdout.readline().strip() != "ready":
                raise RuntimeError("an all-core worker failed to set up")
        for p in procs:
            p.stdin.write("go\n")
            p.stdin.flush()
        rows = [json.loads(p.stdout.readline()) for p in procs]
        for p in procs:
            p.wait(timeout=600)
        span = max(r_["t1"] for r_ in rows) - min(r_["t0"] for r_ in rows)
        work = sum(r_["tets"] * r_["steps"] for r_ in rows)
        nx, ny, nz = ALLCORE_BLOCK[:3]
        out["all_cores"] = {"value": work / span, "unit": METRIC, "cores": n, "kind": "oracle",
                            "sample": "%d single-threaded oracle processes at once, each %d steps of a %dx%dx%d "
                                      "notched block (%d elements, the benchmark's cell shape); %.1f s span"
                                      % (n, allcore_steps, nx, ny, nz, rows[0]["tets"], span)}
    except Exception as ex:   # reported, not hidden
        out["all_cores"] = {"error": repr(ex)}
    return out


# --------------------------------------------------------------------------- arms
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = _workload()
    from oracle import CEMOracle
    o = CEMOracle.from_workload(w)
    o.step(max(1, min(a.warmup, 3)))
    budget_s = 150.0
    t0 = time.perf_counter()
    done = 0
    while done < a.steps and (time.perf_counter() - t0) < budget_s:
        o.step(1)
        done += 1
    dt = time.perf_counter() - t0
    value = w.n_tets * done / dt
    line = {"metric": METRIC, "value": value, "unit": METRIC, "impl": "reference", "n_gpus": a.gpus,
            "steps": done, "warmup": a.warmup, "ms_per_step": 1e3 * dt / done, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tets": w.n_tets, "nodes": w.n_nodes, "precision": "fp64",
                       "split": True},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": "%s, %d steps after %d warm-up steps (capped at %.0f s), single-threaded"
                                       % (WORKLOAD, done, max(1, min(a.warmup, 3)), budget_s),
                             "host": _host_cpu()},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x, world, device):
    """x's maximum over the ranks of the default process group (x itself for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(n_tets, steps, world, t_ms):
    """Whole-job tet-steps/s of `world` independent replicas, timed by the slowest rank."""
    return n_tets * steps * world / (t_ms * 1e-3)


def _reorder(sim, a):
    if a.reorder_growth is not None:
        sim.set_reorder(a.reorder_growth)


def run_cem(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = local

    from paper_2508_04076_gb300 import CEM, probe_fp64_fma

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    w = _workload(a.workload)
    if a.workload == "ensemble" and a.split_capacity == 0:
        a.split_capacity = w.n_tets // 4
    stream = torch.cuda.current_stream(dev)
    if a.save_at > 0 or a.resume:   # checkpointed windows of the job (profiling aid)
        if not a.state:
            raise SystemExit("--save-at and --resume need --state PATH")
        sim = CEM.from_workload(w, device=dev, split_capacity=a.split_capacity, precision=a.precision)
        _reorder(sim, a)
        if a.save_at > 0:
            if not a.no_autotune:
                sim.autotune(reps=10, automatic=True)
            sim.step(a.save_at)
            sim.save(a.state)
            info = sim.info()
            print(json.dumps({"saved": a.state, "step": a.save_at, "elements": info["n_active_tets"],
                              "nodes": info["n_nodes"], "edges": info["n_edges"]}), flush=True)
        else:
            sim.load(a.state)
            if not a.no_autotune:   # variants for the loaded mesh, tuned before the timed window
                sim.autotune(reps=10, automatic=True)
            step0 = sim.energy()["step"]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(a.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            info = sim.info()
            print(json.dumps({"resumed": a.state, "from_step": step0, "steps": a.steps,
                              "ms_per_step": e0.elapsed_time(e1) / max(a.steps, 1),
                              "launch_variants": None if a.no_autotune else sim.tuning(),
                              "elements": info["n_active_tets"], "nodes": info["n_nodes"],
                              "edges": info["n_edges"]}), flush=True)
        sim.close()
        return
    peaks = _peaks()
    hbm, hbm_src = _hbm_peak(peaks)
    fp64_peak = probe_fp64_fma(dev, stream.cuda_stream)

    def timed(precision, clocks_on, w=w, steps=None, split_capacity=None, keep_u=False):
        """W untimed then K timed steps of a fresh context: metrics of the timed region."""
        steps = a.steps if steps is None else steps
        cap = a.split_capacity if split_capacity is None else split_capacity
        sim = CEM.from_workload(w, device=dev, split_capacity=cap, precision=precision)
        _reorder(sim, a)
        info0 = sim.info()
        if not a.no_autotune:   # launch variants for the current sizes; re-tuned in the run as the mesh grows
            sim.autotune(reps=10, automatic=True)
        # clocks: the sampler runs from before the warm-up steps to after the timed region (a
        # short timed region may see no sample of its own at nvidia-smi's 100 ms period)
        clocks = ClockSampler(_bus_id(dev)) if (clocks_on and rank == 0) else None
        if clocks:
            clocks.wait_first()
        sim.step(a.warmup)
        barrier()
        sim.profile(max(1, min(PROFILE_EVERY, steps // 4)))   # at least a few sampled steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # The mesh grows during the run, so the sampled launches' units (elements, edges, nodes)
        # are integrated window by window: each window's sampled kernel time is paired with the
        # mean of its first and last counts.  The counts and timing sums are read on the host
        # between windows; every step already ends with a host read of its split count.
        chunks = []
        c_prev, p_prev = sim.info(), {k: (0.0, 0) for k in KERNEL_UNITS}
        e0.record(stream)
        done = 0
        while done < steps:
            n = min(CHUNK_STEPS, steps - done)
            sim.step(n)
            done += n
            c_now = sim.info()
            p_now = sim.profile_read()[0]
            chunks.append(({u: (c_prev[u] + c_now[u]) / 2.0 for u in ("n_active_tets", "n_edges", "n_nodes")}, n,
                           {k: (p_now[k][0] - p_prev[k][0], p_now[k][1] - p_prev[k][1]) for k in KERNEL_UNITS}))
            c_prev, p_prev = c_now, {k: p_now[k] for k in KERNEL_UNITS}
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms = e0.elapsed_time(e1)
        if clocks:
            time.sleep(0.25)   # one more sample after the region
        clk = clocks.stop() if clocks else None
        if clk is not None:
            clk["window"] = "from before the warm-up steps to 0.25 s after the timed region"
        prof, launches = sim.profile_read()
        sim.profile(0)
        barrier()
        t_ms = max_over_ranks(t_ms, world, "cuda")
        info = sim.info()
        energy = sim.energy()
        u = sim.field("u") if keep_u else None
        cracks = {(r[0], r[3]) for r in sim.crack_state()}
        tuning = {k: {"block": v[0], "batch": v[1]} for k, v in sim.tuning().items()}
        sim.close()
        # timed launches are a sample (every PROFILE_EVERY-th step): scale sums to the whole region
        n_sampled = max(prof["strain"][1], 1)
        if prof["strain"][1] == 0:
            raise RuntimeError("no sampled step in the timed region")
        scale = steps / n_sampled
        kernels, roofline = roofline_accounting(chunks, prof, precision, scale, t_ms, hbm, fp64_peak)
        roofline["whole_step"]["hbm_peak_source"] = hbm_src
        return dict(t_ms=t_ms, value=replica_throughput(w.n_tets, steps, world, t_ms), roofline=roofline,
                    kernels=kernels, clocks=clk, launches=launches, info0=info0, info=info, energy=energy,
                    steps=steps, tuning=tuning, u=u, cracks=cracks)

    main = timed(a.precision, True, keep_u=a.workload == "block")
    other_prec = "mixed" if a.precision == "fp64" else "fp64"

    def other_leg():
        o = timed(other_prec, False, keep_u=a.workload == "block")
        f64, mx = (main, o) if a.precision == "fp64" else (o, main)
        out = {"value": o["value"], "ms_per_step": o["t_ms"] / a.steps, "roofline": o["roofline"],
               "kernels": {k: {kk: v[kk] for kk in ("ms", "share", "per_launch_us", "alg_gbs", "moved_gbs")
                               if kk in v} for k, v in o["kernels"].items()},
               "gpu_launches": o["launches"],
               "speedup_mixed_over_fp64": mx["value"] / f64["value"],
               "after_timed_region": {"steps": a.warmup + a.steps}}
        if f64["u"] is not None and mx["u"] is not None and f64["u"].shape == mx["u"].shape:
            out["after_timed_region"]["rel_l2_u_mixed_vs_fp64"] = float(
                np.linalg.norm(mx["u"] - f64["u"]) / max(np.linalg.norm(f64["u"]), 1e-300))
        out["after_timed_region"]["split_jaccard"] = (len(f64["cracks"] & mx["cracks"]) /
                                                      max(len(f64["cracks"] | mx["cracks"]), 1))
        return out

    other = None if a.no_compare else _leg(other_prec, other_leg)

    # agreement of the two precisions through crack growth (both paths from the same start)
    def agree_leg():
        n_cmp = 500
        s64 = CEM.from_workload(w, device=dev, split_capacity=a.split_capacity, precision="fp64")
        s32 = CEM.from_workload(w, device=dev, split_capacity=a.split_capacity, precision="mixed")
        s64.step(n_cmp)
        s32.step(n_cmp)
        u64, u32 = s64.field("u"), s32.field("u")
        c64 = {(r[0], r[3]) for r in s64.crack_state()}
        c32 = {(r[0], r[3]) for r in s32.crack_state()}
        rel = (float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64)) if u32.shape == u64.shape else None)
        s64.close()
        s32.close()
        return {"steps": n_cmp, "rel_l2_u_mixed_vs_fp64": rel,
                "split_jaccard": len(c64 & c32) / max(len(c64 | c32), 1), "splits_fp64": len(c64)}

    agree = _leg("precision_agreement", agree_leg) if (not a.no_compare and a.workload == "block") else None

    # the 256-specimen ensemble as one union mesh, mixed against FP64 (default block mode only)
    def ens_leg():
        we = _workload("ensemble")
        em = timed("mixed", False, w=we, steps=a.ensemble_steps, split_capacity=we.n_tets // 4)
        ef = timed("fp64", False, w=we, steps=a.ensemble_steps, split_capacity=we.n_tets // 4)
        return {"workload": we.name, "instances": we.params["n_instances"], "tets": we.n_tets,
                "steps": a.ensemble_steps, "warmup": a.warmup,
                "mixed": {"value": em["value"], "ms_per_step": em["t_ms"] / a.ensemble_steps,
                          "roofline": {k: em["roofline"][k] for k in ("bound", "kernel", "achieved", "peak", "unit",
                                                                      "frac", "whole_step")}},
                "fp64": {"value": ef["value"], "ms_per_step": ef["t_ms"] / a.ensemble_steps,
                         "roofline": {k: ef["roofline"][k] for k in ("bound", "kernel", "achieved", "peak", "unit",
                                                                     "frac", "whole_step")}},
                "mixed_speedup_over_fp64": em["value"] / ef["value"],
                "split_elements_at_end_mixed": em["energy"]["n_split"]}

    ens = _leg("ensemble", ens_leg) if (a.workload == "block" and a.ensemble_steps > 0) else None

    # steps launched as one captured CUDA graph (cem_step_graph) against eager launches: on
    # fixed topology (splitting off after the notch) for a small specimen, where launches
    # dominate, and the 256-specimen ensemble; and with splitting on for the ensemble and the
    # benchmark block, whose notches leave crack-front elements, against eager steps that read
    # the split decision after every step (step batch 1) and in batches (the default)
    def graph_leg():
        from cem_inputs import plate_small
        out = {"note": "graph: one capture, then the timed replay; the same kernels and arguments as eager "
                       "stepping (bit-identical).  persistent: one cooperative launch per call, grid barriers "
                       "between the phases (bit-identical).  split_enabled = 0 after the notch, except for the "
                       "cases with crack fronts, where a split ends the replay and the rest of the call runs "
                       "eagerly; 'splits' counts the run-time splits at the end"}
        cases = [("notched_block_20x8x2", plate_small(), 2000, "fp64", False)]
        if a.ensemble_steps > 0:
            we = _workload("ensemble")
            cases.append(("ensemble_256_seed4", we, a.ensemble_steps, "mixed", False))
            cases.append(("ensemble_256_seed4_crack_fronts", we, a.ensemble_steps, "mixed", True))
        cases.append((w.name + "_crack_fronts", w, 100, "fp64", True))
        for name, wk, steps, prec, fronts in cases:
            res = {"tets": wk.n_tets, "steps": steps, "precision": prec}
            for mode in (("eager_per_step", "eager", "graph") if fronts else ("eager", "graph", "persistent")):
                cap = (wk.n_tets // 4 if name.startswith("ensemble") else a.split_capacity) if fronts else 0
                sg = CEM.from_workload(wk, device=dev, split_enabled=fronts, precision=prec, split_capacity=cap)
                if mode == "eager_per_step":
                    sg.set_step_batch(1)
                run = {"graph": sg.step_graph, "persistent": sg.step_persistent}.get(mode, sg.step)
                run(steps)   # warm-up (and the capture)
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run(steps)
                e1.record(stream)
                torch.cuda.synchronize()
                t_ms = e0.elapsed_time(e1)
                res[mode] = {"value": wk.n_tets * steps / (t_ms * 1e-3), "ms_per_step": t_ms / steps}
                if fronts:
                    res[mode]["splits"] = sg.energy()["n_split"]
                sg.close()
            res["graph_speedup"] = res["graph"]["value"] / res["eager"]["value"]
            if not fronts:
                res["persistent_speedup"] = res["persistent"]["value"] / res["eager"]["value"]
            if fronts:
                res["batch_speedup"] = res["eager"]["value"] / res["eager_per_step"]["value"]
            out[name] = res
        return out

    graph = _leg("graph", graph_leg) if (a.workload == "block" and not a.no_graph) else None

    # gradients: FP32 forward + adjoint with sqrt(N) checkpoints on the 102,000-element block,
    # J = final strain energy + mean top-face y displacement, topology frozen after the notch
    def adj_leg():
        from cem_inputs import adjoint_block, top_face_weights
        wa = adjoint_block()
        res = {}
        for prec in ("mixed", "fp64"):
            sa = CEM.from_workload(wa, device=dev, split_enabled=False, precision=prec)
            wu = top_face_weights(sa.field("X"))
            barrier()
            t0 = time.perf_counter()
            J, dE, da = sa.adjoint(a.adjoint_steps, c_strain=1.0, w_u=wu)
            torch.cuda.synchronize()
            res[prec] = (time.perf_counter() - t0, J, dE, da)
            sa.close()
        tm, Jm, dEm, dam = res["mixed"]
        tf, Jf, dEf, daf = res["fp64"]
        return {"workload": wa.name, "tets": wa.n_tets, "steps": a.adjoint_steps,
                "checkpoint_every": int(np.ceil(np.sqrt(a.adjoint_steps))),
                "mixed": {"seconds": tm, "tet_steps_per_s": wa.n_tets * a.adjoint_steps / tm},
                "fp64": {"seconds": tf, "tet_steps_per_s": wa.n_tets * a.adjoint_steps / tf},
                "rel_err_J_mixed": abs(Jm - Jf) / abs(Jf),
                "rel_err_dJdE_mixed": float(np.abs(dEm - dEf).max() / np.abs(dEf).max()),
                "rel_err_dJdalpha_mixed": abs(dam - daf) / abs(daf),
                "note": "wall time of one cem_adjoint call: forward, segment recompute and reverse sweep"}

    adj = _leg("adjoint", adj_leg) if (a.workload == "block" and a.adjoint_steps > 0) else None

    # the ES-H-FEM step on the same block as 160,000 trilinear hexahedra (fixed topology)
    def hex_leg():
        from cem_inputs import hex_block
        wh = hex_block(200, 80, 10, 0.1, 0.04, 0.01, traction=1e6, name="hex_block_200x80x10")
        out = {"workload": wh.name, "elements": wh.n_elems, "steps": a.hex_steps, "warmup": a.warmup}
        for prec in ("mixed", "fp64"):
            sh = CEM.from_hex_workload(wh, device=dev, precision=prec)
            sh.step(a.warmup)
            barrier()
            sh.profile(max(1, min(PROFILE_EVERY, a.hex_steps // 4)))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sh.step(a.hex_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            t_ms = e0.elapsed_time(e1)
            prof, _ = sh.profile_read()
            out[prec] = {"value": wh.n_elems * a.hex_steps / (t_ms * 1e-3), "unit": "hex-steps/s",
                         "ms_per_step": t_ms / a.hex_steps,
                         "per_launch_us": {k: 1e3 * v[0] / v[1] for k, v in prof.items() if v[1]}}
            sh.close()
        return out

    hexres = _leg("hexahedra", hex_leg) if (a.workload == "block" and a.hex_steps > 0) else None

    # end to end through the public API with host buffers: create + material + K steps + read back
    barrier()
    t0 = time.perf_counter()
    sim2 = CEM(w.X, w.tets, w.tfaces, w.tvec, w.notch_tet, w.notch_side, device=dev,
               split_capacity=a.split_capacity, precision=a.precision)
    t1 = time.perf_counter()
    sim2.set_material(w.rho, w.nu, w.E, w.Gc)
    _reorder(sim2, a)
    t2 = time.perf_counter()
    sim2.step(a.steps)   # default launch variants: the autotuner is not part of a plain run
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    u = sim2.field("u")
    sim2.energy()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e_parts = {"create_s": t1 - t0, "material_s": t2 - t1, "steps_s": t3 - t2, "readback_s": t_e2e - (t3 - t0)}
    sim2.close()
    t_e2e = max_over_ranks(t_e2e, world, "cuda")
    h2d = (w.X.nbytes + w.tets.nbytes + w.tfaces.nbytes + w.tvec.nbytes + w.notch_tet.nbytes
           + w.notch_side.nbytes + 16)
    d2h = u.nbytes + 64

    if rank != 0:
        return
    cpu = None
    if world == 1 and not a.no_cpu_baseline and a.workload == "block":
        cpu = _leg("cpu_baseline", lambda: _cpu_baseline(a.cpu_steps))
    info0, info, energy = main["info0"], main["info"], main["energy"]
    dt = info0["dt"]
    line = {
        "metric": METRIC, "value": main["value"], "unit": METRIC, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": main["t_ms"] / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32/f64 mixed", "data": "synthetic",
        "config": {"workload": WORKLOAD if a.workload == "block" else w.name, "tets": w.n_tets, "nodes": w.n_nodes,
                   "edges": info0["n_edges"], "precision": a.precision, "split": True,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: working set %.2f GB > 129 MB L2 (no flush)"
                         % (info["device_bytes"] / 1e9),
                   "dt_s": dt, "simulated_time_s": {"timed_region": a.steps * dt,
                                                    "end_of_timed_region": (a.warmup + a.steps) * dt},
                   "split_elements_at_end": energy["n_split"], "elements_at_end": info["n_active_tets"],
                   "steps_before_timing": a.warmup},
        "roofline": main["roofline"],
        "active_element_steps_per_s": main["roofline"]["whole_step"]["active_element_steps_per_s"],
        "kernels": main["kernels"],
        "clocks": main["clocks"],
        "e2e": {"value": replica_throughput(w.n_tets, a.steps, world, t_e2e * 1e3), "unit": METRIC,
                "h2d_bytes_per_step": h2d / a.steps, "d2h_bytes_per_step": d2h / a.steps,
                "includes": "mesh upload from host arrays and topology build, material and a_0, K steps "
                            "(default launch variants), u and energy read-back", "parts": e2e_parts},
        "gpu_launches": main["launches"],
        "cpu_baseline": cpu,
        "launch_variants": main["tuning"] if not a.no_autotune else "defaults (autotuner off)",
    }
    if other is not None:
        line[other_prec] = other
    if agree is not None:
        line["precision_agreement"] = agree
    if ens is not None:
        line["ensemble"] = ens
    if graph is not None:
        line["graph"] = graph
    if adj is not None:
        line["adjoint"] = adj
    if hexres is not None:
        line["hexahedra"] = hexres
    if a.workload == "ensemble":
        line["config"]["instances"] = w.params["n_instances"]
        line["config"]["split_capacity"] = a.split_capacity
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    a = _args()
    if a.cpu_baseline_worker:
        v, s, t = _oracle_rate(a.cpu_steps)
        print(json.dumps({"value": v, "steps": s, "seconds": t}))
        return
    if a.cpu_allcore_worker:
        _allcore_worker(a.cpu_steps)
        return
    if a.impl == "reference":
        run_reference(a)
    else:
        run_cem(a)


if __name__ == "__main__":
    main()
