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

if "reference" in sys.argv or "--cpu-baseline-worker" in sys.argv:
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

# DRAM bytes (read + write) per unit measured by ncu for the mixed-precision kernels on the
# 960,000-element block (profiles/mixed_kernels_notched_block_200x80x10.md); scaled by the
# units of an average launch for the roofline's "traffic".  None: no capture of the current
# kernel (FP64 path).
DRAM_BYTES_PER_UNIT = {"mixed": {"strain": 62.6, "edge_stress": 68.0, "force": 126.3, "node_update": 564.5},
                       "fp64": {}}


def kernel_costs(T, E, N, precision):
    """Algorithmic FP64 flops (FMA = 2; FP64 path) and bytes per unit of each hot kernel.

    Bytes are the arrays the kernel reads or writes, each once (gathered
    operands counted once per producer: u per node, h per element, sigma per
    edge, element forces per element).  f = mean fan size 6T/E, g = mean node
    incidence 4T/N.  Mixed precision: FP32 geometry, coefficients and
    intermediate records (h, sigma: 32 B; element forces: 64 B), an FP32
    hi/lo copy of the predicted u (32 B per node), FP64 node state; the node
    update also reads and writes u and writes that copy (the fused predictor).
    """
    f, g = 6.0 * T / E, 4.0 * T / N
    flops = {"predict": 12.0, "strain": 57.0, "edge_stress": 6.0 * f + 13.0, "force": 90.0,
             "node_update": 3.0 * g + 18.0}
    if precision == "fp64":
        byts = {"predict": 96.0,
                "strain": 16 + 72 + 48 + 24.0 * N / T,
                "edge_stress": 8 + 4.0 * f + 16 + 48 + 48.0 * T / E,
                "force": 24 + 72 + 96 + 48.0 * E / T,
                "node_update": 8 + 4.0 * g + 24 + 8 + 96 + 96.0 * T / N}
    else:
        byts = {"predict": 0.0,   # carried by the node update
                "strain": 16 + 36 + 32 + 32.0 * N / T,
                "edge_stress": 8 + 4.0 * f + 8 + 32 + 32.0 * T / E,
                "force": 24 + 36 + 64 + 32.0 * E / T,
                "node_update": 8 + 4.0 * g + 24 + 8 + 96 + 80 + 64.0 * T / N}
    return flops, byts


def roofline_accounting(chunks, prof, precision, scale, t_ms, hbm, sm_clock):
    """Per-kernel shares and the dominant step kernel's roofline from sampled kernel times.

    chunks: [(counts, {kernel: (ms, launches)})] for consecutive windows of the timed
    region; counts holds the window's mean n_active_tets, n_edges and n_nodes, and the
    dict the sampled launches' time and number in that window.  prof: {kernel:
    (total ms, launches)} over the whole region; scale = timed steps / sampled steps;
    t_ms the region's time.  The algorithmic bytes (flops) of a sampled launch are the
    per-unit figures of kernel_costs for its window's sizes times its units, so a mesh
    that grows during the run is accounted window by window.  Achieved = the dominant
    kernel's bytes (flops) per launch / its mean launch time; it is FP64-ALU-bound when
    its flops take longer at the FP64 peak than its bytes at the HBM peak (FP64 path only).
    """
    acc = {k: dict(bytes=0.0, flops=0.0, units=0.0, traffic=0.0) for k in KERNEL_UNITS}
    per_unit = DRAM_BYTES_PER_UNIT.get(precision, {})
    for cnt, dp in chunks:
        fl, by = kernel_costs(cnt["n_active_tets"], cnt["n_edges"], cnt["n_nodes"], precision)
        for k, (_, nl) in dp.items():
            units = {"tets": cnt["n_active_tets"], "edges": cnt["n_edges"], "nodes": cnt["n_nodes"]}[KERNEL_UNITS[k]]
            acc[k]["bytes"] += nl * by[k] * units
            acc[k]["flops"] += nl * fl[k] * units
            acc[k]["units"] += nl * units
            acc[k]["traffic"] += nl * per_unit.get(k, 0.0) * units
    kernels = {}
    for k, (ms_tot, nl) in prof.items():
        kernels[k] = {"ms": ms_tot * scale, "launches_timed": nl, "share": ms_tot * scale / max(t_ms, 1e-9)}
        if k in KERNEL_UNITS and nl:
            sec = ms_tot * 1e-3
            kernels[k].update(per_launch_us=sec / nl * 1e6, gbs=acc[k]["bytes"] / sec / 1e9)
            if precision == "fp64":
                kernels[k]["fp64_tflops"] = acc[k]["flops"] / sec / 1e12
    fp64_peak = 152 * 4 * sm_clock * 1e6      # 152 SMs x 2 FP64 FMA/clk x 2 FLOP
    hot = {k: prof[k] for k in KERNEL_UNITS}
    dom = max(hot, key=lambda k: hot[k][0])
    ms_tot, nl = hot[dom]
    nl = max(nl, 1)
    per_launch_s = ms_tot * 1e-3 / nl
    units = acc[dom]["units"] / nl
    flops, bytes_ = acc[dom]["flops"] / nl, acc[dom]["bytes"] / nl
    alu_bound = precision == "fp64" and flops / fp64_peak > bytes_ / ((hbm or 6651.4) * 1e9)
    if alu_bound:
        achieved, peak, unit = flops / per_launch_s / 1e12, fp64_peak / 1e12, "TFLOP/s"
        src = "derived: 152 SMs x 4 FP64 FLOP/clk x %.0f MHz (nominal 1.25 TFLOP/s at 2070 MHz)" % sm_clock
    else:
        achieved, peak, unit = bytes_ / per_launch_s / 1e9, hbm, "GB/s"
        src = "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"
    traffic = acc[dom]["traffic"] / nl if dom in per_unit else None
    roofline = {"bound": "alu" if alu_bound else "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "unit": unit, "frac": achieved / peak if peak else None, "traffic": traffic, "peak_source": src,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per unit on the 960,000-"
                                   "element block, scaled to the units of each sampled launch" if traffic
                                   else None),
                "per_launch_us": per_launch_s * 1e6, "algorithmic_bytes_per_launch": bytes_,
                "algorithmic_flops_per_launch": flops,
                "hbm_gbs_achieved": bytes_ / per_launch_s / 1e9, "hbm_peak_gbs": hbm,
                "units_per_launch": units, "units_integrated_over": "%d chunks of <= %d steps" % (
                    len(chunks), CHUNK_STEPS)}
    return kernels, roofline


# --------------------------------------------------------------------------- helpers
def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=19995)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["cem", "reference"], default="cem")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
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
    p.add_argument("--cpu-steps", type=int, default=80, help=argparse.SUPPRESS)
    return p.parse_args()


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


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


def _cpu_baseline(steps):
    """Run the oracle in a single-threaded subprocess; returns the cpu_baseline object."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker", "--cpu-steps", str(steps)]
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": res["value"], "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": "%s, steps 2-%d of the run (%.1f s of CPU time; setup untimed), "
                      "single-threaded numpy/scipy FP64 oracle" % (WORKLOAD, res["steps"] + 1, res["seconds"]),
            "host": _host_cpu()}


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
    hbm = peaks.get("hbm_gbs")
    fp64_peak_meas = probe_fp64_fma(dev, stream.cuda_stream)

    def timed(precision, clocks_on, w=w, steps=None, split_capacity=None):
        """W untimed then K timed steps of a fresh context: metrics of the timed region."""
        steps = a.steps if steps is None else steps
        cap = a.split_capacity if split_capacity is None else split_capacity
        sim = CEM.from_workload(w, device=dev, split_capacity=cap, precision=precision)
        _reorder(sim, a)
        info0 = sim.info()
        if not a.no_autotune:   # launch variants for the current sizes; re-tuned in the run as the mesh grows
            sim.autotune(reps=10, automatic=True)
        sim.step(a.warmup)
        barrier()
        clocks = ClockSampler(_bus_id(dev)) if (clocks_on and rank == 0) else None
        sim.profile(max(1, min(PROFILE_EVERY, steps // 4)))   # at least a few sampled steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # The mesh grows during the run, so the sampled launches' units (elements, edges, nodes)
        # are integrated chunk by chunk: each chunk's sampled kernel time is paired with the mean
        # of its first and last counts.  The counts and timing sums are read on the host between
        # chunks; every step already ends with a host read of its split count.
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
            chunks.append(({u: (c_prev[u] + c_now[u]) / 2.0 for u in ("n_active_tets", "n_edges", "n_nodes")},
                           {k: (p_now[k][0] - p_prev[k][0], p_now[k][1] - p_prev[k][1]) for k in KERNEL_UNITS}))
            c_prev, p_prev = c_now, {k: p_now[k] for k in KERNEL_UNITS}
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms = e0.elapsed_time(e1)
        clk = clocks.stop() if clocks else None
        prof, launches = sim.profile_read()
        sim.profile(0)
        barrier()
        t_ms = max_over_ranks(t_ms, world, "cuda")
        info = sim.info()
        energy = sim.energy()
        tuning = {k: {"block": v[0], "batch": v[1]} for k, v in sim.tuning().items()}
        sim.close()
        sm_clock = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
        fp64_peak = 152 * 4 * sm_clock * 1e6      # 152 SMs x 2 FP64 FMA/clk x 2 FLOP
        # timed launches are a sample (every PROFILE_EVERY-th step): scale sums to the whole region
        n_sampled = max(prof["strain"][1], 1)
        if prof["strain"][1] == 0:
            raise RuntimeError("no sampled step in the timed region")
        scale = steps / n_sampled
        kernels, roofline = roofline_accounting(chunks, prof, precision, scale, t_ms, hbm, sm_clock)
        flops, per_launch_s = roofline["algorithmic_flops_per_launch"], roofline["per_launch_us"] * 1e-6
        if precision == "fp64":
            roofline.update(fp64_tflops_achieved=flops / per_launch_s / 1e12, fp64_peak_tflops=fp64_peak / 1e12,
                            fp64_fma_measured_tflops=fp64_peak_meas / 1e12)
        else:
            del roofline["algorithmic_flops_per_launch"]
        return dict(t_ms=t_ms, value=replica_throughput(w.n_tets, steps, world, t_ms), roofline=roofline,
                    kernels=kernels,
                    clocks=clk, launches=launches, info0=info0, info=info, energy=energy, steps=steps,
                    tuning=tuning)

    main = timed(a.precision, True)
    other = None
    if not a.no_compare:
        other = timed("fp64" if a.precision == "mixed" else "mixed", False)

    # agreement of the two precisions on a short window (both paths from the same start)
    agree = None
    if not a.no_compare and a.workload == "block":
        n_cmp = 500
        s64 = CEM.from_workload(w, device=dev, split_capacity=a.split_capacity, precision="fp64")
        s32 = CEM.from_workload(w, device=dev, split_capacity=a.split_capacity, precision="mixed")
        s64.step(n_cmp)
        s32.step(n_cmp)
        u64, u32 = s64.field("u"), s32.field("u")
        c64 = {(r[0], r[3]) for r in s64.crack_state()}
        c32 = {(r[0], r[3]) for r in s32.crack_state()}
        rel = (float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64)) if u32.shape == u64.shape else None)
        agree = {"steps": n_cmp, "rel_l2_u_mixed_vs_fp64": rel,
                 "split_jaccard": len(c64 & c32) / max(len(c64 | c32), 1), "splits_fp64": len(c64)}
        s64.close()
        s32.close()

    # the 256-specimen ensemble as one union mesh, mixed against FP64 (default block mode only)
    ens = None
    if a.workload == "block" and a.ensemble_steps > 0:
        we = _workload("ensemble")
        em = timed("mixed", False, w=we, steps=a.ensemble_steps, split_capacity=we.n_tets // 4)
        ef = timed("fp64", False, w=we, steps=a.ensemble_steps, split_capacity=we.n_tets // 4)
        ens = {"workload": we.name, "instances": we.params["n_instances"], "tets": we.n_tets,
               "steps": a.ensemble_steps, "warmup": a.warmup,
               "mixed": {"value": em["value"], "ms_per_step": em["t_ms"] / a.ensemble_steps,
                         "roofline": {k: em["roofline"][k] for k in ("bound", "kernel", "achieved", "peak", "unit",
                                                                     "frac")}},
               "fp64": {"value": ef["value"], "ms_per_step": ef["t_ms"] / a.ensemble_steps},
               "mixed_speedup_over_fp64": em["value"] / ef["value"],
               "split_elements_at_end_mixed": em["energy"]["n_split"]}
        del we

    # gradients: FP32 forward + adjoint with sqrt(N) checkpoints on the 102,000-element block,
    # J = final strain energy + mean top-face y displacement, topology frozen after the notch
    adj = None
    if a.workload == "block" and a.adjoint_steps > 0:
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
        adj = {"workload": wa.name, "tets": wa.n_tets, "steps": a.adjoint_steps,
               "checkpoint_every": int(np.ceil(np.sqrt(a.adjoint_steps))),
               "mixed": {"seconds": tm, "tet_steps_per_s": wa.n_tets * a.adjoint_steps / tm},
               "fp64": {"seconds": tf, "tet_steps_per_s": wa.n_tets * a.adjoint_steps / tf},
               "rel_err_J_mixed": abs(Jm - Jf) / abs(Jf),
               "rel_err_dJdE_mixed": float(np.abs(dEm - dEf).max() / np.abs(dEf).max()),
               "rel_err_dJdalpha_mixed": abs(dam - daf) / abs(daf),
               "note": "wall time of one cem_adjoint call: forward, segment recompute and reverse sweep"}
        del wa

    # the ES-H-FEM step on the same block as 160,000 trilinear hexahedra (fixed topology)
    hexres = None
    if a.workload == "block" and a.hex_steps > 0:
        from cem_inputs import hex_block
        wh = hex_block(200, 80, 10, 0.1, 0.04, 0.01, traction=1e6, name="hex_block_200x80x10")
        hexres = {"workload": wh.name, "elements": wh.n_elems, "steps": a.hex_steps, "warmup": a.warmup}
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
            hexres[prec] = {"value": wh.n_elems * a.hex_steps / (t_ms * 1e-3), "unit": "hex-steps/s",
                            "ms_per_step": t_ms / a.hex_steps,
                            "per_launch_us": {k: 1e3 * v[0] / v[1] for k, v in prof.items() if v[1]}}
            sh.close()
        del wh

    # end to end through the public API with host buffers: create + material + K steps + read back
    barrier()
    t0 = time.perf_counter()
    sim2 = CEM.from_workload(w, device=dev, split_capacity=a.split_capacity, precision=a.precision)
    _reorder(sim2, a)
    if not a.no_autotune:
        sim2.autotune(reps=10, automatic=True)
    sim2.step(a.steps)
    u = sim2.field("u")
    sim2.energy()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    sim2.close()
    t_e2e = max_over_ranks(t_e2e, world, "cuda")
    h2d = (w.X.nbytes + w.tets.nbytes + w.tfaces.nbytes + w.tvec.nbytes + w.notch_tet.nbytes
           + w.notch_side.nbytes + 16)
    d2h = u.nbytes + 64

    if rank != 0:
        return
    cpu = None
    if world == 1 and not a.no_cpu_baseline and a.workload == "block":
        try:
            cpu = _cpu_baseline(a.cpu_steps)
        except Exception as ex:  # reported, not hidden
            cpu = {"value": None, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": "failed: %r" % (ex,)}
    info0, info, energy = main["info0"], main["info"], main["energy"]
    line = {
        "metric": METRIC, "value": main["value"], "unit": METRIC, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": main["t_ms"] / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/f64 mixed" if a.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "tets": w.n_tets, "nodes": w.n_nodes, "edges": info0["n_edges"],
                   "precision": a.precision, "split": True,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "working set %.2f GB > 129 MB L2 (no flush needed)" % (info["device_bytes"] / 1e9),
                   "split_elements_at_end": energy["n_split"], "elements_at_end": info["n_active_tets"],
                   "steps_before_timing": a.warmup},
        "roofline": main["roofline"],
        "kernels": main["kernels"],
        "clocks": main["clocks"],
        "e2e": {"value": replica_throughput(w.n_tets, a.steps, world, t_e2e * 1e3), "unit": METRIC,
                "h2d_bytes_per_step": h2d / a.steps, "d2h_bytes_per_step": d2h / a.steps,
                "includes": "mesh upload and topology build, material, K steps, u and energy read-back"},
        "gpu_launches": main["launches"],
        "cpu_baseline": cpu,
        "launch_variants": main["tuning"] if not a.no_autotune else "defaults (autotuner off)",
    }
    if other is not None:
        line["fp64" if a.precision == "mixed" else "mixed"] = {
            "value": other["value"], "ms_per_step": other["t_ms"] / a.steps, "roofline": other["roofline"],
            "kernels": {k: {kk: v[kk] for kk in ("ms", "share", "per_launch_us") if kk in v}
                        for k, v in other["kernels"].items()},
            "gpu_launches": other["launches"], "speedup_of_main": main["value"] / other["value"]}
    if agree is not None:
        line["precision_agreement"] = agree
    if ens is not None:
        line["ensemble"] = ens
    if adj is not None:
        line["adjoint"] = adj
    if hexres is not None:
        line["hexahedra"] = hexres
    if a.workload == "ensemble":
        line["config"]["workload"] = w.name
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
    if a.impl == "reference":
        run_reference(a)
    else:
        run_cem(a)


if __name__ == "__main__":
    main()
