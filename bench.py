#!/usr/bin/env python
"""Benchmark of the TREVR hot path on GB300: sink fluxes per second.

One step = build the radiation tree from the particles (keys, sort, topology,
source deposit, cell moments) + the flux at every sink (source walk, reverse
rays with tau_ref refinement, flux sum), on inputs already resident in HBM.

Prints one JSON line (rank 0). The default workload is the clumpy medium: 2^22
gas particles with a lognormal absorption field (sigma_ln = 2, correlation
length 0.05) and a x1e3 cube occluder, 2^14 sources in 16 Gaussian clumps,
theta_open = 0.6, tau_ref = 0.1, bucket 8. The roofline of the sink walk is its
instruction issue rate against the SMs' issue limit (the walk is issue-bound,
with cell records served from L1/L2); the logical bytes of cell records it
reads per second are reported beside it. cpu_baseline is the FP64 oracle on the
host cores, on a seeded sample of sinks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload clumpy|stromgren|uniform]
    python bench.py --impl reference ...   # the FP64 CPU oracle as the reference arm
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "sink fluxes/s"
UNIT = "fluxes/s"
L2_BYTES = 129 * 1024 * 1024


def _problem(name, seed_offset=0):
    if name == "clumpy":
        P = workloads.clumpy(seed=2 + seed_offset)
        desc = "clumpy lognormal medium (sigma_ln=2, corr 0.05) + x1e3 cube occluder"
    elif name == "stromgren":
        P = workloads.stromgren(seed=1 + seed_offset)
        desc = "Stromgren-like: one L=1 source at the centre, uniform alpha=20"
    elif name == "uniform":
        P = workloads.uniform_box(seed=0 + seed_offset)
        desc = "uniform box, 4096 gas / 64 sources, alpha=1"
    else:
        raise SystemExit(f"unknown workload {name}")
    return P, desc


def _config(P, name, desc):
    return {"workload": f"{name}: {desc}", "n_gas": int(P["gas_xyz"].shape[1]),
            "n_src": int(P["src_xyz"].shape[1]), "theta_open": P["theta"],
            "tau_ref": P["tau_ref"], "bucket": P["bucket"], "seed": P["seed"],
            "l2": "flushed between timed steps (256 MiB write)"}


def reduce_max(value, world, device):
    """Max of a per-rank scalar over all ranks (the step time of the slowest rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, t_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (t_ms * 1e-3)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, keep_dir=None):
        """keep_dir: also keep the raw samples there as clocks_rank<i>.csv."""
        import tempfile
        self.idx = gpu_index
        self.proc = None
        self.keep = (None if not keep_dir else
                     os.path.join(keep_dir, f"clocks_rank{gpu_index}.csv"))
        fd, self.path = tempfile.mkstemp(prefix="trevr_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            if os.path.exists(self.path):
                os.remove(self.path)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if self.keep:
            os.makedirs(os.path.dirname(os.path.abspath(self.keep)), exist_ok=True)
            shutil.copyfile(self.path, self.keep)
        os.remove(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _kernel_profile(name):
    """Per-sink counters of one kernel from a committed ncu capture
    (profiles/<name>): warp instructions issued, thread instructions executed, DRAM
    bytes, and the cell steps of the captured sinks. None if the kernel's source has
    changed since the capture (the counters would describe another kernel)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", name)
    try:
        d = json.load(open(p))
        src = open(os.path.join(ROOT, d["source"]), "rb").read()
    except (OSError, ValueError, KeyError):
        return None
    if hashlib.sha256(src).hexdigest() != d["source_sha256"]:
        return None
    d["file"] = name
    return d


def _issue_roofline(prof, sinks, t_s, sm_mhz, n_sm, alg_bytes, peak_gbs, peak_kind, kernel):
    """Roofline of an issue-bound walk. achieved = warp instructions issued per launch
    (the capture's per-sink count times the launch's sinks) over the event-timed
    launch; peak = 4 schedulers x n_sm SMs x 1 warp instruction per cycle at the SM
    clock sampled during the timed region. The logical bytes of cell records per
    second stay beside it as a secondary figure against the HBM copy bandwidth."""
    logical = {"achieved": alg_bytes / t_s / 1e9, "peak": peak_gbs, "unit": "GB/s",
               "frac": alg_bytes / t_s / 1e9 / peak_gbs, "bytes_per_launch": alg_bytes,
               "peak_kind": f"{peak_kind} (copy bandwidth)",
               "note": "logical cell-record reads, mostly L1/L2 hits"}
    peak = 4 * n_sm * sm_mhz * 1e6 / 1e9
    if prof is None:
        return {"bound": "issue", "achieved": None, "peak": peak,
                "unit": "G warp-instructions/s", "frac": None, "traffic": None,
                "kernel": kernel, "stale": "kernel source changed since the ncu capture",
                "logical_bytes": logical}
    per_sink = prof["warp_inst_issued"] / prof["sinks"]
    achieved = per_sink * sinks / t_s / 1e9
    steps = prof["cells_tested"] + prof["cells_clipped"]
    return {"bound": "issue", "achieved": achieved, "peak": peak,
            "unit": "G warp-instructions/s", "frac": achieved / peak,
            "traffic": prof["dram_bytes_per_sink"] * sinks, "kernel": kernel,
            "peak_kind": f"issue limit: 4 schedulers x {n_sm} SMs x 1 warp-instruction/cycle "
                         f"at {sm_mhz:.0f} MHz (SM clock sampled under load)",
            "instructions_per_launch": per_sink * sinks,
            "thread_instructions_per_cell_step": prof["thread_inst_executed"] / steps,
            "active_lanes_per_instruction": prof["thread_inst_executed"] /
                                            prof["warp_inst_issued"],
            "counters_from": f"profiles/{prof['file']} ({prof['sinks']} sinks, ncu)",
            "logical_bytes": logical}


def _peaks_clock():
    """Maximum SM clock (MHz) from MEASURED_PEAKS.json, else the GB300's 2070 MHz."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("sm_max_mhz", 2070.0))
    return 2070.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _cpu_model():
    """The host CPU's model name (lscpu), or the platform's description."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _oracle_baseline(P, n_gas, sample_n, seconds, seed=7):
    """Time the FP64 oracle as it stands on the host cores on a bounded sample: the
    full tree build, the flux at `sample_n` seeded sinks (also the parity sample),
    then the flux at as many further seeded sinks as take about `seconds` of walking,
    the timed sample. Returns (info, parity sinks, their flux, tree)."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    T = oracle.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], lo=P["lo"],
                          side=P["side"], bucket=P["bucket"])
    t_build = time.perf_counter() - t0
    sinks = workloads.sink_sample(n_gas, sample_n, seed=seed)
    t0 = time.perf_counter()
    f = T.flux(P["theta"], P["tau_ref"], sinks=sinks, nthreads=cores)
    t_pilot = time.perf_counter() - t0
    m = int(min(n_gas, max(len(sinks), seconds * len(sinks) / max(t_pilot, 1e-6))))
    timed = workloads.sink_sample(n_gas, m, seed=seed + 1)
    t0 = time.perf_counter()
    T.flux(P["theta"], P["tau_ref"], sinks=timed, nthreads=cores)
    t_walk = time.perf_counter() - t0
    # build time is charged in proportion to the sample's share of the sinks
    per_sink = t_walk / m + t_build / n_gas
    info = {"value": 1.0 / per_sink, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": _cpu_model(),
            "sample": f"{m} of {n_gas} sinks walked (seeded) + the full {n_gas}-particle "
                      f"tree build charged pro rata; walk {t_walk:.2f} s, build {t_build:.2f} s",
            "walk_s": t_walk, "build_s": t_build}
    return info, sinks, f, T


def run_reference(args):
    rank, world, _ = _dist()
    if world > 1 and rank != 0:
        return
    P, desc = _problem(args.workload)
    n = int(P["gas_xyz"].shape[1])
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    T = oracle.OracleTree(P["gas_xyz"], P["alpha"], P["src_xyz"], P["src_lum"], lo=P["lo"],
                          side=P["side"], bucket=P["bucket"])
    t_build = time.perf_counter() - t0
    # each step walks a seeded sample sized from a pilot so that the whole run takes
    # about --ref-seconds of walking
    pilot = workloads.sink_sample(n, min(n, 1024), seed=99)
    t0 = time.perf_counter()
    T.flux(P["theta"], P["tau_ref"], sinks=pilot, nthreads=cores)
    per = (time.perf_counter() - t0) / len(pilot)
    sample_n = int(min(n, max(256, args.ref_seconds / (args.warmup + args.steps) / per)))
    times = []
    for step in range(args.warmup + args.steps):
        sinks = workloads.sink_sample(n, sample_n, seed=100 + step)
        t0 = time.perf_counter()
        T.flux(P["theta"], P["tau_ref"], sinks=sinks, nthreads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt + t_build * sample_n / n)
    per_step = sum(times) / len(times)
    value = sample_n / per_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(P, args.workload, desc),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "cpu": _cpu_model(),
                             "value": value, "unit": UNIT,
                             "sample": f"each step walks {sample_n} seeded sinks of {n}; the "
                                       f"{n}-particle tree build ({t_build:.2f} s, once) is "
                                       f"charged pro rata"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _time_ms(fn, reps, stream):
    import torch
    out = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def _bench_batched(args, sm_mhz):
    """64 independent boxes (2^12..2^17 particles, log-uniform): one persistent launch
    replayed from a CUDA graph, launch shape from the autotuner, vs 64 plain calls."""
    import torch
    from paper_1902_08083_gb300 import autotune, trevr
    boxes = workloads.batched_boxes()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    trees = []
    for P in boxes:
        g = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev)
             for k in ("gas_xyz", "alpha", "src_xyz", "src_lum")}
        trees.append(trevr.build_tree(g["gas_xyz"], g["alpha"], g["src_xyz"], g["src_lum"],
                                      lo=P["lo"], side=P["side"], bucket=P["bucket"]))
    th, tr = boxes[0]["theta"], boxes[0]["tau_ref"]
    B = trevr.Batch(trees)
    tune = autotune.tune(B, th, tr)
    shape = dict(sinks_per_warp=tune["sinks_per_warp"], block_size=tune["block_size"],
                 walk_variant=tune.get("walk_variant", 0))
    st = B.run(th, tr, stats=True, **shape)  # counters (untimed) for the roofline
    B.capture(th, tr, **shape)
    for _ in range(args.warmup):
        B.replay()
    t_graph = _time_ms(B.replay, args.steps, stream)
    outs = [torch.empty(t.n_gas, device=dev) for t in trees]

    def sequential():
        for t, o in zip(trees, outs):
            trevr.compute_flux(t, th, tr, out=o)
    sequential()
    t_seq = _time_ms(sequential, args.steps, stream)
    same = all(torch.equal(a, b) for a, b in zip(B.flux, outs))
    n = B.n_sinks
    t_rep = sum(t_graph) / len(t_graph) * 1e-3
    alg_bytes = 20 * n + 32 * st["src_nodes_visited"] + 32 * st["cells_clipped"]
    peak, peak_kind = _peaks()
    dev_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    prof = _kernel_profile("walk_warp_batched_kernel_issue.json")
    if prof is not None and prof.get("launch_shape", {}).get("walk_variant") != \
            shape.get("walk_variant"):
        prof = None  # the capture was of another walk variant
    res = {"workload": f"{len(trees)} boxes, {n} sinks (2^12..2^17 each), theta 0.75, tau_ref 0.1",
           "graph_fluxes_per_s": n / (min(t_graph) * 1e-3),
           "sequential_fluxes_per_s": n / (min(t_seq) * 1e-3),
           "speedup": min(t_seq) / min(t_graph), "bit_equal_to_sequential": bool(same),
           "launch_shape": shape, "tuned_from_cache": bool(tune.get("cached")),
           "per_sink": {"interactions": st["interactions"] / n, "segments": st["segments"] / n,
                        "cells_visited": st["src_nodes_visited"] / n,
                        "cells_clipped": st["cells_clipped"] / n},
           "roofline": _issue_roofline(prof, n, t_rep, sm_mhz, dev_sm, alg_bytes, peak,
                                       peak_kind, "walk_warp_batched_kernel (persistent, "
                                       "graph replay)")}
    if prof is not None:
        res["roofline"]["captured_launch_shape"] = prof.get("launch_shape")
    B.free()
    for t in trees:
        t.free()
    return res


def _bench_adjoint(args):
    """Forward + adjoint on 2^21 particles / 1024 sources (lognormal sigma_ln=1),
    loss sum_p w_p log F_p over every sink."""
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.adjoint_problem()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    g = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev)
         for k in ("gas_xyz", "alpha", "src_xyz", "src_lum")}
    tree = trevr.build_tree(g["gas_xyz"], g["alpha"], g["src_xyz"], g["src_lum"], lo=P["lo"],
                            side=P["side"], bucket=P["bucket"])
    n = tree.n_gas
    w = torch.from_numpy(P["loss_weight"]).to(dev)
    F = trevr.compute_flux(tree, P["theta"], P["tau_ref"])
    gflux = (w / F).contiguous()
    fwd = _time_ms(lambda: trevr.compute_flux(tree, P["theta"], P["tau_ref"], out=F),
                   args.steps, stream)
    bwd = _time_ms(lambda: trevr.compute_flux_backward(tree, gflux, P["theta"], P["tau_ref"]),
                   args.steps, stream)
    tree.free()
    return {"workload": f"{n} gas, {P['src_xyz'].shape[1]} sources, lognormal sigma_ln=1",
            "forward_ms": min(fwd), "backward_ms": min(bwd),
            "backward_sinks_per_s": n / (min(bwd) * 1e-3)}


def _bench_termination(args, P, g):
    """Early ray termination (Sec. 4) on an optically thick copy of the workload: the
    same particles and sources with every absorption coefficient x16. Times the walk
    with and without tau_stop = 10 and checks the bound 0 <= F - F_stop <=
    exp(-tau_stop) F(alpha = 0) at every sink."""
    import torch
    from paper_1902_08083_gb300 import trevr
    stream = torch.cuda.current_stream()
    tau_stop = 10.0
    thick = (g["alpha"] * 16.0).contiguous()
    zero = torch.zeros_like(g["alpha"])
    kw = dict(lo=P["lo"], side=P["side"], bucket=P["bucket"])
    tree = trevr.build_tree(g["gas_xyz"], thick, g["src_xyz"], g["src_lum"], **kw)
    tree0 = trevr.build_tree(g["gas_xyz"], zero, g["src_xyz"], g["src_lum"], **kw)
    F = trevr.compute_flux(tree, P["theta"], P["tau_ref"])
    Fs, st = trevr.compute_flux(tree, P["theta"], P["tau_ref"], tau_stop=tau_stop, stats=True)
    F0 = trevr.compute_flux(tree0, P["theta"], P["tau_ref"])
    plain = _time_ms(lambda: trevr.compute_flux(tree, P["theta"], P["tau_ref"], out=F),
                     args.steps, stream)
    stop = _time_ms(lambda: trevr.compute_flux(tree, P["theta"], P["tau_ref"], out=Fs,
                                               tau_stop=tau_stop), args.steps, stream)
    d = F.double() - Fs.double()
    bound = float(np.exp(-tau_stop)) * F0.double()
    # fp32 rounding of the two sums: a relative 1e-5 of F beside the bound
    ok = bool(torch.all(d >= -1e-5 * F.double()) and torch.all(d <= bound * 1.01 + 1e-5 * F))
    rel = d.abs() / F.double().clamp_min(1e-30)
    tree.free()
    tree0.free()
    return {"workload": f"{P['gas_xyz'].shape[1]} gas, {P['src_xyz'].shape[1]} sources, "
                        f"alpha x16", "tau_stop": tau_stop,
            "walk_ms": min(plain), "walk_ms_terminated": min(stop),
            "speedup": min(plain) / min(stop),
            "rays_terminated_frac": st["rays_terminated"] / max(st["interactions"], 1),
            "median_rel_change": float(rel.median()), "bound_holds": ok}


def _bench_topdown(args, P, g):
    """The top-down ray walk (ray_walk = 1; Sec. 3.1.3, Sec. 4) against the paper's
    bottom-up walk on the workload and on an optically thin copy (every absorption
    coefficient / 16): the walk times (no counters), segments and cells clipped per
    sink, and each walk's RMS and largest fractional error against full refinement
    (tau_ref = 0, where both walks sum the same leaves) on 65536 seeded sinks."""
    import torch
    from paper_1902_08083_gb300 import trevr
    stream = torch.cuda.current_stream()
    n = int(P["gas_xyz"].shape[1])
    sample = torch.from_numpy(workloads.sink_sample(n, 1 << 16, seed=21)).to(g["alpha"].device)
    kw = dict(lo=P["lo"], side=P["side"], bucket=P["bucket"])
    th, tr = P["theta"], P["tau_ref"]
    res = {"sample_sinks": 1 << 16}
    for name, scale in (("workload", 1.0), ("thin_alpha_over_16", 1.0 / 16.0)):
        alpha = (g["alpha"] * scale).contiguous()
        tree = trevr.build_tree(g["gas_xyz"], alpha, g["src_xyz"], g["src_lum"], **kw)
        ref = trevr.compute_flux(tree, th, 0.0, sink_idx=sample).double()
        out = {}
        for walk, rw in (("bottom_up", 0), ("top_down", 1)):
            F, st = trevr.compute_flux(tree, th, tr, stats=True, ray_walk=rw)
            ms = _time_ms(lambda: trevr.compute_flux(tree, th, tr, out=F, ray_walk=rw),
                          args.steps, stream)
            e = (F[sample].double() - ref) / ref
            out[walk] = {"walk_ms": min(ms), "segments_per_sink": st["segments"] / n,
                         "cells_clipped_per_sink": st["cells_clipped"] / n,
                         "rms_error_vs_full_refinement": float(torch.sqrt(torch.mean(e * e))),
                         "max_error_vs_full_refinement": float(e.abs().max())}
        out["speedup"] = out["bottom_up"]["walk_ms"] / out["top_down"]["walk_ms"]
        res[name] = out
        tree.free()
    return res


def _bench_bands(args, P, g):
    """Four bands on the workload's particles and sources (absorption x1, x1/2, x1/4, x2;
    luminosity factors 1/2, 1/4, 1/8, 1/8): the band walk against the single-band walk
    of band 0 (Sec. 4 expects a small constant factor)."""
    import torch
    from paper_1902_08083_gb300 import trevr
    stream = torch.cuda.current_stream()
    fa = torch.tensor([1.0, 0.5, 0.25, 2.0], device=g["alpha"].device)
    fl = torch.tensor([0.5, 0.25, 0.125, 0.125], device=g["alpha"].device)
    A = (fa[:, None] * g["alpha"][None, :]).contiguous()
    L = (fl[:, None] * g["src_lum"][None, :]).contiguous()
    kw = dict(lo=P["lo"], side=P["side"], bucket=P["bucket"])
    tb = trevr.build_tree(g["gas_xyz"], A, g["src_xyz"], L, **kw)
    t1 = trevr.build_tree(g["gas_xyz"], g["alpha"], g["src_xyz"], g["src_lum"], **kw)
    Fb, st = trevr.compute_flux_bands(tb, P["theta"], P["tau_ref"], stats=True)
    F1, st1 = trevr.compute_flux(t1, P["theta"], P["tau_ref"], stats=True)
    multi = _time_ms(lambda: trevr.compute_flux_bands(tb, P["theta"], P["tau_ref"], out=Fb),
                     args.steps, stream)
    single = _time_ms(lambda: trevr.compute_flux(t1, P["theta"], P["tau_ref"], out=F1),
                      args.steps, stream)
    tb.free()
    t1.free()
    return {"workload": f"{P['gas_xyz'].shape[1]} gas, {P['src_xyz'].shape[1]} sources, "
                        "4 bands", "walk_ms_4_bands": min(multi),
            "walk_ms_1_band": min(single), "cost_ratio": min(multi) / min(single),
            "segments_ratio": st["segments"] / max(st1["segments"], 1)}


def _bench_sub_bucket(args):
    """Sub-bucket particle trace (Sec. 2.2.3, 3.1.3) on 2^18 particles of equal volume
    with a lognormal absorption field (sigma_ln=1.5) and 32-neighbour smoothing
    lengths, 1024 sources: the neighbour-list build and the walk with and without
    the trace."""
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.sub_bucket_problem(n_gas=1 << 18, n_src=1024, seed=12)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    t = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev)
         for k in ("gas_xyz", "alpha", "src_xyz", "src_lum", "weight", "hsml")}
    tree = trevr.build_tree(t["gas_xyz"], t["alpha"], t["src_xyz"], t["src_lum"],
                            weight=t["weight"], lo=P["lo"], side=P["side"], bucket=P["bucket"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tree.set_smoothing(t["hsml"])
    e1.record(stream)
    torch.cuda.synchronize()
    nbr_ms = e0.elapsed_time(e1)
    F, st = trevr.compute_flux(tree, P["theta"], P["tau_ref"], sub_bucket=1, stats=True)
    F0 = trevr.compute_flux(tree, P["theta"], P["tau_ref"])
    sub = _time_ms(lambda: trevr.compute_flux(tree, P["theta"], P["tau_ref"], out=F,
                                              sub_bucket=1), args.steps, stream)
    plain = _time_ms(lambda: trevr.compute_flux(tree, P["theta"], P["tau_ref"], out=F0),
                     args.steps, stream)
    rel = ((F.double() - F0.double()).abs() / F0.double().clamp_min(1e-30))
    tree.free()
    return {"workload": f"{P['gas_xyz'].shape[1]} gas, {P['src_xyz'].shape[1]} sources, "
                        "lognormal sigma_ln=1.5, 32-neighbour smoothing",
            "theta": P["theta"], "tau_ref": P["tau_ref"], "neighbour_lists_ms": nbr_ms,
            "walk_ms_sub_bucket": min(sub), "walk_ms_cell_means": min(plain),
            "sub_bucket_segments_frac": st["sub_bucket_segments"] / max(st["segments"], 1),
            "median_rel_change": float(rel.median())}


def _bench_glass(args):
    """The perturbed-glass stand-in at the paper's size (64^3 gas, 64^3 stars;
    Sec. 3.1, Appendix A): rays and segments per element and the RMS flux error
    against theta = 0 (512 seeded sinks) and against tau_ref = 1e-8 (every sink),
    beside the values the paper prints for its glass (Sec. 3.1.2, 3.1.3)."""
    import torch
    from paper_1902_08083_gb300 import trevr
    P = workloads.perturbed_glass(64)
    dev = torch.device("cuda", torch.cuda.current_device())
    t = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev)
         for k in ("gas_xyz", "alpha", "src_xyz", "src_lum", "weight")}
    tree = trevr.build_tree(t["gas_xyz"], t["alpha"], t["src_xyz"], t["src_lum"],
                            weight=t["weight"], lo=P["lo"], side=P["side"], bucket=P["bucket"])
    n = tree.n_gas
    sinks = torch.from_numpy(workloads.sink_sample(n, 512, seed=16)).to(dev)

    def rms(f, ref):
        return float(torch.sqrt(torch.mean(((f.double() - ref.double()) / ref.double()) ** 2)))

    f0 = trevr.compute_flux(tree, 0.0, 0.1, sink_idx=sinks)
    theta = {}
    for th in (0.45, 0.6, 0.75, 1.0):
        f, st = trevr.compute_flux(tree, th, 0.1, stats=True)
        theta[str(th)] = {"rays_per_element": st["interactions"] / n,
                          "rms_error_vs_theta0": rms(f[sinks], f0)}
    fr = trevr.compute_flux(tree, 0.75, 1e-8)
    tau = {}
    for tr in (0.01, 0.1, 1.0, 1e6):
        f, st = trevr.compute_flux(tree, 0.75, tr, stats=True)
        tau[str(tr)] = {"segments_per_element": st["segments"] / n,
                        "rms_error_vs_tau_ref_1e-8": rms(f, fr)}
    tree.free()
    return {"workload": "perturbed-glass stand-in, 64^3 gas + 64^3 stars, 24 tabulated modes",
            "theta_sweep_tau_ref_0.1": theta, "tau_ref_sweep_theta_0.75": tau,
            "paper_prints": "theta 0.75: 200 rays, 3 %; theta 0.45: 500 rays, 1 %; "
                            "tau_ref 0.1: 850 segments, 1 % (Sec. 3.1.2, 3.1.3)"}


def run_ours(args):
    import torch
    from paper_1902_08083_gb300 import autotune, trevr

    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    # weak scaling: every rank solves its own instance of the workload (seed + rank)
    P, desc = _problem(args.workload, seed_offset=rank)
    n = int(P["gas_xyz"].shape[1])
    stream = torch.cuda.current_stream()
    g = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev)
         for k in ("gas_xyz", "alpha", "src_xyz", "src_lum")}
    flux = torch.empty(n, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    shape = {}  # the walk's launch shape, picked by the autotuner below

    def step(timed_events=None):
        tree = trevr.build_tree(g["gas_xyz"], g["alpha"], g["src_xyz"], g["src_lum"],
                                lo=P["lo"], side=P["side"], bucket=P["bucket"], stream=stream)
        if timed_events is not None:
            timed_events[1].record(stream)
        trevr.compute_flux(tree, P["theta"], P["tau_ref"], out=flux, stream=stream, **shape)
        if timed_events is not None:
            timed_events[2].record(stream)
        return tree

    # the walk's shape from the autotuner, timed on this tree (untimed here); then
    # counters (untimed) for the algorithmic-bytes figure
    tree = step()
    tuned = autotune.tune_walk(tree, P["theta"], P["tau_ref"], use_cache=False)
    shape.update(walk_variant=tuned["walk_variant"], sinks_per_warp=tuned["sinks_per_warp"])
    _, st = trevr.compute_flux(tree, P["theta"], P["tau_ref"], out=flux, stats=True,
                               stream=stream, **shape)
    tree.free()
    for _ in range(args.warmup):
        step().free()
    torch.cuda.synchronize()

    clocks = Clocks(local, args.clocks_dir)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = trevr.kernel_launches()
    evs = []
    for _ in range(args.steps):
        flush.zero_()  # L2 flush outside the timed interval
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        t = step(e)
        evs.append(e)
        t.free()
    torch.cuda.synchronize()
    launches = trevr.kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[2]) for e in evs]
    build_ms = [e[0].elapsed_time(e[1]) for e in evs]
    walk_ms = [e[1].elapsed_time(e[2]) for e in evs]
    t_step = reduce_max(sum(step_ms) / len(step_ms), world, dev)
    if world > 1:
        torch.distributed.barrier()
    value = job_value(n, world, t_step)

    # end to end through the public API with host buffers: pinned H2D of the
    # step's inputs, build, flux, D2H of the fluxes, all inside the timed region
    host = {k: torch.from_numpy(np.ascontiguousarray(P[k])).pin_memory()
            for k in ("gas_xyz", "alpha", "src_xyz", "src_lum")}
    hflux = torch.empty(n, dtype=torch.float32).pin_memory()
    dbuf = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = hflux.numel() * 4

    def e2e_step():
        for k in host:
            dbuf[k].copy_(host[k], non_blocking=True)
        tr = trevr.build_tree(dbuf["gas_xyz"], dbuf["alpha"], dbuf["src_xyz"], dbuf["src_lum"],
                              lo=P["lo"], side=P["side"], bucket=P["bucket"], stream=stream)
        trevr.compute_flux(tr, P["theta"], P["tau_ref"], out=flux, stream=stream, **shape)
        hflux.copy_(flux, non_blocking=True)
        stream.synchronize()
        tr.free()

    e2e_step()
    e2e_ms = []
    for _ in range(max(2, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    t_e2e = reduce_max(sum(e2e_ms) / len(e2e_ms), world, dev)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # roofline of the dominant kernel (the sink walk). Its cell records are L1/L2 hits
    # (DRAM carries ~80 B per sink), and it is bound by instruction issue: achieved =
    # warp instructions issued per launch / the walk's event-timed duration, against
    # the issue limit of the SMs at the sampled clock. Secondary: the logical bytes,
    # 20 B per sink (position, leaf, flux) + 32 B per source cell tested + 32 B per
    # cell clipped by a ray, per second against the HBM copy bandwidth.
    alg_bytes = 20 * n + 32 * st["src_nodes_visited"] + 32 * st["cells_clipped"]
    t_walk = sum(walk_ms) / len(walk_ms) * 1e-3
    peak, peak_kind = _peaks()
    sm_mhz = clk.get("sm_mhz") or _peaks_clock()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # the committed counters are those of the merged-ray walk (variant 3)
    prof = (_kernel_profile("walk_warp_kernel_issue.json")
            if shape["walk_variant"] in (0, 3) else None)
    roofline = _issue_roofline(prof, n, t_walk, sm_mhz, n_sm, alg_bytes, peak, peak_kind,
                               "walk_warp_kernel, variant 3 (warp-shared walk, merged rays, "
                               "flux, no counters)")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _config(P, args.workload, desc),
            "build_ms": sum(build_ms) / len(build_ms), "walk_ms": t_walk * 1e3,
            "walk_only_fluxes_per_s": world * n / t_walk,
            "interactions_per_s": world * st["interactions"] / t_walk,
            "per_sink": {"interactions": st["interactions"] / n, "segments": st["segments"] / n,
                         "cells_visited": st["src_nodes_visited"] / n,
                         "refinements": st["refine_expansions"] / n,
                         "cells_clipped": st["cells_clipped"] / n},
            "roofline": roofline,
            "walk_autotune": {"walk_variant": tuned["walk_variant"],
                              "sinks_per_warp": tuned["sinks_per_warp"],
                              "ms_per_shape": tuned["table"]},
            "e2e": {"value": job_value(n, world, t_e2e), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches), "clocks": clk}

    if world == 1 and not args.no_extras:
        line["batched"] = _bench_batched(args, sm_mhz)
        line["adjoint"] = _bench_adjoint(args)
        line["terminated"] = _bench_termination(args, P, g)
        line["top_down"] = _bench_topdown(args, P, g)
        line["bands"] = _bench_bands(args, P, g)
        line["sub_bucket"] = _bench_sub_bucket(args)
        if args.glass:
            line["glass"] = _bench_glass(args)

    if world == 1 and not args.no_cpu_baseline:
        info, sinks, fo, _ = _oracle_baseline(P, n, args.cpu_sample, args.cpu_seconds)
        fg = flux.cpu().numpy()[sinks].astype(np.float64)
        big = fo >= 1e-30
        rel = np.abs(fg[big] - fo[big]) / fo[big]
        line["cpu_baseline"] = {k: info[k] for k in ("value", "unit", "cores", "kind", "sample",
                                                      "cpu")}
        line["parity"] = {"sinks": int(len(sinks)), "median_rel_err": float(np.median(rel)),
                          "max_rel_err": float(rel.max()),
                          "pass": bool(np.median(rel) <= 1e-5 and rel.max() <= 1e-3)}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_profile(args):
    """A short program for ncu: one tree build, then on a contiguous Morton-ordered run
    of --sink-sample sinks the walk with counters (launch 0, whose counters are
    printed) and the walk the benchmark times, without counters (launch 1, the one
    to capture: -k regex:walk_warp_kernel -s 1 -c 1)."""
    import torch
    from paper_1902_08083_gb300 import trevr
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    P, desc = _problem(args.workload)
    n = int(P["gas_xyz"].shape[1])
    g = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev)
         for k in ("gas_xyz", "alpha", "src_xyz", "src_lum")}
    tree = trevr.build_tree(g["gas_xyz"], g["alpha"], g["src_xyz"], g["src_lum"], lo=P["lo"],
                            side=P["side"], bucket=P["bucket"])
    m = min(n, args.sink_sample) if args.sink_sample > 0 else n
    # a contiguous run of sinks in Morton order (what the full walk's warps see)
    perm = tree.export()["perm"]
    start = (n - m) // 2
    sinks = perm[start:start + m].to(torch.int64).contiguous()
    _, st = trevr.compute_flux(tree, P["theta"], P["tau_ref"], sink_idx=sinks, stats=True)
    f = trevr.compute_flux(tree, P["theta"], P["tau_ref"], sink_idx=sinks)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.workload, "n_gas": n, "sinks": m,
                      "cells_tested": st["src_nodes_visited"],
                      "cells_clipped": st["cells_clipped"],
                      "flux_sum": float(f.double().sum())}), flush=True)
    tree.free()


def run_profile_sub(args):
    """A short program for ncu on the sub-bucket walk: the 2^18-particle sub-bucket
    workload, its neighbour lists, one walk with counters (launch 0, counters
    printed) and one without (launch 1, the one to capture:
    -k regex:walk_warp_kernel -s 1 -c 1)."""
    import torch
    from paper_1902_08083_gb300 import trevr
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    P = workloads.sub_bucket_problem(n_gas=1 << 18, n_src=1024, seed=12)
    t = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev)
         for k in ("gas_xyz", "alpha", "src_xyz", "src_lum", "weight", "hsml")}
    tree = trevr.build_tree(t["gas_xyz"], t["alpha"], t["src_xyz"], t["src_lum"],
                            weight=t["weight"], lo=P["lo"], side=P["side"], bucket=P["bucket"])
    tree.set_smoothing(t["hsml"])
    _, st = trevr.compute_flux(tree, P["theta"], P["tau_ref"], sub_bucket=1, stats=True)
    f = trevr.compute_flux(tree, P["theta"], P["tau_ref"], sub_bucket=1)
    torch.cuda.synchronize()
    n = int(P["gas_xyz"].shape[1])
    print(json.dumps({"profile": "sub_bucket", "sinks": n,
                      "cells_tested": st["src_nodes_visited"],
                      "cells_clipped": st["cells_clipped"], "segments": st["segments"],
                      "sub_bucket_segments": st["sub_bucket_segments"],
                      "flux_sum": float(f.double().sum())}), flush=True)
    tree.free()


def run_profile_batched(args):
    """A short program for ncu on the batched walk: the 64 boxes, the autotuned launch
    shape, one batched call with counters (launch 0, counters printed) and one without
    (launch 1, the one to capture: -k regex:walk_warp_batched_kernel -s 1 -c 1)."""
    import torch
    from paper_1902_08083_gb300 import autotune, trevr
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    boxes = workloads.batched_boxes()
    trees = []
    for P in boxes:
        g = {k: torch.from_numpy(np.ascontiguousarray(P[k])).to(dev)
             for k in ("gas_xyz", "alpha", "src_xyz", "src_lum")}
        trees.append(trevr.build_tree(g["gas_xyz"], g["alpha"], g["src_xyz"], g["src_lum"],
                                      lo=P["lo"], side=P["side"], bucket=P["bucket"]))
    th, tr = boxes[0]["theta"], boxes[0]["tau_ref"]
    B = trevr.Batch(trees)
    tune = autotune.tune(B, th, tr)
    shape = dict(sinks_per_warp=tune["sinks_per_warp"], block_size=tune["block_size"],
                 walk_variant=tune.get("walk_variant", 0))
    st = B.run(th, tr, stats=True, **shape)
    B.run(th, tr, **shape)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "batched", "sinks": B.n_sinks, "launch_shape": shape,
                      "cells_tested": st["src_nodes_visited"],
                      "cells_clipped": st["cells_clipped"]}), flush=True)
    B.free()
    for t in trees:
        t.free()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clumpy", choices=["clumpy", "stromgren", "uniform"])
    ap.add_argument("--cpu-sample", type=int, default=2048)
    ap.add_argument("--clocks-dir", default=None,
                    help="directory in which to keep the raw nvidia-smi clock samples")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="seconds of oracle walking timed for cpu_baseline")
    ap.add_argument("--ref-seconds", type=float, default=90.0,
                    help="seconds of oracle walking over all steps of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (64 boxes) and adjoint (2^21) measurements")
    ap.add_argument("--glass", action="store_true",
                    help="also run the perturbed-glass stand-in sweeps (off by default)")
    ap.add_argument("--profile", action="store_true",
                    help="build once and run the walk twice on --sink-sample sinks (for ncu)")
    ap.add_argument("--profile-batched", action="store_true",
                    help="the 64 boxes: one batched walk with counters, one without (for ncu)")
    ap.add_argument("--profile-sub", action="store_true",
                    help="the sub-bucket workload: one walk with counters, one without (for ncu)")
    ap.add_argument("--sink-sample", type=int, default=1 << 20)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile:
        run_profile(args)
    elif args.profile_batched:
        run_profile_batched(args)
    elif args.profile_sub:
        run_profile_sub(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
