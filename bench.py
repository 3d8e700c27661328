#!/usr/bin/env python
"""Benchmark of the exponential Leja integrator on one GB300 (or N replicas).

Workload (default): the 4096 x 4096 precision-form workload on [-1, 1]^2 in
its full-FP64 path: zero Dirichlet boundaries, field lines of a seeded
8-mode random-phase stream function, D_par = 1, D_perp = 10^U(-6,-2)
(seeded), a = 0, 16 seeded Gaussian sources (sigma 0.02), Gaussian u0
(sigma 0.2), exponential midpoint (Eq. exp_midpoint) at dt = 100 Delta
t_CFL, tol 1e-10.  One benchmark step = one exponential-midpoint step
(A u + S, the Leja series of phi_1, the update).  The 512^2 two-stage
workload and the 64^2 periodic workload are measured as forms.

Metric: Mcell-steps/s = cells x steps / time.  ``value`` is device time
(CUDA events on the operator's stream, inputs resident, L2 flushed before
every step by writing a 256 MiB buffer); ``e2e`` is the same metric through
the C ABI with the state in pinned host memory (host->device and
device->host copies inside the timed region).  ``roofline`` reports the
fused Leja iteration kernel; ``cpu_baseline`` times the FP64 CPU oracle on
a bounded sample of the same workload in a subprocess that runs beside the
GPU measurements, and its first step is the reference for the errors.

Multi-GPU: replicas only (the workload does not shard); each rank runs the
same problem and ``value`` is the sum over ranks of cell-steps / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: how to build the problem (workloads.configs) and its step size in Delta t_CFL
    "c2-4096sq-dirichlet-stream-midpoint-fp64": dict(kind="c2", nx=4096, tol=1e-10,
                                                     dt_over_cfl=100.0),
    "c1-512sq-dirichlet-circular-expquad2-dt200cfl": dict(kind="c1", nx=512, dt_over_cfl=200.0),
    "c0-64sq-periodic-uniform30-midpoint": dict(kind="c0", nx=64, dt_over_cfl=100.0),
}
DEFAULT_WORKLOAD = "c2-4096sq-dirichlet-stream-midpoint-fp64"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz


def _measured_hbm_gbs() -> float:
    """Copy bandwidth from the measured peaks beside this file (falls back to 6.8 TB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


HBM_PEAK_GBS = _measured_hbm_gbs()
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--reference-seconds", type=float, default=60.0,
                    help="bound on the reference arm's timed oracle steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=9)
    ap.add_argument("--nx", type=int, default=0,
                    help="override the workload's grid side (smaller cases for profiling)")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--form-steps", type=int, default=5)
    ap.add_argument("--learned-fields", type=int, default=10000)
    ap.add_argument("--forms", default="fp32,c1,c0,cn,paper,batched,learned,momentum,adaptive",
                    help="comma list of extra forms to measure: fp32, c1, c0, cn, batched, "
                         "learned, paper, momentum, adaptive")
    return ap.parse_args()


def problem(name, nx=0):
    from workloads import config0, config1, config2
    w = WORKLOADS[name]
    nx = nx or w["nx"]
    if w["kind"] == "c2":
        return config2(nx=nx, tol=w["tol"])
    if w["kind"] == "c1":
        return config1(nx=nx, dt_factor=w["dt_over_cfl"])
    return config0(nx=nx)


# --------------------------------------------------------------------------- oracle leg
ORACLE_CODE = """
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from bench import problem
from oracle import operator as oop, spectral, integrators
t_setup = time.perf_counter()
p = problem({workload!r})
A = oop.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
alpha = spectral.gershgorin(A)
S = lambda t: p.source_at(t).ravel()
setup_s = time.perf_counter() - t_setup
u, t, steps, iters = p.u0.ravel().copy(), 0.0, 0, 0
for _ in range({warmup}):
    u, st = integrators.expquad_step(A, u, t, p.dt, p.s, p.c, S, alpha, tol=p.tol)
    t += p.dt
t0 = time.perf_counter()
el = 0.0
first_iters = None
while True:
    u, st = integrators.expquad_step(A, u, t, p.dt, p.s, p.c, S, alpha, tol=p.tol)
    t += p.dt; steps += 1; iters += st.iters
    el = time.perf_counter() - t0
    if steps == 1:
        first_iters = int(st.iters)
        if {out_npy!r} is not None:
            np.save({out_npy!r}, u)
    if el >= {seconds} or steps >= {max_steps}:
        break
print(json.dumps(dict(steps=steps, seconds=el, cells=p.grid.n, iters=iters, alpha=alpha,
                      setup_s=setup_s, first_step_iters=first_iters)))
"""


def start_oracle_sample(workload: str, seconds: float, max_steps: int, out_npy: str | None,
                        warmup: int = 0):
    """Start the CPU oracle (one core: BLAS threads pinned to 1) from the
    workload's initial state in a subprocess: ``warmup`` untimed steps, then
    steps until ``seconds`` have passed (at least one) or ``max_steps``; the
    first timed step's state is saved to ``out_npy``.  Returns the process."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_CODE.format(root=ROOT, workload=workload, warmup=warmup, out_npy=out_npy,
                              seconds=seconds, max_steps=max_steps)
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                            stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT)


def finish_oracle_sample(proc):
    """Wait for the oracle subprocess; returns a dict with its throughput."""
    out, err = proc.communicate()
    if proc.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + err[-3000:])
    d = json.loads(out.strip().splitlines()[-1])
    d["value"] = d["cells"] * d["steps"] / d["seconds"] / 1e6
    return d


def oracle_sample(workload: str, seconds: float, max_steps: int, out_npy: str | None,
                  warmup: int = 0):
    return finish_oracle_sample(start_oracle_sample(workload, seconds, max_steps, out_npy, warmup))


def run_reference(args):
    """The reference arm: the FP64 CPU oracle on this arm's workload, one
    oracle step per benchmark step, on one host core.  The timed steps are
    bounded by --reference-seconds (at least one step), so the run ends within
    a few minutes even where one oracle step takes tens of seconds."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    d = oracle_sample(args.workload, seconds=args.reference_seconds,
                      max_steps=max(1, args.steps), out_npy=None, warmup=0)
    line = {
        "impl": "reference", "metric": "Mcell-steps/s", "value": round(d["value"], 6),
        "unit": "Mcell-steps/s", "n_gpus": args.gpus, "steps": d["steps"],
        "ms_per_step": 1e3 * d["seconds"] / d["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "cells": d["cells"]}, "warmup": 0,
        "cpu_baseline": {"value": round(d["value"], 6), "unit": "Mcell-steps/s", "cores": 1,
                         "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{d['steps']} full exponential steps from t=0 "
                                   f"({d['seconds']:.1f} s timed; requested {args.steps} steps "
                                   f"after {args.warmup} warm-up, bounded by "
                                   f"{args.reference_seconds:.0f} s; operator assembly "
                                   f"{d['setup_s']:.0f} s untimed)"},
        "e2e": {"value": round(d["value"], 6), "unit": "Mcell-steps/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx),
                                          f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.f.close()

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except FileNotFoundError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def source_digest(files) -> str:
    """sha256 over the named source files (package csrc/), in order."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2307_12276_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def traffic_per_launch(files, summary: str):
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary
    (lines "source_sha256: ..." and "dram_bytes_per_launch: ..."), or None when
    the kernel's sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        text = open(path).read()
    except FileNotFoundError:
        return None
    fields = {}
    for line in text.splitlines():
        line = line.strip().lstrip("-* ").replace("`", "")
        if ":" in line:
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    if fields.get("source_sha256") != source_digest(files):
        return None
    try:
        return float(fields["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# sources that define each profiled kernel (the digest in its summary covers these)
F64_SERIES_SOURCES = ("persistent_f64.cu", "stencil9.cuh", "ad_internal.h")
F64_ITER_SOURCES = ("stencil_kernels.cu", "stencil9.cuh", "series_finish.cuh", "tile_f32.cuh",
                    "ad_internal.h", "sqsum.cuh")
F32_ITER_SOURCES = ("stencil_kernels.cu", "tile_f32.cuh", "tile_f32_vec.cuh", "tile_f32_ring.cuh",
                    "ad_internal.h")
F32_PAIR_SOURCES = F32_ITER_SOURCES + ("tile_f32_pair.cuh",)
F32_TMA_SOURCES = F32_PAIR_SOURCES + ("tile_f32_bulk.cuh", "tile_f32_pair_tma.cuh")
MOM_SOURCES = ("momentum.cu", "series_finish.cuh", "tile_f32.cuh", "ad_internal.h", "sqsum.cuh")

# the FP64 series kernel behind each path that ad_series_timing reports
SERIES_KERNEL_NAMES = {"graph loop of per-iteration kernels": "leja_iter_f64_k",
                       "host-driven per-iteration kernels": "leja_iter_f64_k"}


def _dev_f64(dev):
    import numpy as np
    import torch
    return lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=dev)


# --------------------------------------------------------------------------- ours
def measure_workload(ad, dev, stream, p, flush, steps, warmup, e2e_steps, world=1,
                     label="", dt_over_cfl=None):
    """FP64 exponential steps of problem ``p`` through the C ABI.

    One step from u0 (kept on the host: compared with the oracle's first
    step), warm-up steps, then ``steps`` timed steps enqueued without host
    round trips (CUDA events per step, L2 flushed before each), the device
    time of every Newton series inside them (the roofline's kernel time), and
    ``e2e_steps`` steps through the C ABI with the state in pinned host
    memory.  Returns (result dict, first-step state as a NumPy array)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    g = p.grid
    T = _dev_f64(dev)
    op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), p.ax, p.ay,
                            ad.FP64, stream=stream)
    src = ad.Source([T(gk) for gk in p.source.g], list(p.source.h)) if len(p.source) else None
    u0 = T(p.u0)
    u = u0.clone()
    st1 = ad.expquad_step(op, u, 0.0, p.dt, p.s, p.c, src, tol=p.tol)
    torch.cuda.synchronize()
    u1 = u.cpu().numpy()
    t = p.dt
    for _ in range(max(0, warmup - 1)):
        ad.expquad_step(op, u, t, p.dt, p.s, p.c, src, tol=p.tol)
        t += p.dt
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ad.time_series(op)          # event pair around every series kernel launch in the timed steps
    # The steps are enqueued without a host round trip between them (the
    # asynchronous entry point); the totals call synchronises and reports
    # their iterations, launches and worst status.
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(steps):
            flush.zero_()
            starts[k].record(stream)
            ad.expquad_step_async(op, u, t, p.dt, p.s, p.c, src, tol=p.tol)
            ends[k].record(stream)
            t += p.dt
        tot = ad.async_totals(op)
        torch.cuda.synchronize()
    launches = tot["kernel_launches"]
    assert tot["converged"] and tot["substeps"] == steps
    series_t = ad.series_timing(op)
    ad.time_series(op, False)
    if world > 1:
        dist.barrier()
    dev_ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
    dev_ms, value = job_throughput(dev_ms, g.n, steps, world, dev)

    # e2e: the state lives in pinned host memory; the C ABI stages it per call
    # through device buffers the operator allocated at creation
    uh = torch.empty(g.n, dtype=torch.float64, pin_memory=True)
    uh.copy_(u0.cpu())
    ue = uh.numpy()
    te = []
    for k in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ad.expquad_step(op, ue, k * p.dt, p.dt, p.s, p.c, src, tol=p.tol)
        te.append(time.perf_counter() - t0)
    # host wall time per step: the median (a single host hiccup of a few ms
    # would otherwise dominate a short run); the mean is reported beside it
    e2e_value = g.n / statistics.median(te) / 1e6

    # roofline of the series kernel, from the event pairs around its launches in the timed steps
    aug = p.s == 2
    kernel = SERIES_KERNEL_NAMES.get(series_t["kernel"], str(series_t["kernel"]))
    path = series_t["kernel"]
    fma = 14 if aug else 13   # 9 stencil, shift, (coupling), p, 2 norms: FP64 FMA-class per cell
    flops = 2.0 * fma * g.n
    # 9 weights + y + p (r/w) + y_next (+ w2 for the augmented series), 8 B each
    bytes_alg = (112.0 if aug else 104.0) * g.n
    ms_it = series_t["ms"] / max(series_t["iters"], 1)
    fused = launches == steps and series_t["series"] == steps
    step_flops = 24.0 * g.n if fused else 0.0   # 9 stencil + 2 source + 1 update FMA per cell
    achieved = ((flops * series_t["iters"] + step_flops * series_t["series"])
                / (series_t["ms"] * 1e-3) / 1e12)
    ms_forced = ad.profile_leja_iteration(op, aug=int(aug), reps=300 if g.n < 10 ** 6 else 60)
    fma_peak = ad.fp64_fma_rate(2, 1 << 16, stream=stream)    # this device's DFMA loop, live
    traffic = None
    if kernel == "leja_nsync_f64_k" and g.nx == 512:
        traffic = traffic_per_launch(F64_SERIES_SOURCES, "leja_nsync_f64_512sq.md")
    elif kernel == "leja_tile_f64_k" and g.nx == 512:
        traffic = traffic_per_launch(F64_SERIES_SOURCES, "leja_tile_f64_512sq.md")
    elif kernel == "leja_iter_f64_k" and g.nx == 4096 and not aug:
        traffic = traffic_per_launch(F64_ITER_SOURCES, "leja_iter_f64_4096sq.md")
    hbm_gbs = bytes_alg / (ms_it * 1e-3) / 1e9
    roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
            "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
            "traffic": traffic, "kernel": f"{kernel}<{'true' if aug else 'false'}>",
            "series_path": path,
            "work_unit": ("one launch = one whole step: A u + sources, the Newton series "
                          "(all its Leja iterations), u += P" if fused else
                          "one launch = one Leja iteration (y_{m+1}, p_{m+1}, both squared "
                          "norms, the stopping rule in the last block)"),
            "alg_flops_per_launch_outside_series": step_flops,
            "launches_timed": series_t["series"] if fused else series_t["iters"],
            "iterations_timed": series_t["iters"],
            "ms_per_launch": round(series_t["ms"] / max(series_t["series"], 1) if fused
                                   else ms_it, 5),
            "ms_per_iteration": round(ms_it, 5),
            "ms_per_iteration_forced": round(ms_forced, 5),
            "alg_flops_per_iteration": flops,
            "alg_bytes_per_iteration": bytes_alg,
            "hbm": {"achieved_GBps": round(hbm_gbs, 1), "peak_GBps": HBM_PEAK_GBS,
                    "frac": round(hbm_gbs / HBM_PEAK_GBS, 4),
                    "note": "algorithmic bytes per iteration / iteration time, of measured copy "
                            "bandwidth (the FP64 pipe, not HBM, bounds this kernel)"},
            "measured_fp64_fma_tflops": round(fma_peak, 4),
            "frac_of_measured_fp64_fma": round(achieved / fma_peak, 4),
            "peak_note": "of derived FP64 peak: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz; "
                         "measured_fp64_fma_tflops is a DFMA loop on every SM timed in this "
                         "run (ad_fp64_fma_rate)"}
    if kernel == "leja_iter_f64_k":
        # the library's rule: the large-grid iteration forms the norms' two
        # squares per cell on the integer and FP32 pipes unless AD_F64_NORMS=fp64
        off_pipe = not os.environ.get("AD_F64_NORMS", "").startswith("f")
        pipe_ops = fma - 2 if off_pipe else fma
        roof["fp64_pipe_ops_per_cell"] = pipe_ops
        roof["frac_of_measured_fp64_fma_pipe_ops"] = round(achieved * pipe_ops / fma / fma_peak, 4)
        roof["fp64_pipe_note"] = ("achieved counts the method's FP64 FMA-class operations per cell "
                                  f"({fma}); {fma - pipe_ops} of them (the norms' squares) run off "
                                  "the FP64 pipe, so the pipe itself executes "
                                  f"{pipe_ops} per cell")
    res = {"workload": label or p.name, "nx": g.nx, "ny": g.ny, "cells": g.n,
           "value": value, "dev_ms": dev_ms, "ms_per_step": dev_ms / steps,
           "leja_iters_per_step": tot["iters"] / steps, "gpu_launches": launches,
           "first_step_iters": st1["iters"],
           "e2e": {"value": round(e2e_value, 4), "unit": "Mcell-steps/s",
                   "h2d_bytes_per_step": 8 * g.n, "d2h_bytes_per_step": 8 * g.n,
                   "steps": len(te), "stat": "median of per-step host wall times",
                   "mean_ms_per_step": round(1e3 * statistics.mean(te), 4)},
           "roofline": roof, "clocks": clk.summary(),
           "config": {"workload": label or p.name, "nx": g.nx, "ny": g.ny, "cells": g.n,
                      "dt_over_cfl": dt_over_cfl, "s": p.s, "c": list(p.c), "tol": p.tol,
                      "l2": "flushed before every timed step (256 MiB write)",
                      "parallelism": "replicas" if world > 1 else "single"}}
    op.close()
    del u, u0, src
    torch.cuda.empty_cache()
    return res, u1


def measure_fp32_form(ad, dev, stream, flush, steps, p=None):
    """The FP32-storage form of the 4096^2 stream-function workload
    (exponential midpoint, tol 1e-6): throughput, Leja iterations and the
    fused FP32 kernel's algorithmic HBM bandwidth against the copy peak.
    Returns (result dict, state after one step from u0 as float64 NumPy)."""
    import numpy as np
    import torch
    from workloads import config2
    if p is None:
        p = config2(nx=4096)
    g = p.grid
    T = _dev_f64(dev)
    op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), 0.0, 0.0,
                            ad.FP32_STORAGE, stream=stream)
    src = ad.Source([T(p.source.g[0]).float()], None)
    u = T(p.u0).float()
    ad.expquad_step(op, u, 0.0, p.dt, 1, (0.5,), src, tol=1e-6)
    torch.cuda.synchronize()
    u1 = u.double().cpu().numpy()
    t = p.dt
    ad.expquad_step(op, u, t, p.dt, 1, (0.5,), src, tol=1e-6)
    t += p.dt
    torch.cuda.synchronize()
    ms, iters = 0.0, []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ad.expquad_step(op, u, t, p.dt, 1, (0.5,), src, tol=1e-6)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        iters.append(st["iters"])
        t += p.dt
    ms_iter = ad.profile_leja_iteration(op, aug=0, reps=100)
    ad.time_series(op)
    ad.expquad_step(op, u, t, p.dt, 1, (0.5,), src, tol=1e-6)
    path = ad.series_timing(op)["kernel"] or ""
    ad.time_series(op, False)
    kind = os.environ.get("AD_F32_KERNEL", "ring")[:1]
    kernel = {"b": "leja_iter_f32_bulk_k", "t": "leja_iter_f32_k",
              "v": "leja_iter_f32_vec_k"}.get(kind, "leja_iter_f32_ring_k")
    pair = "two-iteration" in path
    tma = "TMA" in path
    # one launch: y, p read and written, 3 coefficient fields read, 4 B each;
    # the two-iteration kernel does this once for two iterations
    iters_per_launch = 2 if pair else 1
    ms_launch = ms_iter * iters_per_launch
    alg_bytes = 28.0 * g.n
    gbs = alg_bytes / (ms_launch * 1e-3) / 1e9
    if pair and tma:
        kernel = "leja_iter2_f32_tma_k"
        traffic = traffic_per_launch(F32_TMA_SOURCES, "leja_iter2_f32_tma_4096sq.md")
    elif pair:
        kernel = "leja_iter2_f32_ring_k"
        traffic = traffic_per_launch(F32_PAIR_SOURCES, "leja_iter2_f32_ring_4096sq.md")
    elif kernel == "leja_iter_f32_ring_k":
        traffic = traffic_per_launch(F32_ITER_SOURCES, "leja_iter_f32_ring_4096sq.md")
    else:
        traffic = None
    op.close()
    del u, src
    torch.cuda.empty_cache()
    value = g.n * steps / (ms * 1e-3) / 1e6
    return {"workload": "c2-4096sq-dirichlet-stream-midpoint-fp32", "cells": g.n,
            "value": round(value, 2), "unit": "Mcell-steps/s",
            "ms_per_step": round(ms / steps, 4), "leja_iters_per_step": statistics.mean(iters),
            "tol": 1e-6, "dtype": "f32 storage/arithmetic, f64 Leja scalars and norm sums",
            "series_path": path,
            "roofline": {"bound": "hbm",
                         "kernel": kernel + (("<0, %d>" % (0 if os.environ.get("AD_F32_MARCH", "1")
                                                           [:1] == "0" else 1)) if pair and not tma
                                             else ("<0>" if pair else "<0,0>")),
                         "iterations_per_launch": iters_per_launch, "ms_per_launch":
                         round(ms_launch, 5), "achieved": round(gbs, 1), "peak": HBM_PEAK_GBS,
                         "unit": "GB/s", "frac": round(gbs / HBM_PEAK_GBS, 4),
                         "traffic": traffic, "alg_bytes_per_launch": alg_bytes,
                         "peak_note": "of measured copy bandwidth"}}, u1


def measure_fp64_at_tol(ad, dev, stream, flush, steps, p, tol):
    """The plain FP64 path on the FP32 form's workload at the FP32 form's
    tolerance (exponential midpoint, the same steps and timing as
    measure_fp32_form): the FP32 form's speed-up at equal tolerance."""
    import torch
    g = p.grid
    T = _dev_f64(dev)
    op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), 0.0, 0.0,
                            ad.FP64, stream=stream)
    src = ad.Source([T(p.source.g[0])], None)
    u = T(p.u0)
    ad.expquad_step(op, u, 0.0, p.dt, 1, (0.5,), src, tol=tol)
    t = p.dt
    ad.expquad_step(op, u, t, p.dt, 1, (0.5,), src, tol=tol)
    t += p.dt
    torch.cuda.synchronize()
    ms, iters = 0.0, []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ad.expquad_step(op, u, t, p.dt, 1, (0.5,), src, tol=tol)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        iters.append(st["iters"])
        t += p.dt
    op.close()
    del u, src
    torch.cuda.empty_cache()
    return {"value": round(g.n * steps / (ms * 1e-3) / 1e6, 2), "unit": "Mcell-steps/s",
            "ms_per_step": round(ms / steps, 4), "leja_iters_per_step": statistics.mean(iters),
            "tol": tol, "dtype": "f64"}


def measure_momentum_form(ad, dev, stream, steps=3):
    """The momentum-coupled operator of Eq. cr_full on a 256^2 x 32 grid
    (2.1 M unknowns, FP64, Dirichlet, circular field, constant advection):
    exponential midpoint steps with a time-independent source at
    100 Delta t_CFL of the most diffusive slice, tol 1e-10; and the fused
    iteration kernel's FP64 rate from a forced 100-iteration series."""
    import numpy as np
    import torch
    from workloads.fields import BC_DIRICHLET0
    from workloads.momentum import momentum_problem
    mp = momentum_problem(256, 256, 32, BC_DIRICHLET0, "circular", adv=(0.1, 0.05),
                          dt_factor=100.0)
    s = mp.spatial
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=dev)
    op = ad.create_momentum_operator(s.grid.nx, s.grid.ny, s.grid.bc, T(s.Dxx), T(s.Dxy),
                                     T(s.Dyy), mp.mom.P, mp.mom.beta, mp.mom.dpp, mp.mom.b,
                                     mp.mom.loss, ax=s.ax, ay=s.ay, stream=stream)
    N = op.N
    u, S = T(mp.u0), T(mp.S)
    ad.momentum_step(op, u, mp.dt, S, tol=mp.tol)            # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    e0.record(stream)
    for _ in range(steps):
        iters.append(ad.momentum_step(op, u, mp.dt, S, tol=mp.tol)["iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = torch.empty_like(u)
    e0.record(stream)
    ad.momentum_leja_phi1(op, S, out, mp.dt, force_iters=100)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_iter = e0.elapsed_time(e1) / 100
    flops = 42.0 * N          # 21 FP64 FMA-class operations per unknown (constant advection)
    tf = flops / (ms_iter * 1e-3) / 1e12
    op.close()
    del u, S, out
    torch.cuda.empty_cache()
    return {"workload": "momentum-256sq-x32p-dirichlet-circular-midpoint-fp64", "unknowns": N,
            "value": round(N / (ms * 1e-3) / 1e6, 2), "unit": "Munknown-steps/s",
            "ms_per_step": round(ms, 4), "leja_iters_per_step": float(np.mean(iters)),
            "tol": mp.tol, "dt_over_cfl": 100.0,
            "roofline": {"bound": "alu", "kernel": "mom_iter_k<true, true>",
                         "ms_per_iteration": round(ms_iter, 5),
                         # the library's rule: the norms' two squares per unknown run off
                         # the FP64 pipe unless AD_F64_NORMS=fp64
                         "fp64_pipe_ops_per_unknown":
                             21 if os.environ.get("AD_F64_NORMS", "").startswith("f") else 19,
                         "alg_flops_per_iteration": flops, "achieved": round(tf, 4),
                         "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                         "frac": round(tf / FP64_PEAK_TFLOPS, 4),
                         "traffic": traffic_per_launch(MOM_SOURCES, "mom_iter_256sq_x32p.md"),
                         "peak_note": "of derived FP64 peak; iteration time includes the "
                                      "host-driven chunk reads of the control block"}}


def measure_adaptive_substeps(ad, dev, stream, dt_factor=2000.0):
    """Adaptive substep control on the 512^2 workload: one two-stage step of
    dt_factor Delta t_CFL with the fixed rule (rho_max 200, equal substeps) and
    with the adaptive controller (no rho_max, a 100-iteration budget per
    series).  Error against the same step with the fixed rule at tol 1e-12."""
    import numpy as np
    import torch
    from workloads import config1
    p = config1(nx=512, dt_factor=dt_factor)
    g = p.grid
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=dev)
    op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), p.ax, p.ay, ad.FP64,
                            stream=stream)
    src = ad.Source([T(gk) for gk in p.source.g], list(p.source.h))
    ref = T(p.u0)
    ad.expquad_step(op, ref, 0.0, p.dt, p.s, p.c, src, tol=1e-12)
    out = {}
    for name, adaptive, rho_max, budget in (("fixed", False, 200.0, 500),
                                            ("adaptive", True, 1e9, 100)):
        ad.set_options(op, rho_max=rho_max, max_iters=budget)
        ad.set_substep_control(op, adaptive)
        u = T(p.u0)
        ad.expquad_step(op, u, 0.0, p.dt, p.s, p.c, src, tol=p.tol)    # warm-up
        u = T(p.u0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ad.expquad_step(op, u, 0.0, p.dt, p.s, p.c, src, tol=p.tol)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"ms": round(e0.elapsed_time(e1), 3), "iters": st["iters"],
                     "substeps": st["substeps"], "rejected": st["rejected"],
                     "err_vs_tol1e-12_step": float(torch.linalg.norm(u - ref) /
                                                   torch.linalg.norm(ref))}
    op.close()
    return {"workload": f"c1-512sq-dirichlet-circular-expquad2-dt{int(dt_factor)}cfl",
            "tol": p.tol, **out}


def measure_cn_vs_exp(ad, dev, stream, T_cfl=1000.0, cn_budget_ms=60000.0):
    """Crank-Nicolson (GMRES) and the penalised IMEX step (conjugate gradients)
    against two-stage exponential quadrature on the 512^2 workload, to
    T = T_cfl Delta t_CFL: the exponential method at 200 Delta t_CFL, CN at the
    largest step (halving from 200) whose error matches it, the penalised step
    at 200, 50, 12.5 and 3.125 Delta t_CFL.  Reference: the FP64 GPU path, Gauss nodes, step 12.5 Delta t_CFL,
    tol 1e-12 (its per-step parity with the oracle is pinned by the GPU tests)."""
    import numpy as np
    import torch
    from workloads import config1
    p = config1(nx=512, dt_factor=200.0)
    g = p.grid
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=dev)
    op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), p.ax, p.ay, ad.FP64,
                            stream=stream)
    src = ad.Source([T(gk) for gk in p.source.g], list(p.source.h))
    ad.reserve_gmres(op, 50)
    t_end = T_cfl * p.cfl
    gauss = (0.5 - 0.5 / 3 ** 0.5, 0.5 + 0.5 / 3 ** 0.5)

    def run(method, factor, tol=1e-10, gmres_tol=1e-10):
        n = int(round(T_cfl / factor))
        dt = t_end / n
        u = T(p.u0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        it = 0
        for k in range(n):
            if method == "cn":
                st = ad.cn_step(op, u, k * dt, dt, src, gmres_tol=gmres_tol, restart=50)
            elif method == "penalised":
                st = ad.penalised_step(op, u, k * dt, dt, src, beta=beta, cg_tol=1e-10)
            elif method == "gauss":
                st = ad.expquad_step(op, u, k * dt, dt, 2, gauss, src, tol=tol)
            else:
                st = ad.expquad_step(op, u, k * dt, dt, 2, p.c, src, tol=tol)
            it += st["matvecs"]
        e1.record(stream)
        torch.cuda.synchronize()
        return u, e0.elapsed_time(e1), it, n

    beta = ad.penalty_beta(g.nx, g.ny, T(p.Dxx), T(p.Dxy), T(p.Dyy), stream=stream)
    ref, _, _, _ = run("gauss", 12.5, tol=1e-12)
    nref = float(torch.linalg.norm(ref))
    ue, ms_e, mv_e, n_e = run("exp", 200.0)
    err_e = float(torch.linalg.norm(ue - ref)) / nref
    # CN: halve the step from 200 Delta t_CFL until its error matches the
    # exponential step's (GMRES tolerance well below that error), within a
    # budget of GPU time
    tried = []
    factor = 200.0
    spent = 0.0
    while True:
        uc, ms_c, mv_c, n_c = run("cn", factor, gmres_tol=min(1e-10, 1e-2 * err_e))
        spent += ms_c
        err_c = float(torch.linalg.norm(uc - ref)) / nref
        tried.append({"dt_over_cfl": factor, "steps": n_c, "err": err_c, "ms": round(ms_c, 3),
                      "matvecs": mv_c})
        if err_c <= err_e or spent > cn_budget_ms:
            break
        factor /= 2.0
    # penalised IMEX Euler (first order): step sizes from 200 Delta t_CFL down by 4
    pen = []
    for factor in (200.0, 50.0, 12.5, 3.125):
        up, ms_p, mv_p, n_p = run("penalised", factor)
        pen.append({"dt_over_cfl": factor, "err": float(torch.linalg.norm(up - ref)) / nref,
                    "ms": round(ms_p, 3), "matvecs": mv_p})
    op.close()
    best = tried[-1]
    # the matched pair: the cheapest CN run at or below the exponential's
    # error (when the budget allowed one)
    return {"workload": "c1-512sq-dirichlet-circular", "T_over_cfl": T_cfl,
            "penalised_imex": pen, "penalty_beta": beta,
            "exp": {"dt_over_cfl": 200.0, "steps": n_e, "err": err_e, "ms": round(ms_e, 3),
                    "matvecs": mv_e},
            "cn_tried": tried, "cn_matched": best["err"] <= err_e,
            "speedup_exp_over_cn": round(best["ms"] / ms_e, 2),
            "matvec_ratio_cn_over_exp": round(best["matvecs"] / mv_e, 2)}


def measure_cn_same_steps_c0(ad, dev, stream, n_steps=10):
    """Crank-Nicolson (GMRES, tol 1e-10) on the same ten steps of 100
    Delta t_CFL as the exponential midpoint rule (Leja tol 1e-10) on the 64^2
    periodic workload.  Its source does not depend on time, so the midpoint
    rule is exact up to the Leja tolerance and one exponential step over the
    whole interval gives the same state: the reference is that single step at
    tol 1e-12, and the ten-step run at tol 1e-12 is reported beside it as a
    check of the exactness."""
    import torch
    p = problem("c0-64sq-periodic-uniform30-midpoint")
    g = p.grid
    T = _dev_f64(dev)
    op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), p.ax, p.ay, ad.FP64,
                            stream=stream)
    src = ad.Source([T(gk) for gk in p.source.g], list(p.source.h))
    ad.reserve_gmres(op, 50)

    def run(method, n, dt, tol=1e-10):
        u = T(p.u0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mv = 0
        for k in range(n):
            if method == "cn":
                st = ad.cn_step(op, u, k * dt, dt, src, gmres_tol=1e-10, restart=50)
            else:
                st = ad.expquad_step(op, u, k * dt, dt, 1, (0.5,), src, tol=tol)
            mv += st["matvecs"]
        e1.record(stream)
        torch.cuda.synchronize()
        return u, e0.elapsed_time(e1), mv

    t_end = n_steps * p.dt
    ref, _, _ = run("exp", 1, t_end, tol=1e-12)
    nref = float(torch.linalg.norm(ref))
    ref10, _, _ = run("exp", n_steps, p.dt, tol=1e-12)
    ue, ms_e, mv_e = run("exp", n_steps, p.dt)
    uc, ms_c, mv_c = run("cn", n_steps, p.dt)
    op.close()
    err = lambda u: float(torch.linalg.norm(u - ref)) / nref
    return {"workload": "c0-64sq-periodic-uniform30-midpoint", "steps": n_steps,
            "dt_over_cfl": 100.0,
            "reference": "one exponential step of the whole interval, tol 1e-12",
            "ten_steps_vs_one_step_tol1e-12": err(ref10),
            "exp": {"err": err(ue), "ms": round(ms_e, 3), "matvecs": mv_e},
            "cn": {"err": err(uc), "ms": round(ms_c, 3), "matvecs": mv_c},
            "err_ratio_cn_over_exp": round(err(uc) / max(err(ue), 1e-300), 1)}


def measure_paper_cases(ad, dev, stream, nx=128):
    """The paper's work-precision experiments (Section 3, Figs. 3-5) on this
    implementation: error against a reference vs matrix-vector products (the
    paper's cost measure) and GPU time.  Cases I (ring) and II (spiral 2 with
    advection and time-independent sources): one exponential step of the
    whole interval T at tolerances 1e-2 .. 1e-10, against Crank-Nicolson with
    N steps.  Cases III and IV (spirals with time-dependent sources):
    exponential midpoint and two-stage Gauss quadrature with N steps (tol
    1e-10) against CN.  References: the exponential step at tol 1e-13 (I, II),
    Gauss with 64 steps at tol 1e-12 (III, IV).  FP64, Gershgorin bounds."""
    import numpy as np
    import torch
    from workloads.configs import paper_case
    gauss = (0.5 - 0.5 / 3 ** 0.5, 0.5 + 0.5 / 3 ** 0.5)
    out = {}
    for case in ("I", "II", "III", "IV"):
        p = paper_case(case, nx)
        g = p.grid
        T_end = p.dt
        Tt = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(),
                                       device=dev)
        op = ad.create_operator(g.nx, g.ny, g.bc, Tt(p.Dxx), Tt(p.Dxy), Tt(p.Dyy), p.ax, p.ay,
                                ad.FP64, stream=stream)
        src = ad.Source([Tt(gk) for gk in p.source.g], list(p.source.h)) if len(p.source) else None
        ad.reserve_gmres(op, 50)

        def run(method, nsteps, tol):
            dt = T_end / nsteps
            u = Tt(p.u0)
            mv, ok = 0, True
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            try:
                for k in range(nsteps):
                    if method == "cn":
                        st = ad.cn_step(op, u, k * dt, dt, src, gmres_tol=1e-10, restart=50)
                    elif method == "gauss":
                        st = ad.expquad_step(op, u, k * dt, dt, 2, gauss, src, tol=tol)
                    else:
                        st = ad.expquad_step(op, u, k * dt, dt, 1, (0.5,), src, tol=tol)
                    mv += st["matvecs"]
            except ad.AdError:
                ok = False
            e1.record(stream)
            torch.cuda.synchronize()
            return u, e0.elapsed_time(e1), mv, ok

        points = []
        if case in ("I", "II"):
            ref, _, _, _ = run("midpoint", 1, 1e-13)
            nref = float(torch.linalg.norm(ref))
            for tol in (1e-2, 1e-4, 1e-6, 1e-8, 1e-10):
                u, ms, mv, ok = run("midpoint", 1, tol)
                points.append({"method": "exp", "steps": 1, "tol": tol, "matvecs": mv,
                               "ms": round(ms, 3), "converged": ok,
                               "err": float(torch.linalg.norm(u - ref)) / nref})
            for nsteps in (8, 32, 128):
                u, ms, mv, ok = run("cn", nsteps, 0.0)
                points.append({"method": "cn", "steps": nsteps, "matvecs": mv, "ms": round(ms, 3),
                               "converged": ok, "err": float(torch.linalg.norm(u - ref)) / nref})
        else:
            ref, _, _, _ = run("gauss", 64, 1e-12)
            nref = float(torch.linalg.norm(ref))
            for method in ("midpoint", "gauss"):
                for nsteps in (1, 2, 4, 8, 16):
                    u, ms, mv, ok = run(method, nsteps, 1e-10)
                    points.append({"method": method, "steps": nsteps, "matvecs": mv,
                                   "ms": round(ms, 3), "converged": ok,
                                   "err": float(torch.linalg.norm(u - ref)) / nref})
            for nsteps in (8, 32, 128):
                u, ms, mv, ok = run("cn", nsteps, 0.0)
                points.append({"method": "cn", "steps": nsteps, "matvecs": mv, "ms": round(ms, 3),
                               "converged": ok, "err": float(torch.linalg.norm(u - ref)) / nref})
        out[case] = {"workload": p.name, "T": T_end, "T_over_cfl": round(T_end / p.cfl, 1),
                     "points": points}
        op.close()
    return out


def _slice_operators(ad, dev, stream, nslices, sides):
    """The momentum-slice batch: per slice a side drawn from ``sides`` (seed 3),
    D_par = p^0.5 for p log-spaced in [1, 1e4], D_perp = 1e-3 D_par, circular
    b, a = (0.05, 0), constant Gaussian source, Gaussian initial field."""
    import numpy as np
    import torch
    from workloads import config3_slices, slice_problem
    specs = config3_slices(nslices, sides=sides)
    ops, us, srcs, probs, fields = [], [], [], [], []
    for side, dpar, dperp in specs:
        p = slice_problem(side, dpar, dperp, dt=1.0)
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=dev)
        D = (T(p.Dxx), T(p.Dxy), T(p.Dyy))
        op = ad.create_operator(side, side, p.grid.bc, *D, 0.05, 0.0, ad.FP32_STORAGE, stream=stream)
        ops.append(op)
        us.append(T(p.u0).float())
        srcs.append(ad.Source([T(p.source.g[0]).float()], None))
        probs.append(p)
        fields.append(D)
    return ops, us, srcs, probs, fields


def _batched_oracle_slice(spec):
    """One slice of the batch on the CPU oracle (worker of a spawned pool):
    the operator, a 30-step power-iteration bound from the SplitMix64 start
    of the GPU side, then one exponential-midpoint step at tol 1e-6, timed;
    untimed, the same step at tol 1e-10 from the FP32-rounded initial field
    the GPU starts from (the reference its first step is compared with)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import integrators, spectral
    from oracle import operator as oop
    from workloads import slice_problem
    side, dpar, dperp, dt, seed = spec
    p = slice_problem(side, dpar, dperp, dt=dt)
    A = oop.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    alpha, _ = spectral.power_iteration(A, spectral.splitmix64_uniform(p.grid.n, seed),
                                        iters=30, safety=1.1)
    S = lambda t: p.source_at(t).ravel()
    t0 = time.perf_counter()
    integrators.expquad_step(A, p.u0.ravel(), 0.0, dt, 1, (0.5,), S, alpha, tol=1e-6)
    secs = time.perf_counter() - t0
    u32 = p.u0.ravel().astype(np.float32).astype(np.float64)
    S32 = lambda t: p.source_at(t).ravel().astype(np.float32).astype(np.float64)
    ref, _ = integrators.expquad_step(A, u32, 0.0, dt, 1, (0.5,), S32, alpha, tol=1e-10)
    return p.grid.n, secs, seed - 1, ref


def batched_oracle_baseline(specs, dt, max_side=512):
    """The CPU oracle on the batch's slices of side <= max_side, one step
    each, in a spawned process pool over every host core (one BLAS thread
    per worker).  Throughput = cells stepped / (sum of step seconds /
    workers): the pool's aggregate rate with every core busy."""
    import concurrent.futures as cf
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    workers = os.cpu_count() or 1
    jobs = [(side, dpar, dperp, dt, k + 1) for k, (side, dpar, dperp) in enumerate(specs)
            if side <= max_side]
    t0 = time.perf_counter()
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_batched_oracle_slice, jobs))
    wall = time.perf_counter() - t0
    cells = sum(r[0] for r in res)
    secs = sum(r[1] for r in res)
    refs = {r[2]: r[3] for r in res}
    return refs, {"value": round(cells / (secs / workers) / 1e6, 4), "unit": "Mcell-steps/s",
            "cores": workers, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(jobs)} of {len(specs)} slices (sides <= {max_side}), one "
                      f"exponential-midpoint step each at tol 1e-6, {workers} spawned workers "
                      f"(one core each); {secs:.1f} s of step time, {wall:.1f} s wall "
                      f"including operator assembly"}


def measure_batched_form(ad, dev, stream, steps, nslices=128, sides=(256, 512, 1024, 2048),
                         learned_fields=0, cpu_baseline=True):
    """The 128-slice batch (FP32 storage, tol 1e-6): one graph launch per step
    against the same slices stepped one operator call at a time; optionally the
    learned spectral bound against power iteration."""
    import numpy as np
    import torch
    t_setup = time.perf_counter()
    ops, us, srcs, probs, fields = _slice_operators(ad, dev, stream, nslices, sides)
    setup_s = time.perf_counter() - t_setup
    # bounds: power iteration per slice (timed), dt = 100 Delta t_CFL of the stiffest slice
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, op in enumerate(ops):
        ad.spectral_bound(op, ad.BOUND_POWER, seed=k + 1, power_iters=30, safety=1.1)
    torch.cuda.synchronize()
    power_s = time.perf_counter() - t0
    dt = 100.0 * min(p.cfl for p in probs)
    cells = sum(p.grid.n for p in probs)
    batch = ad.create_batch(ops, autotune=True)
    info = ad.batch_info(batch)
    u_start = [u.clone() for u in us]
    ad.batch_bind(batch, us, srcs)          # the vectors and sources every step advances
    ad.batch_step(batch, 0.0, dt, tol=1e-6)      # warm-up
    torch.cuda.synchronize()
    # the first step of the slices the CPU baseline also steps, for its error
    step1 = {k: us[k].double().cpu().numpy() for k, p in enumerate(probs) if p.grid.nx <= 512}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    torch.cuda.profiler.start()       # the range a profiler started with capture off records
    ev0.record(stream)
    for k in range(steps):
        st = ad.batch_step(batch, (k + 1) * dt, dt, tol=1e-6)
        iters.append(sum(s["iters"] for s in st))
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    ms_batch = ev0.elapsed_time(ev1) / steps
    # the same slices, one operator call each
    u2 = [u.clone() for u in u_start]
    for op, u, src in zip(ops, u2, srcs):
        ad.expquad_step(op, u, 0.0, dt, 1, (0.5,), src, tol=1e-6)
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(steps):
        for op, u, src in zip(ops, u2, srcs):
            ad.expquad_step(op, u, (k + 1) * dt, dt, 1, (0.5,), src, tol=1e-6)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_seq = ev0.elapsed_time(ev1) / steps
    # the plain FP64 GPU method on the same slices (one call per slice, the
    # same bounds, steps and tolerance): the batch's speedup at the accuracy
    # both reach, and how far the batch's FP32 states are from the FP64 ones
    ops64, u64, srcs64 = [], [], []
    for op, D, p, u0, src in zip(ops, fields, probs, u_start, srcs):
        o = ad.create_operator(p.grid.nx, p.grid.ny, p.grid.bc, *D, 0.05, 0.0, ad.FP64,
                               stream=stream)
        ad.set_spectral_bound(o, ad.get_spectral_bound(op))
        ops64.append(o)
        u64.append(u0.double())
        srcs64.append(ad.Source([src.g[0].double()], None))
    for o, u, src in zip(ops64, u64, srcs64):
        ad.expquad_step(o, u, 0.0, dt, 1, (0.5,), src, tol=1e-6)
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(steps):
        for o, u, src in zip(ops64, u64, srcs64):
            ad.expquad_step(o, u, (k + 1) * dt, dt, 1, (0.5,), src, tol=1e-6)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_fp64 = ev0.elapsed_time(ev1) / steps
    err_fp64 = max(float(torch.linalg.vector_norm(a.double() - b) / torch.linalg.vector_norm(b))
                   for a, b in zip(us, u64))
    for o in ops64:
        o.close()
    del ops64, u64, srcs64
    torch.cuda.empty_cache()
    # algorithmic HBM bytes of the iteration passes: 28 B per cell and iteration
    per_slice_iters = [s["iters"] for s in st]
    # one pass over a slice moves 28 B per cell (y, p read and written, three
    # coefficient fields read); the two-iteration kernel makes one pass per
    # two iterations (the default; AD_F32_PAIR=0 selects one per iteration)
    pair = os.environ.get("AD_F32_PAIR", "1")[:1] != "0"
    passes = [(it + 1) // 2 if pair else it for it in per_slice_iters]
    pass_bytes = sum(28.0 * p.grid.n * n for p, n in zip(probs, passes))
    equiv_bytes = sum(28.0 * p.grid.n * it for p, it in zip(probs, per_slice_iters))
    out = {"workload": f"c3-{nslices}-slices-sides{'-'.join(map(str, sides))}-fp32-midpoint",
           "cells": cells, "value": round(cells / (ms_batch * 1e-3) / 1e6, 2),
           "unit": "Mcell-steps/s", "ms_per_step": round(ms_batch, 4),
           "sequential_ms_per_step": round(ms_seq, 4),
           "speedup_vs_one_call_per_slice": round(ms_seq / ms_batch, 3),
           "plain_fp64": {"ms_per_step": round(ms_fp64, 4), "tol": 1e-6,
                          "speedup_batch_over_plain_fp64": round(ms_fp64 / ms_batch, 3),
                          "max_slice_rel_l2_batch_vs_fp64": err_fp64,
                          "note": "one FP64 call per slice, same bounds, steps and tolerance"},
           "leja_iters_per_slice": {"min": int(min(per_slice_iters)), "max": int(max(per_slice_iters)),
                                    "mean": round(float(np.mean(per_slice_iters)), 1)},
           "alg_GBps_iteration_passes": round(pass_bytes / (ms_batch * 1e-3) / 1e9, 1),
           "GBps_one_pass_per_iteration_equivalent":
               round(equiv_bytes / (ms_batch * 1e-3) / 1e9, 1),
           "bandwidth_note": "bytes of the iteration passes only (28 B per cell and pass) "
                             "over the whole step time, which also holds the apply, "
                             "series start, update and the tail of slow slices",
           "autotune": info, "power_iteration_bounds_s": round(power_s, 4),
           "setup_s": round(setup_s, 1), "tol": 1e-6}
    if cpu_baseline:
        from workloads import config3_slices
        refs, out["cpu_baseline"] = batched_oracle_baseline(config3_slices(nslices, sides=sides),
                                                            dt)
        errs = [float(np.linalg.norm(step1[k] - r) / np.linalg.norm(r)) for k, r in refs.items()]
        mx = [float(np.max(np.abs(step1[k] - r)) / np.max(np.abs(r))) for k, r in refs.items()]
        out["err_vs_oracle_step1"] = {
            "slices": len(errs), "max_rel_l2": max(errs), "median_rel_l2": float(np.median(errs)),
            "max_rel_max": max(mx),
            "note": "the batch's first step (FP32 storage, tol 1e-6) of every slice of side "
                    "<= 512 against the FP64 oracle's step at tol 1e-10 from the same "
                    "FP32-rounded field, same power-iteration start"}
    if learned_fields:
        out["learned"] = measure_learned(ad, dev, stream, ops, us, u_start, srcs, probs, fields,
                                         dt, batch, steps, ms_batch, power_s, learned_fields,
                                         ms_fp64=ms_fp64)
    for op in ops:
        op.close()
    return out


def measure_learned(ad, dev, stream, ops, us, u_start, srcs, probs, fields, dt, batch, steps,
                    ms_batch, power_s, nfields, margin=1.1, ms_fp64=None):
    """Train the bound network on generated fields (inputs and labels from
    ad_bound_training_sample: power-iteration spectra and Leja iteration
    counts; sides 64..2048, D_par in [1, 100], dt in [10, 1000] Delta t_CFL),
    hold out a tenth as many fields, then set every slice's bound with one
    batched inference (ad_learned_bounds) and run the batch with fallback.
    The comparison with power-iteration bounds counts bound time plus
    ``steps`` batched steps on both sides."""
    import numpy as np
    import torch
    from paper_2307_12276_gb300 import learned
    nhold = max(1, nfields // 10)
    t0 = time.perf_counter()
    X, Y = learned.build_dataset(nfields + nhold, seed=4, device=dev,
                                 workers=min(16, os.cpu_count() or 1))
    label_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    model = learned.train_bound_model(X[:nfields], Y[:nfields], dev, epochs=3000, lr=3e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    hold = model.predict(torch.as_tensor(X[nfields:], device=dev)).cpu().numpy()
    alpha_err = np.abs(np.exp(hold[:, 0] - Y[nfields:, 0]) - 1.0)
    iters_err = np.abs(np.exp(hold[:, 1] - Y[nfields:, 1]) - 1.0)   # the second output
    sides = np.round(np.exp(-X[:, 3].astype(np.float64)) * 2.0).astype(int)
    power_alpha = [ad.get_spectral_bound(op) for op in ops]
    # bounds for the slices: one batched inference from the features the
    # operators recorded at creation
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    alpha, it_pred = learned.predict_bounds(model, ops, dt, margin=margin, batch=batch)
    torch.cuda.synchronize()
    predict_s = time.perf_counter() - t0
    for s in range(len(us)):
        us[s].copy_(u_start[s])
    # warm-up step (the plain batch had one too), then the timed steps
    learned.batched_step_with_fallback(batch, ops, us, 0.0, dt, srcs, tol=1e-6)
    fallbacks = 0
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    iters = []
    for k in range(steps):
        st, fb = learned.batched_step_with_fallback(batch, ops, us, (k + 1) * dt, dt, srcs,
                                                    tol=1e-6)
        fallbacks += len(fb)
        iters.append(sum(s["iters"] for s in st))
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_learned = ev0.elapsed_time(ev1) / steps
    for op, a in zip(ops, power_alpha):
        ad.set_spectral_bound(op, a)
    plain_total = power_s + steps * ms_batch * 1e-3
    learned_total = predict_s + steps * ms_learned * 1e-3
    ratio = np.asarray(alpha) / np.asarray(power_alpha)
    actual = np.array([max(s["iters"], 1) for s in st], dtype=np.float64)
    slice_iters_err = np.abs(np.asarray(it_pred, dtype=np.float64) / actual - 1.0)
    return {"training_fields": nfields, "heldout_fields": nhold,
            "training_sides": {str(k): int(v) for k, v in
                               zip(*np.unique(sides[:nfields], return_counts=True))},
            "label_s": round(label_s, 1), "train_s": round(train_s, 2),
            "heldout_iters_rel_err_median": round(float(np.median(iters_err)), 4),
            "slice_iters_pred_rel_err_median": round(float(np.median(slice_iters_err)), 4),
            "heldout_alpha_rel_err_median": round(float(np.median(alpha_err)), 4),
            "heldout_alpha_rel_err_p90": round(float(np.quantile(alpha_err, 0.9)), 4),
            "margin": margin, "bounds_s": round(predict_s, 4),
            "power_iteration_bounds_s": round(power_s, 4),
            "ms_per_step": round(ms_learned, 4), "power_bound_ms_per_step": round(ms_batch, 4),
            "fallback_rate": round(fallbacks / (steps * len(ops)), 4),
            "pred_over_power_alpha": {"mean": round(float(ratio.mean()), 3),
                                      "min": round(float(ratio.min()), 3),
                                      "max": round(float(ratio.max()), 3)},
            "speedup_vs_power_iteration_bounds": round(plain_total / learned_total, 3),
            "speedup_over_plain_fp64_gpu": (
                round((power_s + steps * ms_fp64 * 1e-3) / learned_total, 3)
                if ms_fp64 else None),
            "speedup_note": "bound time plus the steps; plain FP64 GPU: power-iteration bounds "
                            "and one FP64 call per slice at tol 1e-6",
            "steps_in_comparison": steps}


def job_throughput(dev_ms, cells, steps, world, device):
    """Whole-job throughput of `world` replicas: every rank advanced `cells`
    cells by `steps` steps; the job took as long as its slowest rank (max
    over ranks).  Returns (max ms, Mcell-steps/s over all ranks)."""
    import torch
    import torch.distributed as dist
    tmax = torch.tensor([float(dev_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    ms = float(tmax.item())
    return ms, cells * steps * world / (ms * 1e-3) / 1e6


def _rel_errors(got, ref):
    import numpy as np
    d = np.asarray(got, dtype=np.float64) - ref
    return {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)),
            "rel_max": float(np.max(np.abs(d)) / np.max(np.abs(ref)))}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    # the oracle runs beside the GPU work in its own process (one core); its
    # first step from u0 is the reference for the errors reported below
    oracle_proc = None
    ref_npy = os.path.join(tempfile.gettempdir(), f"anidiff_oracle_step1_{os.getpid()}.npy")
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.nx:
        oracle_proc = start_oracle_sample(args.workload, args.cpu_sample_seconds, 10 ** 6,
                                          ref_npy)

    import paper_2307_12276_gb300 as ad
    w = WORKLOADS[args.workload]
    p = problem(args.workload, args.nx)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    label = args.workload if not args.nx else f"{args.workload} at {args.nx}^2"
    head, u1 = measure_workload(ad, dev, stream, p, flush, args.steps, args.warmup,
                                args.e2e_steps, world=world, label=label,
                                dt_over_cfl=w["dt_over_cfl"])

    forms = {}
    fp32_u1 = None
    wanted = set() if args.no_forms or rank != 0 else set(args.forms.split(","))
    if "fp32" in wanted:
        forms["fp32_4096sq"], fp32_u1 = measure_fp32_form(
            ad, dev, stream, flush, args.form_steps,
            p if w["kind"] == "c2" and not args.nx else None)
        if w["kind"] == "c2" and not args.nx:
            forms["fp32_4096sq"]["speedup_over_fp64_path"] = round(
                forms["fp32_4096sq"]["value"] / head["value"], 2)
            # the same comparison at equal tolerance: the FP64 path at tol 1e-6
            try:
                same = measure_fp64_at_tol(ad, dev, stream, flush, args.form_steps, p, 1e-6)
                same["speedup_of_fp32_form"] = round(
                    forms["fp32_4096sq"]["value"] / same["value"], 2)
            except Exception as exc:   # a side figure: never costs the line
                same = {"error": repr(exc)[:300]}
            forms["fp32_4096sq"]["fp64_path_same_tol"] = same
    if w["kind"] == "c2":
        del p
    for key, name in (("c1", "c1-512sq-dirichlet-circular-expquad2-dt200cfl"),
                      ("c0", "c0-64sq-periodic-uniform30-midpoint")):
        if key in wanted and name != args.workload:
            r, _ = measure_workload(ad, dev, stream, problem(name), flush, 20, 3, 9, label=name,
                                    dt_over_cfl=WORKLOADS[name]["dt_over_cfl"])
            r["value"] = round(r["value"], 2)
            if key == "c0":
                r["cn_same_steps"] = measure_cn_same_steps_c0(ad, dev, stream)
            forms[f"{key}_fp64"] = r
    if "cn" in wanted:
        forms["cn_vs_exp"] = measure_cn_vs_exp(ad, dev, stream)
    if "momentum" in wanted:
        forms["momentum"] = measure_momentum_form(ad, dev, stream)
    if "adaptive" in wanted:
        forms["adaptive_substeps"] = measure_adaptive_substeps(ad, dev, stream)
    if "paper" in wanted:
        forms["paper_cases"] = measure_paper_cases(ad, dev, stream)
    if "batched" in wanted:
        forms["batched"] = measure_batched_form(
            ad, dev, stream, args.form_steps,
            learned_fields=args.learned_fields if "learned" in wanted else 0,
            cpu_baseline=not args.no_cpu_baseline)

    cpu, err, err32 = None, None, None
    if oracle_proc is not None:
        cpu = finish_oracle_sample(oracle_proc)
        if os.path.exists(ref_npy):
            ref = np.load(ref_npy)
            os.remove(ref_npy)
            err = _rel_errors(u1, ref)
            err["oracle_iters"] = cpu.get("first_step_iters")
            err["gpu_iters"] = head["first_step_iters"]
            if fp32_u1 is not None and w["kind"] == "c2":
                err32 = _rel_errors(fp32_u1, ref)
                forms["fp32_4096sq"]["err_vs_oracle_step1"] = err32
                forms["fp32_4096sq"]["err_note"] = (
                    "one FP32 step (tol 1e-6) from u0 against the FP64 oracle's step (tol "
                    "1e-10), every cell")

    if rank == 0:
        line = {
            "metric": "Mcell-steps/s", "value": round(head["value"], 4), "unit": "Mcell-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(head["dev_ms"] / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": head["config"],
            "leja_iters_per_step": head["leja_iters_per_step"],
            "err_vs_oracle_step1": err,
            "gpu_launches": head["gpu_launches"],
            "e2e": head["e2e"],
            "roofline": head["roofline"],
            "clocks": head["clocks"],
        }
        if forms:
            line["forms"] = forms
        if cpu is not None:
            line["cpu_baseline"] = {
                "value": round(cpu["value"], 6), "unit": "Mcell-steps/s", "cores": 1,
                "host_cores": os.cpu_count(), "kind": "oracle",
                "sample": f"{cpu['steps']} exponential step(s) of the same workload from t=0 "
                          f"({cpu['seconds']:.1f} s timed; operator assembly "
                          f"{cpu['setup_s']:.0f} s untimed), run beside the GPU measurements"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
