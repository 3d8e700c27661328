#!/usr/bin/env python
"""Benchmark of the exponential Leja integrator on one GB300 (or N replicas).

Workload (default): 512 x 512 cell-centred grid on [-1, 1]^2, zero Dirichlet
boundaries, FP64, circular field lines (isotropic blend for r < 0.05),
D_par = 1, D_perp = 1e-4, a = (0.1, 0.05), S = Gaussian(sigma 0.05 at
(0.3, 0.3)) (1 + sin 2 pi t), two-stage exponential quadrature with
c = (1/3, 2/3), tol 1e-10, dt = 200 Delta t_CFL.  One benchmark step = one
exponential quadrature step (A u, the augmented Leja series, the update).

Metric: Mcell-steps/s = cells x steps / time.  ``value`` is device time
(CUDA events on the operator's stream, inputs resident, L2 flushed before
every step by writing a 256 MiB buffer); ``e2e`` is the same metric through
the C ABI with the state in pinned host memory (host->device and
device->host copies inside the timed region).  ``roofline`` reports the
fused Leja iteration kernel; ``cpu_baseline`` times the FP64 CPU oracle on
a bounded sample of the same workload in a subprocess.

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
    # name: (config builder kwargs, integrator)
    "c1-512sq-dirichlet-circular-expquad2-dt200cfl": dict(nx=512, dt_factor=200.0),
}
DEFAULT_WORKLOAD = "c1-512sq-dirichlet-circular-expquad2-dt200cfl"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--form-steps", type=int, default=5)
    return ap.parse_args()


def problem(name):
    from workloads import config1
    return config1(**WORKLOADS[name])


# --------------------------------------------------------------------------- oracle leg
def oracle_sample(workload: str, seconds: float, max_steps: int, out_npy: str | None,
                  warmup: int = 0):
    """Run the CPU oracle from the workload's initial state for about
    ``seconds`` (at least one step) after ``warmup`` untimed steps; returns a
    dict with its throughput."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
from bench import problem
from oracle import operator as oop, spectral, integrators
p = problem({workload!r})
A = oop.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
alpha = spectral.gershgorin(A)
S = lambda t: p.source_at(t).ravel()
u, t, steps, iters = p.u0.ravel().copy(), 0.0, 0, 0
for _ in range({warmup}):
    u, st = integrators.expquad_step(A, u, t, p.dt, p.s, p.c, S, alpha, tol=p.tol)
    t += p.dt
t0 = time.perf_counter()
while True:
    u, st = integrators.expquad_step(A, u, t, p.dt, p.s, p.c, S, alpha, tol=p.tol)
    t += p.dt; steps += 1; iters += st.iters
    if steps == 1 and {out_npy!r} is not None:
        np.save({out_npy!r}, u)
    el = time.perf_counter() - t0
    if el >= {seconds} or steps >= {max_steps}:
        break
print(json.dumps(dict(steps=steps, seconds=el, cells=p.grid.n, iters=iters, alpha=alpha)))
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-3000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    d["value"] = d["cells"] * d["steps"] / d["seconds"] / 1e6
    return d


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each of the K steps is one oracle step of the same workload (about 0.5 s each)
    d = oracle_sample(args.workload, seconds=1e9, max_steps=max(1, args.steps), out_npy=None,
                      warmup=args.warmup)
    line = {
        "impl": "reference", "metric": "Mcell-steps/s", "value": round(d["value"], 6),
        "unit": "Mcell-steps/s", "n_gpus": args.gpus, "steps": d["steps"],
        "ms_per_step": 1e3 * d["seconds"] / d["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "cells": d["cells"]}, "warmup": args.warmup,
        "cpu_baseline": {"value": round(d["value"], 6), "unit": "Mcell-steps/s", "cores": 1,
                         "kind": "oracle",
                         "sample": f"{d['steps']} full exponential quadrature steps from t=0"},
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


def traffic_per_launch(kernel_file: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    or None when the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "leja_iter_traffic.json")
    try:
        d = json.load(open(path))
    except (FileNotFoundError, ValueError):
        return None
    sha = hashlib.sha256(open(kernel_file, "rb").read()).hexdigest()
    if d.get("source_sha256") != sha:
        return None
    return d.get("dram_bytes_per_launch_full_size")


# --------------------------------------------------------------------------- ours
def measure_fp32_form(ad, dev, stream, flush, steps):
    """The FP32-storage form on the 4096^2 stream-function workload
    (exponential midpoint, tol 1e-6): throughput, Leja iterations and the
    fused FP32 kernel's algorithmic HBM bandwidth against the copy peak."""
    import numpy as np
    import torch
    from workloads import config2
    p = config2(nx=4096)
    g = p.grid
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=dev)
    op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), 0.0, 0.0,
                            ad.FP32_STORAGE, stream=stream)
    src = ad.Source([T(p.source.g[0]).float()], None)
    u = T(p.u0).float()
    t = 0.0
    for _ in range(2):
        ad.expquad_step(op, u, t, p.dt, 1, (0.5,), src, tol=p.tol)
        t += p.dt
    torch.cuda.synchronize()
    ms, iters = 0.0, []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ad.expquad_step(op, u, t, p.dt, 1, (0.5,), src, tol=p.tol)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        iters.append(st["iters"])
        t += p.dt
    ms_launch = ad.profile_leja_iteration(op, aug=0, reps=100)
    alg_bytes = 28.0 * g.n      # 3 fields + y + p r/w + y_next, 4 B each
    gbs = alg_bytes / (ms_launch * 1e-3) / 1e9
    op.close()
    del u, src
    torch.cuda.empty_cache()
    return {"workload": "c2-4096sq-dirichlet-stream-midpoint-fp32", "cells": g.n,
            "value": round(g.n * steps / (ms * 1e-3) / 1e6, 2), "unit": "Mcell-steps/s",
            "ms_per_step": round(ms / steps, 4), "leja_iters_per_step": statistics.mean(iters),
            "tol": p.tol, "dtype": "f32 storage/arithmetic, f64 Leja scalars and norm sums",
            "roofline": {"bound": "hbm", "kernel": "leja_iter_f32_k", "ms_per_launch":
                         round(ms_launch, 5), "achieved": round(gbs, 1), "peak": 6750.4,
                         "unit": "GB/s", "frac": round(gbs / 6750.4, 4),
                         "alg_bytes_per_launch": alg_bytes}}


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

    cpu = None
    ref_npy = os.path.join(tempfile.gettempdir(), f"anidiff_oracle_step1_{os.getpid()}.npy")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.workload, args.cpu_sample_seconds, 10 ** 6, ref_npy)

    import paper_2307_12276_gb300 as ad
    p = problem(args.workload)
    g = p.grid
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=dev)
    stream = torch.cuda.current_stream(dev)
    op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), p.ax, p.ay,
                            ad.FP64, stream=stream)
    src = ad.Source([T(gk) for gk in p.source.g], list(p.source.h))
    u0 = T(p.u0)
    u = u0.clone()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # first step from u0 (compared with the oracle's first step)
    st1 = ad.expquad_step(op, u, 0.0, p.dt, p.s, p.c, src, tol=p.tol)
    torch.cuda.synchronize()
    err = None
    if cpu is not None and os.path.exists(ref_npy):
        ref = np.load(ref_npy)
        err = float(np.linalg.norm(u.cpu().numpy() - ref) / np.linalg.norm(ref))
        os.remove(ref_npy)
    t = p.dt
    for _ in range(max(0, args.warmup - 1)):
        ad.expquad_step(op, u, t, p.dt, p.s, p.c, src, tol=p.tol)
        t += p.dt
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches, iters = 0, []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            st = ad.expquad_step(op, u, t, p.dt, p.s, p.c, src, tol=p.tol)
            ends[k].record(stream)
            launches += st["kernel_launches"]
            iters.append(st["iters"])
            t += p.dt
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    tmax = torch.tensor([dev_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dev_ms = float(tmax.item())
    value = g.n * args.steps * world / (dev_ms * 1e-3) / 1e6

    # e2e: the state lives in pinned host memory; the C ABI stages it per call
    uh = torch.empty(g.n, dtype=torch.float64, pin_memory=True)
    uh.copy_(u0.cpu())
    ue = uh.numpy()
    te = 0.0
    for k in range(args.e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ad.expquad_step(op, ue, k * p.dt, p.dt, p.s, p.c, src, tol=p.tol)
        el = time.perf_counter() - t0
        if k > 0:                       # the first call allocates the staging buffers
            te += el
    e2e_value = g.n * args.e2e_steps / te / 1e6

    # roofline of the fused (augmented) Leja iteration kernel
    ms_launch = ad.profile_leja_iteration(op, aug=1, reps=300)
    flops = 28.0 * g.n        # 14 FP64 FMA per cell: 9 stencil, shift, coupling, p, 2 norms
    bytes_alg = 112.0 * g.n   # 9 weights + y + w2 + p (r/w) + y_next, 8 B each
    achieved = flops / (ms_launch * 1e-3) / 1e12
    traffic = traffic_per_launch(os.path.join(ROOT, "paper_2307_12276_gb300", "csrc",
                                              "stencil_kernels.cu"))
    roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
            "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
            "traffic": traffic, "kernel": "leja_iter_f64_k<aug>",
            "ms_per_launch": round(ms_launch, 5),
            "alg_bytes_per_launch": bytes_alg,
            "alg_GBps": round(bytes_alg / (ms_launch * 1e-3) / 1e9, 1),
            "peak_note": "FP64: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (derived)"}

    forms = {}
    if not args.no_forms:
        forms["fp32_4096sq"] = measure_fp32_form(ad, dev, stream, flush, args.form_steps)

    if rank == 0:
        line = {
            "metric": "Mcell-steps/s", "value": round(value, 4), "unit": "Mcell-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dev_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nx": g.nx, "ny": g.ny, "cells": g.n,
                       "dt_over_cfl": 200.0, "s": p.s, "c": list(p.c), "tol": p.tol,
                       "l2": "flushed before every timed step (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "leja_iters_per_step": statistics.mean(iters),
            "err_vs_oracle_step1": err,
            "gpu_launches": launches,
            "e2e": {"value": round(e2e_value, 4), "unit": "Mcell-steps/s",
                    "h2d_bytes_per_step": 8 * g.n, "d2h_bytes_per_step": 8 * g.n},
            "roofline": roof,
            "clocks": clk.summary(),
        }
        if forms:
            line["forms"] = forms
        if cpu is not None:
            line["cpu_baseline"] = {"value": round(cpu["value"], 6), "unit": "Mcell-steps/s",
                                    "cores": 1, "kind": "oracle",
                                    "sample": f"{cpu['steps']} exponential quadrature steps of "
                                              f"the same workload from t=0 ({cpu['seconds']:.1f} s)"}
        print(json.dumps(line), flush=True)
    op.close()
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
