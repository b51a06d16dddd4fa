#!/usr/bin/env python3
"""Throughput of the fused LB stream-collide path on GB300: MLUPS and fraction
of the HBM roofline for FP32 storage (FP16/BF16 storage beside it), with the
Lorenz-Mie error of the far-field intensity it produces.

Workload: the 384^3 dielectric sphere (n = 1.33, x = 5, lambda = 30 cells,
x-polarised plane wave along +z, 16-cell absorbing layer).  One bench step is
one pass of the whole hot path: one DFT window of T = 3 lambda = 90 lattice
updates (pull streaming with the Eq. 4 boundary, TF/SF source, moments,
running FP64 DFT on the NTFF box, collision, absorbing layer) followed by the
near-to-far-field projection to |S(theta, phi)|^2 at 181 x 3 angles (an FP32
contraction with FP64 sums above chunks of face rows; the FP64-throughout
projection is timed beside it, outside the timed region).
The default 3 warm-up + 27 timed steps run the 30 periods of the workload, so
the last step's |S|^2 is the steady-state result compared with Mie.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lbem|reference]

N > 1 (launched under torchrun): independent replicas, one problem per GPU.
--impl reference times the FP64 CPU oracle on a bounded slab of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")
PROFILES = os.path.join(ROOT, "profiles")
METRIC = "MLUPS and % of HBM roofline at 1 GB300 (FP32 vs FP16 storage) at stated Mie error"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def b_cell(mode: str, storage: str) -> int:
    q = 42 if mode == "3d" else 21
    s = 4 if storage == "f32" else 2
    return 2 * q * s + 4


def kernel_source_hash() -> str:
    """Hash of the step kernels' source: step.cu, step2.cu, step_cell.cuh and
    the StepArgs definition."""
    csrc = os.path.join(ROOT, "paper_2510_11042_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("step.cu", "step2.cu", "step_cell.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    hdr = open(os.path.join(csrc, "lbem_internal.cuh")).read()
    i = hdr.index("struct StepArgs {")
    h.update(hdr[i:hdr.index("};", i)].encode())
    return h.hexdigest()[:16]


def traffic_from_profile(workload: str, storage: str):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when the kernel source changed since the counters were taken."""
    path = os.path.join(PROFILES, "step_kernel_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d[workload][storage]
        if e.get("kernel_hash") != kernel_source_hash():
            return None
        return float(e["bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def mie_reference():
    d = np.loadtxt(os.path.join(GOLDEN, "mie_sphere_x5_m1.33.txt"))
    return d[:, 1:4]  # [181][phi = 0, 45, 90]


def nrms(s, ref):
    """Eq. 13: RMS of the difference over the angles / max of the reference."""
    return float(np.sqrt(np.mean((s - ref) ** 2)) / np.max(ref))


def angles():
    th = np.radians(np.arange(181.0))
    return (np.concatenate([th, th, th]),
            np.concatenate([np.zeros(181), np.full(181, math.pi / 4), np.full(181, math.pi / 2)]))


# ------------------------------------------------------------------ GPU arm
def max_over_ranks(t_ms: float, world: int, device=None) -> float:
    """The job's time: the slowest rank's timed region (all-reduce MAX over the
    default process group; NCCL on GPUs, any backend works)."""
    if world == 1:
        return t_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(cells: int, updates_per_step: int, steps: int, world: int, t_ms: float) -> float:
    """Whole-job throughput: every rank advances its own replica of the
    workload, so the job updates cells x updates x steps x world sites."""
    return cells * updates_per_step * steps * world / (t_ms / 1e3) / 1e6


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2510_11042_gb300 import build as lib_build
    from paper_2510_11042_gb300 import lbem

    if rank == 0:
        lib_build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    lbem.lib()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    prob = W.sphere_problem(n=args.size)
    nx, ny, nz = prob.shape
    cells = nx * ny * nz
    T = prob.period
    theta, phi = angles()
    ref = mie_reference()
    results = {}

    def one_storage(storage, K, Wm, timed_main):
        solver = lbem.Solver(prob.shape, prob.eps, "3d", storage, prob.absorber_width,
                             prob.sigma_max, device=dev)
        solver.inject(prob.wave)
        h = solver.h
        stream = solver.stream
        steps_per_pass = solver.step_fusion()   # the kernel lbem_step takes, as the library reports it

        def bench_step(ev_pair=None):
            lbem.lbem_set_dft_window(h, solver.time + 1, 1)
            if ev_pair:
                ev_pair[0].record(stream)
            lbem.lbem_step(h, T)
            if ev_pair:
                ev_pair[1].record(stream)
            return lbem.lbem_far_field(h, theta, phi)

        for _ in range(Wm):
            bench_step()
        torch.cuda.synchronize(dev)
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(K)]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local_rank) if timed_main else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        launches0 = lbem.lbem_kernel_launches(h)
        torch.cuda.synchronize(dev)
        barrier()
        start.record(stream)
        s2 = None
        for k in range(K):
            s2 = bench_step(evs[k])
        end.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        clocks = sampler.stop() if sampler else None
        launches = lbem.lbem_kernel_launches(h) - launches0
        total_ms = start.elapsed_time(end)
        step_kernel_ms = sum(a.elapsed_time(b) for a, b in evs) / (K * T)
        s2 = s2.reshape(3, 181).T
        out = dict(total_ms=total_ms, ms_per_step=total_ms / K, kernel_ms=step_kernel_ms,
                   steps_per_pass=steps_per_pass,
                   launches=launches, clocks=clocks, periods=solver.time // T,
                   mie_nrms=[nrms(s2[:, j], ref[:, j]) for j in range(3)],
                   incident=lbem.lbem_incident_amplitude(h))
        # end-to-end: host (pinned) permittivity in, |S|^2 out, through the C ABI
        if timed_main:
            eps_host = torch.from_numpy(prob.eps).pin_memory()
            E = min(K, 3)
            torch.cuda.synchronize(dev)
            barrier()
            t0 = time.perf_counter()
            for _ in range(E):
                lbem.lbem_set_permittivity(h, eps_host)
                bench_step()          # ends with the |S|^2 copy to the host
            torch.cuda.synchronize(dev)
            barrier()
            t_e2e = (time.perf_counter() - t0) / E
            out["e2e_s_per_step"] = t_e2e
            out["h2d_bytes"] = int(prob.eps.nbytes + theta.nbytes + phi.nbytes)
            out["d2h_bytes"] = int(theta.size * 8)
            # the projection's two precisions on this window's DFT (outside the timed region)
            ff, vals = {}, {}
            for prec in ("mixed", "fp64"):
                lbem.lbem_set_far_field_precision(h, prec)
                lbem.lbem_far_field(h, theta, phi)
                t0 = time.perf_counter()
                for _ in range(3):
                    vals[prec] = lbem.lbem_far_field(h, theta, phi)
                ff[prec + "_ms_per_call"] = round((time.perf_counter() - t0) / 3 * 1e3, 3)
            lbem.lbem_set_far_field_precision(h, "mixed")
            d = vals["mixed"] - vals["fp64"]
            ff["rel_l2_mixed_vs_fp64"] = float(np.linalg.norm(d) / np.linalg.norm(vals["fp64"]))
            out["far_field"] = ff
        solver.close()
        del solver
        torch.cuda.empty_cache()
        return out

    K, Wm = args.steps, args.warmup
    main = one_storage("f32", K, Wm, True)
    probe_2d = None if (args.no_batch or world > 1) else run_probe_2d(dev)
    variants_3d = None if (args.no_batch or world > 1) else run_variants_3d(dev)
    in_place = None if (args.no_batch or world > 1) else run_in_place(dev, n=args.size)
    cyl_1024 = None if (args.no_batch or world > 1) else run_cylinder_1024(dev)
    batched = None if (args.no_batch or world > 1) else run_batched(dev)
    adjoint = None if (args.no_adjoint or world > 1) else run_adjoint(dev)
    secondary = {}
    if not args.fp32_only:
        for st in ("f16", "bf16"):
            secondary[st] = one_storage(st, K, Wm, False)

    # max over ranks of the timed region
    t_main = max_over_ranks(main["total_ms"], world, dev)
    if rank != 0:
        return
    hbm, peak_kind = peaks()
    two_step = main["steps_per_pass"] == 2
    value = job_mlups(cells, T, K, world, t_main)
    bc = b_cell("3d", "f32")
    achieved = bc * cells / (main["kernel_ms"] / 1e3) / 1e9
    traffic = traffic_from_profile(f"sphere_{args.size}", "f32")
    e2e_val = cells * T / main["e2e_s_per_step"] / 1e6 * world
    storage_modes = {"f32": {"mlups": round(value / world, 1),
                             "kernel_ms": round(main["kernel_ms"], 4),
                             "hbm_frac": round(achieved / hbm, 4),
                             "steps_per_pass": main["steps_per_pass"],
                             "mie_nrms_phi_0_45_90": [round(v, 5) for v in main["mie_nrms"]]}}
    for st, r in secondary.items():
        bcs = b_cell("3d", st)
        ach = bcs * cells / (r["kernel_ms"] / 1e3) / 1e9
        storage_modes[st] = {"mlups": round(cells * T * K / (r["total_ms"] / 1e3) / 1e6, 1),
                             "kernel_ms": round(r["kernel_ms"], 4),
                             "hbm_frac": round(ach / hbm, 4),
                             "speedup_vs_f32": round(main["kernel_ms"] / r["kernel_ms"], 3),
                             "mlups_vs_f32": round(cells * T * K / (r["total_ms"] / 1e3) / 1e6 / (value / world), 3),
                             "steps_per_pass": r["steps_per_pass"],
                             "mie_nrms_phi_0_45_90": [round(v, 5) for v in r["mie_nrms"]]}
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": K,
        "warmup": Wm,
        "ms_per_step": round(t_main / K, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"sphere_{args.size}^3_n1.33_x5_lambda30_W16_fp32_storage",
                   "cells": cells, "lattice_updates_per_step": T,
                   "step": "one DFT window (T = 90 updates) + NTFF at 543 angles",
                   "l2": "inputs larger than L2 (working set %.1f GB)" % (
                       (2 * 42 * 4 + 4) * cells / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 4), "traffic": traffic,
                     "peak_source": peak_kind,
                     "kernel": ("step2_kernel: two lattice updates per launch, populations read and "
                                "written once per launch" if two_step else "step_kernel_cell: one update"),
                     "units_per_launch": (2 if two_step else 1) * cells,
                     "algorithmic_bytes_per_launch": (2 if two_step else 1) * bc * cells},
        "e2e": {"value": round(e2e_val, 1), "unit": "MLUPS",
                "h2d_bytes_per_step": main["h2d_bytes"], "d2h_bytes_per_step": main["d2h_bytes"]},
        "gpu_launches": int(main["launches"]),
        "clocks": main["clocks"],
        "mie": {"nrms_phi_0_45_90": [round(v, 5) for v in main["mie_nrms"]],
                "periods_run": main["periods"], "incident_amplitude": round(main["incident"], 6)},
        "storage_modes": storage_modes,
        "far_field": dict(main["far_field"], angles=int(theta.size),
                          default="mixed: FP32 products, FP32 sums over <= 32 face rows and a 64-column "
                                  "tile, FP64 sums above"),
    }
    if probe_2d:
        line["bandwidth_probe_2d"] = probe_2d
    if variants_3d:
        line["kernel_variants_3d"] = variants_3d
    if in_place:
        line["in_place_streaming"] = in_place
    if cyl_1024:
        line["cylinder_1024"] = cyl_1024
    if batched:
        line["batched"] = batched
    if adjoint:
        line["adjoint"] = adjoint
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.size, budget_s=args.cpu_seconds)
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched workload
def small_problems(count=64, seed=7):
    """Launch-bound batch: cylinders of N = 64..192 (multiples of 32), W = 8,
    eps_r in [1.5, 6], x in [1, 3], lambda = 8..16 cells, 300 steps each."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = 32 * int(rng.integers(2, 7))
        lam = float(rng.integers(8, 17))
        x = float(rng.uniform(1.0, 3.0))
        eps_in = float(rng.uniform(1.5, 6.0))
        a = x * lam / (2 * math.pi)
        if 2 * a + 2 * (8 + 6) > n:
            continue
        p = W.cylinder_problem(n=n, x=x, wavelength=lam, eps_in=eps_in, w=8, mode="ez", periods=1,
                               gap_ntff=2, gap_tf=2)
        out.append(W.with_steps(p, 300))
    return out


def run_batched(dev, count=32, seed=20251011):
    """32 seeded cylinders (N = 256..1024, eps_r in [1.5, 6], x in [1, 10],
    lambda = 24..48 cells, W = 16, 40 periods each) in one persistent batched
    run (autotuned launch shape) and, for comparison, stepped one problem after
    another with one launch per step.  Aggregate MLUPS = sum(cells x steps) / s."""
    import torch
    from paper_2510_11042_gb300 import lbem
    out = {}
    mie = None
    if (count, seed) == (32, 20251011):
        mie = np.loadtxt(os.path.join(GOLDEN, "mie_batch_cylinders_seed20251011.txt"))[:, 1:]
    for label, probs in (("cylinders_256_1024", W.batched_problems(count, seed)),
                         ("small_64_192", small_problems())):
        out[label] = _batch_vs_sequential(dev, probs, mie if label == "cylinders_256_1024" else None)
    out["cylinders_256_1024"]["workload"] = (f"{count} cylinders, seed {seed}, N 256-1024, "
                                             "40 periods each, FP32, EZ")
    out["small_64_192"]["workload"] = "64 cylinders, seed 7, N 64-192, 300 steps each, FP32, EZ"
    return out


def _batch_vs_sequential(dev, probs, mie=None):
    """Persistent batched run against one problem after another; with mie
    ([181][problem] Lorenz-Mie TM |S|^2), also each batched problem's far
    field at theta = 0..180 deg against it (Eq. 13)."""
    import torch
    from paper_2510_11042_gb300 import lbem
    work = sum(p.shape[0] * p.shape[1] * p.steps for p in probs)

    def solvers():
        out = []
        for p in probs:
            s = lbem.Solver(p.shape, p.eps, p.mode, "f32", p.absorber_width, p.sigma_max, device=dev)
            s.inject(p.wave)
            s.set_dft_window(p.dft_start, p.dft_periods)
            out.append(s)
        torch.cuda.synchronize(dev)
        return out

    sol = solvers()
    batch = lbem.Batch(sol)
    t0 = time.perf_counter()
    batch.run([p.steps for p in probs], autotune=True)
    torch.cuda.synchronize(dev)
    t_batch = time.perf_counter() - t0
    bps, rpi, _, split = batch.config()
    batch.close()
    mie_nrms = None
    if mie is not None:
        th = np.radians(np.arange(181.0))
        mie_nrms = [round(nrms(s.far_field(th), mie[:, j]), 5) for j, s in enumerate(sol)]
    for s in sol:
        s.close()
    del sol
    torch.cuda.empty_cache()

    sol = solvers()
    t0 = time.perf_counter()
    for s, p in zip(sol, probs):
        s.step(p.steps)
    torch.cuda.synchronize(dev)
    t_seq = time.perf_counter() - t0
    for s in sol:
        s.close()
    del sol
    torch.cuda.empty_cache()
    out = {"cell_updates": work, "persistent_mlups": round(work / t_batch / 1e6, 1),
           "sequential_mlups": round(work / t_seq / 1e6, 1),
           "speedup": round(t_seq / t_batch, 3),
           "autotuned": {"blocks_per_sm": bps, "rows_per_item": rpi, "split": split}}
    if mie_nrms is not None:
        out["mie_nrms_per_problem"] = mie_nrms
        out["mie_nrms_max"] = max(mie_nrms)
        out["mie_nrms_median"] = float(np.median(mie_nrms))
        out["mie_reference"] = "tests/golden/mie_batch_cylinders_seed20251011.txt (TM, theta 0..180 deg)"
    return out


# ------------------------------------------------------------------ 2D bandwidth probe
def run_probe_2d(dev, n=4096, updates=60):
    """Step throughput of the 2D EZ path on a grid well above L2 (4096^2 x 21
    populations, 2.8 GB in FP32): a cylinder of the cylinder workload's
    proportions, CUDA events around `updates` lattice updates, with the pass
    lbem_step takes by default (two updates per pass where the library
    reports it) and with single steps.  hbm_frac is the byte model
    (B_cell per update) over the time per update."""
    import torch
    from paper_2510_11042_gb300 import lbem
    p = W.cylinder_problem(n=n, x=5.0, wavelength=40.0, eps_in=2.25, w=20, mode="ez", periods=1)
    hbm, _ = peaks()
    out = {"workload": f"cylinder {n}x{n} EZ, lambda 40, W 20", "cells": n * n}
    for st in ("f32", "f16", "bf16"):
        rec = {}
        for fuse in (2, 1):
            s = lbem.Solver(p.shape, p.eps, "ez", st, p.absorber_width, p.sigma_max, device=dev)
            s.set_step_fusion(fuse)
            s.inject(p.wave)
            s.step(10)
            torch.cuda.synchronize(dev)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(s.stream)
            s.step(updates)
            ev[1].record(s.stream)
            torch.cuda.synchronize(dev)
            ms = ev[0].elapsed_time(ev[1]) / updates
            bc = b_cell("ez", st)
            gbs = bc * n * n / (ms / 1e3) / 1e9
            rec[fuse] = {"kernel_ms": round(ms, 4), "mlups": round(n * n / (ms / 1e3) / 1e6, 1),
                         "bytes_per_cell": bc, "achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                         "steps_per_pass": s.step_fusion()}
            s.close()
            del s
            torch.cuda.empty_cache()
        out[st] = dict(rec[2], single_step=rec[1], speedup_vs_single_step=round(rec[1]["kernel_ms"] /
                                                                                rec[2]["kernel_ms"], 3))
        # the two-step kernel's own DRAM traffic (ncu, committed summary), over the time of its launch
        traffic = traffic_from_profile(f"cylinder_{n}_ez", st) if rec[2]["steps_per_pass"] == 2 else None
        if traffic:
            gbs_t = traffic / (2 * rec[2]["kernel_ms"] / 1e3) / 1e9
            out[st]["dram_traffic_per_launch"] = traffic
            out[st]["dram_traffic_gbs"] = round(gbs_t, 1)
            out[st]["dram_traffic_frac"] = round(gbs_t / hbm, 4)
    return out


# ------------------------------------------------------------------ the 1024^2 cylinder workload
def run_cylinder_1024(dev, updates=120):
    """Step throughput on the cylinder workload itself (1024^2, a = 31.83,
    eps_r = 2.25, W = 20, TM and TE) over one DFT window of 120 updates, with
    the pass lbem_step takes (single steps: two 1024^2 buffers stay in L2).
    The byte model's fraction is labelled L2-assisted where the working set is
    under three times the L2 size."""
    import torch
    from paper_2510_11042_gb300 import lbem
    hbm, _ = peaks()
    props = torch.cuda.get_device_properties(dev)
    l2 = int(getattr(props, "L2_cache_size", 0)) or None
    out = {"workload": "cylinder 1024^2, a 31.83, eps_r 2.25, lambda 40, W 20", "updates_timed": updates,
           "l2_bytes": l2}
    for mode in ("ez", "hz"):
        p = W.cylinder_problem(n=1024, x=5.0, wavelength=40.0, eps_in=2.25, w=20, mode=mode, periods=40)
        cells = int(np.prod(p.shape))
        for st in ("f32", "f16", "bf16"):
            s = lbem.Solver(p.shape, p.eps, mode, st, p.absorber_width, p.sigma_max, device=dev)
            s.inject(p.wave)
            s.step(10)
            s.set_dft_window(s.time + 1, 1)
            torch.cuda.synchronize(dev)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(s.stream)
            s.step(updates)
            ev[1].record(s.stream)
            torch.cuda.synchronize(dev)
            ms = ev[0].elapsed_time(ev[1]) / updates
            bc = b_cell(mode, st)
            gbs = bc * cells / (ms / 1e3) / 1e9
            working = (2 * (42 if mode == "3d" else 21) * (4 if st == "f32" else 2) + 4) * cells
            out[f"{mode}_{st}"] = {"kernel_ms": round(ms, 4), "mlups": round(cells / (ms / 1e3) / 1e6, 1),
                                   "bytes_per_cell": bc, "achieved_gbs": round(gbs, 1),
                                   "hbm_frac": round(gbs / hbm, 4), "steps_per_pass": s.step_fusion(),
                                   "working_set_mb": round(working / 1e6, 1),
                                   "label": ("L2-assisted" if l2 and working < 3 * l2 else "HBM")}
            s.close()
            del s
            torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ other step-kernel instantiations
def run_variants_3d(dev, updates=44, storages=("f32", "f16"), n=384):
    """The step kernel's other instantiations on the 384^3 sphere: single steps
    (lbem_set_step_fusion(1)), and with a mu_r map (mu_r = 2 in the sphere; 4
    more bytes per cell for 1/mu_r) and with the closed-form source at 30
    degrees, each with the pass lbem_step takes by default (two updates per
    pass where the library reports it) and with single steps."""
    import dataclasses
    import torch
    from paper_2510_11042_gb300 import lbem
    p = W.sphere_problem(n=n)
    cells = int(np.prod(p.shape))
    hbm, _ = peaks()
    th = math.radians(30.0)
    oblique = dataclasses.replace(p.wave, direction=(math.sin(th), 0.0, math.cos(th)),
                                  polarization=(math.cos(th), 0.0, -math.sin(th)), analytic=True,
                                  origin=tuple(float(v) for v in p.wave.tf_lo))
    out = {"workload": f"sphere {n}^3" + (" (the bench workload)" if n == 384 else "")}

    def timed(st, fuse, mu, wave, dft):
        s = lbem.Solver(p.shape, p.eps, "3d", st, p.absorber_width, p.sigma_max, device=dev)
        s.set_step_fusion(fuse)
        if mu:
            s.set_permeability(np.where(p.eps > 1.0, np.float32(2.0), np.float32(1.0)))
        s.inject(wave)
        s.step(6)
        if dft:   # like a bench step: the DFT window on
            s.set_dft_window(s.time + 1, 1)
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(s.stream)
        s.step(updates)
        ev[1].record(s.stream)
        torch.cuda.synchronize(dev)
        ms = ev[0].elapsed_time(ev[1]) / updates
        spp = s.step_fusion()
        s.close()
        del s
        torch.cuda.empty_cache()
        return ms, spp

    for st in storages:
        base = b_cell("3d", st)
        for name, mu, wave, bc, fuses in (("single_step", False, p.wave, base, (1,)),
                                           ("magnetic_mu2", True, p.wave, base + 4, (2, 1)),
                                           ("closed_form_source_30deg", False, oblique, base + 4, (2, 1))):
            rec = {}
            for fuse in fuses:
                ms, spp = timed(st, fuse, mu, wave, name == "single_step")
                gbs = bc * cells / (ms / 1e3) / 1e9
                rec[fuse] = {"kernel_ms": round(ms, 4), "mlups": round(cells / (ms / 1e3) / 1e6, 1),
                             "bytes_per_cell": bc, "achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4),
                             "steps_per_pass": spp}
            entry = dict(rec[fuses[0]])
            if len(fuses) == 2:
                entry["single_step"] = rec[1]
                entry["speedup_vs_single_step"] = round(rec[1]["kernel_ms"] / rec[2]["kernel_ms"], 3)
            out[name if st == "f32" else f"{name}_{st}"] = entry
    return out


def run_in_place(dev, updates=40, storages=("f32", "f16", "bf16"), n=384):
    """In-place streaming (one population buffer) on the sphere against the
    two-buffer single step it is bitwise equal to, both with the DFT window on,
    over an even number of updates (push and in-place steps alternate): CUDA
    event time per update, the B_cell byte model's bandwidth, and the
    workspace each scheme needs."""
    import torch
    from paper_2510_11042_gb300 import lbem
    p = W.sphere_problem(n=n)
    cells = int(np.prod(p.shape))
    hbm, _ = peaks()
    out = {"workload": f"sphere {n}^3" + (" (the bench workload)" if n == 384 else ""),
           "updates_timed": updates}

    def timed(st, streaming):
        s = lbem.Solver(p.shape, p.eps, "3d", st, p.absorber_width, p.sigma_max, device=dev, streaming=streaming)
        s.set_step_fusion(1)
        s.inject(p.wave)
        s.step(6)
        s.set_dft_window(s.time + 1, 1)
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(s.stream)
        s.step(updates)
        ev[1].record(s.stream)
        torch.cuda.synchronize(dev)
        ms = ev[0].elapsed_time(ev[1]) / updates
        ws = int(s.workspace.numel())
        s.close()
        del s
        torch.cuda.empty_cache()
        return ms, ws

    for st in storages:
        bc = b_cell("3d", st)
        rec = {}
        for streaming in ("in_place", "two_buffers"):
            ms, ws = timed(st, streaming)
            gbs = bc * cells / (ms / 1e3) / 1e9
            rec[streaming] = {"kernel_ms": round(ms, 4), "mlups": round(cells / (ms / 1e3) / 1e6, 1),
                              "bytes_per_cell": bc, "achieved_gbs": round(gbs, 1),
                              "hbm_frac": round(gbs / hbm, 4), "workspace_gb": round(ws / 1e9, 3)}
        entry = dict(rec["in_place"], two_buffers_single_step=rec["two_buffers"])
        entry["time_vs_two_buffers"] = round(rec["in_place"]["kernel_ms"] / rec["two_buffers"]["kernel_ms"], 3)
        entry["workspace_vs_two_buffers"] = round(rec["in_place"]["workspace_gb"] / rec["two_buffers"]["workspace_gb"], 3)
        out[st] = entry
    return out


# ------------------------------------------------------------------ adjoint workload
def run_adjoint(dev, K=200):
    """Permittivity gradient of |S(theta)|^2 at theta = 0, 45, 90 degrees on the
    512 x 512 hexagon design workload (EZ, 4000 steps, design 128 x 128):
    one checkpointed forward run, then one adjoint run per objective.  The
    adjoint step kernel's bandwidth is its algorithmic bytes per cell (mu in
    and out, 1/eps_r, the recorded D, the FP64 gradient read and written) over
    its CUDA-event time; the 512^2 working set (~100 MB) fits in L2."""
    import torch
    from paper_2510_11042_gb300 import lbem
    p = W.adjoint_problem()
    nx, ny, nz = p.shape
    cells = nx * ny * nz
    theta = np.array(p.meta["angles"])
    s = lbem.Solver(p.shape, p.eps, p.mode, "f32", p.absorber_width, p.sigma_max, device=dev)
    s.inject(p.wave)
    s.set_dft_window(p.dft_start, p.dft_periods)
    l0 = s.kernel_launches()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s.forward_checkpointed(p.steps, K)
    torch.cuda.synchronize(dev)
    t_fwd = time.perf_counter() - t0
    runs = []
    for k in range(3):
        wk = np.zeros(3)
        wk[k] = 1.0
        t0 = time.perf_counter()
        J, g = s.adjoint(theta, None, wk)
        torch.cuda.synchronize(dev)
        runs.append((time.perf_counter() - t0, J, lbem.lbem_adjoint_timing(s.h),
                     float(g.abs().max().item())))
    launches = s.kernel_launches() - l0
    s.close()
    torch.cuda.empty_cache()
    probe = _adjoint_probe_3d(dev)
    hbm, _ = peaks()
    q, ne = 21, 1
    bytes_adj = 2 * q * 4 + 4 + 4 * ne + 16
    back_ms = statistics.median(r[2][1] for r in runs)
    replay_ms = statistics.median(r[2][0] for r in runs)
    t_adj = statistics.median(r[0] for r in runs)
    ach = bytes_adj * cells * p.steps / (back_ms / 1e3) / 1e9
    return {"workload": f"hexagon {nx}x{ny} EZ, side 60, design 128x128 (seed 7), lambda 40, "
                        f"W 20, {p.steps} steps, checkpoint every {K}, FP32",
            "objectives": "|S(theta)|^2 at 0, 45, 90 deg, one adjoint run each",
            "forward_checkpointed_s": round(t_fwd, 4),
            "adjoint_s_per_objective": round(t_adj, 4),
            "adjoint_over_forward": round(t_adj / t_fwd, 3),
            "replay_ms": round(replay_ms, 3), "backward_ms": round(back_ms, 3),
            "gradient_mlups": round(cells * p.steps / t_adj / 1e6, 1),
            "J": [r[1] for r in runs], "max_abs_grad": [round(r[3], 6) for r in runs],
            "gpu_launches": int(launches),
            "adjoint_step_roofline": {"bound": "hbm", "bytes_per_cell": bytes_adj,
                                      "achieved": round(ach, 1), "peak": hbm,
                                      "unit": "GB/s", "frac": round(ach / hbm, 4),
                                      "note": "working set L2-resident at 512^2"},
            "hbm_probe_3d": probe}


def _adjoint_probe_3d(dev, n=128, K=60):
    """The adjoint kernels on a 3D grid well above L2 (128^3 sphere, lambda 8,
    240 steps; adjoint populations 0.7 GB): replay and backward bandwidth."""
    import torch
    from paper_2510_11042_gb300 import lbem
    p = W.sphere_problem(n=n, x=3.0, wavelength=8.0, eps_in=2.25, w=10, periods=10, gap_ntff=2, gap_tf=2)
    cells = n ** 3
    s = lbem.Solver(p.shape, p.eps, "3d", "f32", p.absorber_width, p.sigma_max, device=dev)
    s.inject(p.wave)
    s.set_dft_window(p.dft_start, p.dft_periods)
    s.forward_checkpointed(p.steps, K)
    s.adjoint([0.0], [0.0], [1.0])          # warm
    s.adjoint([0.0], [0.0], [1.0])
    replay_ms, back_ms = lbem.lbem_adjoint_timing(s.h)
    s.close()
    torch.cuda.empty_cache()
    hbm, _ = peaks()
    b_back = 2 * 42 * 4 + 4 + 12 + 16
    b_rep = b_cell("3d", "f32") + 12
    gb = b_back * cells * p.steps / (back_ms / 1e3) / 1e9
    gr = b_rep * cells * p.steps / (replay_ms / 1e3) / 1e9
    return {"workload": f"sphere {n}^3, lambda 8, {p.steps} steps, checkpoint every {K}, FP32",
            "backward": {"ms_per_step": round(back_ms / p.steps, 4), "bytes_per_cell": b_back,
                         "achieved_gbs": round(gb, 1), "hbm_frac": round(gb / hbm, 4)},
            "replay": {"ms_per_step": round(replay_ms / p.steps, 4), "bytes_per_cell": b_rep,
                       "achieved_gbs": round(gr, 1), "hbm_frac": round(gr / hbm, 4)}}


# ------------------------------------------------------------------ CPU oracle
class OracleSlab:
    """The FP64 oracle on a z-slab of the workload through the sphere's centre:
    the slab's own permittivity, absorbing layer (global coordinates) and TF/SF
    links, fed by the oracle's incident line.  The oracle is used as it is."""

    def __init__(self, size, dz=8):
        from oracle import lb
        self.size, self.dz = size, dz
        wl, x, eps_in, w = 30.0, 5.0, 1.33 ** 2, 16
        a = x * wl / (2 * math.pi)
        z0 = size // 2 - dz // 2
        eps = W.sphere_eps(size, a, eps_in, z_range=(z0, z0 + dz))
        wave = W.axis_wave("3d", (size, size, size), w, wl)
        self.lat = lb.Lattice((size, size, dz), eps, origin=(0, 0, z0),
                              global_shape=(size, size, size), sponge_w=w,
                              sigma_max=W.DEFAULT_SIGMA_MAX)
        self.lat.set_tfsf_line(wave.tf_lo, wave.tf_hi, 2)
        rng = np.random.default_rng(0)
        self.lat.f = rng.standard_normal(self.lat.f.shape) * 1e-3
        self.inc = rng.standard_normal((size, 42)) * 1e-3
        self.cells = size * size * dz
        self.n = 0

    def step(self, k):
        for _ in range(k):
            self.lat.step(self.n, inc_line=self.inc)
            self.n += 1


def cpu_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_baseline(size, budget_s=15.0):
    """Time the oracle on a bounded sample (a slab) of the workload for about
    budget_s seconds of CPU work; MLUPS = slab cells x updates / seconds."""
    slab = OracleSlab(size)
    slab.step(1)
    t0 = time.perf_counter()
    n = 0
    while True:
        slab.step(1)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    value = slab.cells * n / el / 1e6
    # the same sample on one core
    from oracle import lb
    lb.set_threads(1)
    t0 = time.perf_counter()
    n1 = 0
    while True:
        slab.step(1)
        n1 += 1
        el1 = time.perf_counter() - t0
        if el1 >= budget_s / 3:
            break
    lb.set_threads(cpu_cores())
    return {"value": round(value, 3), "unit": "MLUPS", "cores": cpu_cores(),
            "kind": "oracle", "single_core_value": round(slab.cells * n1 / el1 / 1e6, 3),
            "sample": f"FP64 oracle, z-slab {size}x{size}x{slab.dz} through the centre of the "
                      f"{size}^3 sphere workload, {n} lattice updates in {el:.1f} s "
                      f"({n1} in {el1:.1f} s on one core)"}


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle as it stands, each bench step a
    bounded sample (a slab, --ref-updates lattice updates) of the workload."""
    if rank != 0:
        return
    K, Wm = args.steps, args.warmup
    per_step = max(1, int(round(args.ref_updates)))
    slab = OracleSlab(args.size)
    for _ in range(Wm):
        slab.step(per_step)
    t0 = time.perf_counter()
    for _ in range(K):
        slab.step(per_step)
    el = time.perf_counter() - t0
    value = slab.cells * per_step * K / el / 1e6
    sample = f"z-slab {args.size}x{args.size}x{slab.dz} of the workload, {per_step} lattice updates per step"
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": world,
        "steps": K, "warmup": Wm, "ms_per_step": round(el / K * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": f"sphere_{args.size}^3_n1.33_x5_lambda30_W16_fp32_storage",
                   "sample": sample},
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": cpu_cores(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=27)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lbem", choices=["lbem", "reference"])
    ap.add_argument("--size", type=int, default=384)
    ap.add_argument("--fp32-only", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-updates", type=float, default=2)
    ap.add_argument("--section", default="all",
                    choices=["all", "adjoint_probe", "probe_2d", "variants_3d", "in_place", "cylinder_1024"],
                    help="adjoint_probe / probe_2d / variants_3d / in_place / cylinder_1024: only that "
                         "measurement (profiling)")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.section in ("adjoint_probe", "probe_2d", "variants_3d", "in_place", "cylinder_1024"):
        import torch
        from paper_2510_11042_gb300 import build as lib_build
        lib_build.build()
        dev = torch.device("cuda", local_rank)
        if args.section == "variants_3d":
            out = run_variants_3d(dev, n=args.size)
        elif args.section == "in_place":
            out = run_in_place(dev, n=args.size)
        elif args.section == "cylinder_1024":
            out = run_cylinder_1024(dev)
        else:
            out = {"adjoint_probe": _adjoint_probe_3d, "probe_2d": run_probe_2d}[args.section](dev)
        print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
