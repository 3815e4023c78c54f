#!/usr/bin/env python3
"""Benchmark: finest-grid MDOF/s of the level-dependent Helmholtz multigrid
solved to a 1e-6 relative residual, plus the dominant kernel's bandwidth
against the measured HBM peak.

Workload (default): 1023 x 1023 interior points (h = 1/1024), constant
k = 640 (kh = 0.625), ECS absorbing layers of 32 cells, unit point source at
(0.5, 0.5); complex64 V(1,1)-cycles inside FP64 iterative refinement.  One
step = one complete solve from u = 0 to ||f - A u|| / ||f|| <= 1e-6 (setup
excluded).  Inputs are resident in HBM; L2 is flushed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own replica of the workload (replicas
only: the single-grid solve has no data-parallel split); value = the units
of all ranks / the slowest rank's time.  --impl reference times the FP64 CPU
oracle on this host (a bounded sample of the same workload).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

# Algorithmic bytes per finest-grid point of the level-0 kernels of the
# complex64 cycle (c64 = 8 B; the k^2 field, float32 = 4 B, is not read when
# k is constant; coarse arrays are 1/4 of the fine ones):
#   down pass (pre-smoothing + residual + restriction):
#       read u, f (+k2); write v, f_c/4            = 26 B (30 B with a k2 field)
#   up pass (correction + post-smoothing):
#       read v, e/4, f (+k2); write u              = 26 B (30 B)
#   FP64 refinement: read u64, e32, f64, k2_64; write u64, rhs32 = 72 B
# complex128 cycles: twice the cycle figures.
KERNELS = {0: "down_pass", 2: "up_pass", 3: "refine_fp64", 4: "tail_levels"}
# 3-D (7-point) cycle: the tile-staged level kernels, algorithmic bytes per
# fine point in complex64 (k^2 field: + 4 B read per pass):
#   sweep (Jacobi):                 read u, f; write u         = 24 B
#   residual + restriction:         read u, f; write f_c / 8   = 17 B
#   correction + sweep:             read u, e / 8, f; write u  = 25 B
KERNELS3 = {0: "sweep_3d", 1: "resid_restrict_3d", 2: "correct_sweep_3d"}
BYTES3 = {0: 24.0, 1: 17.0, 2: 25.0}


def kernel_bytes(kid, kconst, mixed):
    if kid == 3:
        return 72.0
    if kid == 4:
        return 0.0
    b = 26.0 if kconst else 30.0
    return b if mixed else 2.0 * b


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x, dist, device):
    """The largest x over the ranks of the process group (x without one):
    the job's time is the slowest replica's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mdofs(points_per_rank, steps, world, seconds):
    """Whole-job throughput of `world` replicas (each solving points_per_rank
    per step for `steps` steps) over the slowest replica's time."""
    return points_per_rank * steps * world / seconds / 1e6


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profile_one(args):
    """Launch one level-0 kernel of the workload twice (warm-up + timed,
    replayed from a captured graph) and exit: the target of ncu captures."""
    import numpy as np
    import torch
    import ctypes as ct
    from paper_1211_4752_gb300 import HelmholtzMG, workloads as W
    from paper_1211_4752_gb300 import _binding as B
    w = getattr(W, args.workload)(**({"n": args.kernel_n} if args.kernel_n else {}))
    k2 = w["k2"]
    k2_t = torch.from_numpy(k2).cuda() if isinstance(k2, np.ndarray) else float(k2)
    gm = args.kernel == "gmres_step"
    mg = HelmholtzMG(w["n"], dim=w["dim"], k2=k2_t, layers=w["layers"],
                     precision=args.precision, max_batch=1,
                     **({"smoother": "gmres"} if gm else {}))
    names = {v: k for k, v in KERNELS.items()}
    names.update({v: k for k, v in KERNELS3.items()})   # the 3-D level kernels (dim 3)
    names["gmres_step"] = 6                             # one level-0 GMRES(3) step
    kid = names[args.kernel]
    ms = ct.c_double()
    stream = torch.cuda.current_stream()
    B.check(B.lib().hh_time_kernel(mg._h, kid, 0, 1, 1, ct.byref(ms),
                                   ct.c_void_p(stream.cuda_stream)))
    print(json.dumps({"kernel": args.kernel, "level": 0, "ms": ms.value,
                      "tile": mg.tile_shape(0), "workload": w["name"]}))
    mg.close()


def run_ours(args):
    import numpy as np
    import torch

    from paper_1211_4752_gb300 import HelmholtzMG, workloads as W
    from paper_1211_4752_gb300 import _binding as B

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = getattr(W, args.workload)(*args.workload_arg)
    n, dim = w["n"], w["dim"]
    pts = (n - 1) ** dim
    k2 = w["k2"]
    k2_t = torch.from_numpy(k2).cuda() if isinstance(k2, np.ndarray) else float(k2)
    mixed = args.precision == "mixed"
    t0 = time.perf_counter()
    mg = HelmholtzMG(n, dim=dim, k2=k2_t, layers=w["layers"], precision=args.precision,
                     max_batch=1, smoother=args.smoother)
    setup_s = time.perf_counter() - t0
    f = torch.from_numpy(w["rhs"][:1].copy()).cuda()   # the first right-hand side
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    fgm = args.solver == "fgmres"

    def solve_once(rhs):
        if fgm:
            return mg.fgmres(rhs, tol=args.tol, restart=args.fgmres_restart)
        return mg.solve(rhs, tol=args.tol)

    infos = []
    for _ in range(args.warmup):
        _, info = solve_once(f)
        infos.append(info[0])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    times = []
    launches = 0
    for _ in range(args.steps):
        flush.fill_(1.0)                       # evict L2 between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info = solve_once(f)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        infos.append(info[0])
        launches += mg.solve_kernels
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total = max_over_ranks(sum(times), dist, "cuda")
    if dist:
        dist.barrier()
    last = infos[-1]
    ok = all(i["status"] == "OK" for i in infos)
    value = job_mdofs(pts, args.steps, world, total)

    # end to end through the host-buffer C-ABI call (pinned host memory);
    # FGMRES: pinned copies in and out around the device call
    fh = torch.from_numpy(w["rhs"][:1].copy()).pin_memory()
    uh = torch.empty_like(fh).pin_memory()

    def e2e_once():
        if fgm:
            u_d, _ = solve_once(fh.to("cuda", non_blocking=True))
            uh.copy_(u_d, non_blocking=True)
        else:
            mg.solve_host(fh, uh, tol=args.tol)
    e2e_once()
    e_times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_once()
        e1.record(stream)
        e1.synchronize()
        e_times.append(e0.elapsed_time(e1) / 1e3)
    e2e_total = max_over_ranks(sum(e_times), dist, "cuda")

    # dominant kernel, timed live on this stream (level 0, back to back)
    import ctypes as ct
    peak, peak_kind = measured_peaks()
    kconst = not isinstance(k2, np.ndarray)
    kt = {}
    fused = mg.tile_shape(0) is not None
    for kid in ((0, 2, 4) if fused else ()) + ((3,) if mixed else ()):
        ms = ct.c_double()
        B.check(B.lib().hh_time_kernel(mg._h, kid, 0, 1, 50, ct.byref(ms),
                                       ct.c_void_p(stream.cuda_stream)))
        kt[kid] = ms.value
    roofline = None
    if dim == 3 and args.smoother == "jacobi":
        # the 3-D cycle's level-0 kernels, timed live back to back
        kt3 = {}
        for kid in (0, 1, 2):
            ms = ct.c_double()
            B.check(B.lib().hh_time_kernel(mg._h, kid, 0, 1, 20, ct.byref(ms),
                                           ct.c_void_p(stream.cuda_stream)))
            kt3[kid] = ms.value
        dom = max(kt3, key=lambda k: kt3[k])
        bpp = (BYTES3[dom] + (0.0 if kconst else 4.0)) * (1.0 if mixed else 2.0)
        achieved = bpp * pts / (kt3[dom] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": KERNELS3[dom], "achieved": achieved, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": None, "bytes_per_point": bpp,
                    "launch_ms": {KERNELS3[k]: v for k, v in kt3.items()}}
    if args.smoother == "gmres":
        # one level-0 GMRES(3) smoothing step (start, 3 Arnoldi steps, update),
        # timed live back to back; a k^2 field adds 4 B per operator application
        ms = ct.c_double()
        B.check(B.lib().hh_time_kernel(mg._h, 6, 0, 1, 20, ct.byref(ms),
                                       ct.c_void_p(stream.cuda_stream)))
        bpp = (GMRES_STEP_BYTES + (0.0 if kconst else 16.0)) * (1.0 if mixed else 2.0)
        achieved = bpp * pts / (ms.value * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": "gmres_step_level0", "achieved": achieved,
                    "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": achieved / peak,
                    "traffic": stored_traffic(w["name"], args.precision, "gmres_step_level0"),
                    "bytes_per_point": bpp, "launch_ms": {"gmres_step_level0": ms.value}}
    if fused:
        dom = max((0, 2), key=lambda k: kt[k])
        name = KERNELS[dom]
        bpp = kernel_bytes(dom, kconst, mixed)
        achieved = bpp * pts / (kt[dom] * 1e-3) / 1e9
        traffic = None
        tf = ROOT / "profiles" / "traffic.json"
        if tf.exists():
            d = json.loads(tf.read_text())
            traffic = d.get(f"{w['name']}:{args.precision}:{name}")
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "bytes_per_point": bpp,
                    "tile_level0": mg.tile_shape(0),
                    "launch_ms": {KERNELS[k]: v for k, v in kt.items()}}

    # the same level-0 kernels on a grid whose arrays exceed the 129 MB L2
    # (constant k, kh = 0.625, ECS n/32): the HBM-bound figure
    roofline_large = None
    if fused and args.large_n > 0:
        wl = W.ecs_const(n=args.large_n)
        mgl = HelmholtzMG(wl["n"], k2=wl["k2"], layers=wl["layers"], precision=args.precision,
                          max_batch=1)
        ptsl = (wl["n"] - 1) ** 2
        ktl = {}
        for kid in (0, 2):
            ms = ct.c_double()
            B.check(B.lib().hh_time_kernel(mgl._h, kid, 0, 1, 20, ct.byref(ms),
                                           ct.c_void_p(stream.cuda_stream)))
            ktl[kid] = ms.value
        dom = max((0, 2), key=lambda k: ktl[k])
        bpp = kernel_bytes(dom, True, mixed)
        achieved = bpp * ptsl / (ktl[dom] * 1e-3) / 1e9
        traffic = None
        tf = ROOT / "profiles" / "traffic.json"
        if tf.exists():
            traffic = json.loads(tf.read_text()).get(f"{wl['name']}:{args.precision}:{KERNELS[dom]}")
        roofline_large = {"bound": "hbm", "kernel": KERNELS[dom], "workload": wl["name"],
                          "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                          "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                          "bytes_per_point": bpp, "tile_level0": mgl.tile_shape(0),
                          "launch_ms": {KERNELS[k]: v for k, v in ktl.items()}}
        mgl.close()

    fp64 = None
    if mixed and args.compare_fp64:
        mg64 = HelmholtzMG(n, dim=dim, k2=k2_t, layers=w["layers"], precision="fp64", max_batch=1,
                           smoother=args.smoother)
        solve64 = ((lambda r: mg64.fgmres(r, tol=args.tol, restart=args.fgmres_restart)) if fgm
                   else (lambda r: mg64.solve(r, tol=args.tol)))
        solve64(f)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, i64 = solve64(f)
        e1.record(stream)
        e1.synchronize()
        s64 = e0.elapsed_time(e1) / 1e3
        fp64 = {"value": pts / s64 / 1e6, "unit": "MDOF/s", "cycles": i64[0]["cycles"],
                "status": i64[0]["status"], "ms_per_solve": s64 * 1e3}
        mg64.close()

    # the same problem by flexible GMRES with one cycle per iteration as the
    # preconditioner (Table 3's LVL-MG-FGMRES), timed once after a warm-up
    fg = None
    if args.fgmres_restart > 0 and not fgm:
        mg.fgmres(f, tol=args.tol, restart=args.fgmres_restart)
        torch.cuda.synchronize()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, ifg = mg.fgmres(f, tol=args.tol, restart=args.fgmres_restart)
        e1.record(stream)
        e1.synchronize()
        sfg = e0.elapsed_time(e1) / 1e3
        fg = {"value": pts / sfg / 1e6, "unit": "MDOF/s", "ms_per_solve": sfg * 1e3,
              "restart": args.fgmres_restart, "iterations": ifg[0]["cycles"],
              "restarts": ifg[0]["refinements"], "rel_residual": ifg[0]["rel_residual"],
              "status": ifg[0]["status"], "kernels": mg.solve_kernels}

    batched = None
    if args.batched and args.workload == "ecs_const" and not fgm:
        batched = group_record(args, max(1, min(args.steps, 2)), 1)

    gmres = None
    if args.gmres_record and args.workload == "ecs_const" and args.smoother == "jacobi" and not fgm:
        gmres = gmres_record(w, args, k2_t, f, stream, flush)

    cpu = cpu_all = None
    if rank == 0 and not args.no_cpu_baseline and fgm:
        cpu = cpu_baseline_fgmres(w, args, last["cycles"])
    elif rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args, last["cycles"])
        if args.cpu_all_cores:
            cyc = int(cpu["sample"].split(" scaled to ")[1].split(" cycles")[0])
            cpu_all = cpu_baseline_all_cores(w, args, cyc)
    if rank == 0:
        line = {
            "metric": "finest-grid MDOF/s solved to 1e-6 rel. residual",
            "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+f64" if mixed else "c128",
            "data": ("synthetic (the analytic coefficient and source of the ionization model)"
                     if w["name"].startswith("ionization") else
                     "synthetic (seeded point sources; " + ("k^2 field" if isinstance(w["k2"], np.ndarray) else "constant k") + ")"),
            "config": {"workload": w["name"], "n": n, "interior": n - 1, "dim": dim,
                       "k2": float(k2) if not isinstance(k2, np.ndarray) else "field",
                       "ecs_layer": w["layers"], "precision": args.precision,
                       "smoother": "GMRES(3)" if args.smoother == "gmres" else "Jacobi 0.8",
                       "solver": (f"FGMRES({args.fgmres_restart}), one cycle per iteration as "
                                  "the preconditioner" if fgm else "V(1,1) cycles"),
                       "tol": args.tol, "parallelism": f"replicas{world}",
                       "l2": "flushed between steps (256 MB write)",
                       "setup_s": setup_s,
                       "tuner": {"key": mg.tuner_key, "coarse_schedule": mg.coarse_schedule,
                                 "tile_level0": mg.tile_shape(0),
                                 "tile_levels": [mg.tile_shape(l) for l in range(mg.levels)
                                                 if mg.tile_shape(l) is not None]}},
            "solve": {("iterations" if fgm else "cycles"): last["cycles"],
                      ("restarts" if fgm else "refinements"): last["refinements"],
                      "rel_residual": last["rel_residual"], "all_ok": ok},
            "e2e": {"value": job_mdofs(pts, args.steps, world, e2e_total), "unit": "MDOF/s",
                    "h2d_bytes_per_step": pts * 16, "d2h_bytes_per_step": pts * 16},
            "roofline": roofline,
            "roofline_large": roofline_large,
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "fp64_gpu": fp64,
            "fgmres": fg,
            "batched": batched,
            "gmres": gmres,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    mg.close()
    if dist:
        dist.destroy_process_group()


def stored_traffic(workload, precision, kernel):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from one
    ncu capture of the current kernels (profiles/traffic.json), or None."""
    tf = ROOT / "profiles" / "traffic.json"
    if not tf.exists():
        return None
    return json.loads(tf.read_text()).get(f"{workload}:{precision}:{kernel}")


# Algorithmic bytes per point of one GMRES(3) smoothing step on a level
# (complex64 vectors, constant k; each kernel reads and writes its vectors
# once): start: u, f -> q_0 (24 B); Arnoldi steps J = 0, 1: q_0..q_J -> w
# (8 (J + 2)); orthogonalisations J = 0, 1: w, q_0..q_J -> q_{J+1}
# (8 (J + 3)); the last Arnoldi step reads q_0..q_2 and forms only sums
# (24 B; |q_3| follows from them); update: u, q_0..q_2 -> u (40 B).
# Sum: 184 B.
GMRES_STEP_BYTES = 184.0


def gmres_record(w, args, k2_t, f, stream, flush):
    """The same workload with GMRES(3) smoothing (the paper's smoother): the
    cycle's time (captured graph, hh_time_kernel kernel 5), one level-0
    smoothing step against its algorithmic bytes, and a solve to the tolerance
    capped at --gmres-max-cycles cycles."""
    import ctypes as ct
    import torch
    from paper_1211_4752_gb300 import HelmholtzMG
    from paper_1211_4752_gb300 import _binding as B
    n, dim = w["n"], w["dim"]
    pts = (n - 1) ** dim
    mixed = args.precision == "mixed"
    mg = HelmholtzMG(n, dim=dim, k2=k2_t, layers=w["layers"], precision=args.precision,
                     max_batch=1, smoother="gmres", max_cycles=args.gmres_max_cycles)
    sp = ct.c_void_p(stream.cuda_stream)
    ms = ct.c_double()
    B.check(B.lib().hh_time_kernel(mg._h, 5, 0, 1, 20, ct.byref(ms), sp))
    cycle_ms = ms.value
    B.check(B.lib().hh_time_kernel(mg._h, 6, 0, 1, 20, ct.byref(ms), sp))
    step_ms = ms.value
    peak, peak_kind = measured_peaks()
    bpp = GMRES_STEP_BYTES * (1.0 if mixed else 2.0)
    achieved = bpp * pts / (step_ms * 1e-3) / 1e9
    flush.fill_(1.0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, info = mg.solve(f, tol=args.tol)
    e1.record(stream)
    e1.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    rec = {"smoother": "GMRES(3)", "cycle_ms": cycle_ms, "kernels_per_cycle": mg.cycle_kernels,
           "solve": {"value": pts / s / 1e6 if info[0]["status"] == "OK" else None,
                     "unit": "MDOF/s", "ms": s * 1e3, "cycles": info[0]["cycles"],
                     "status": info[0]["status"], "rel_residual": info[0]["rel_residual"],
                     "max_cycles": args.gmres_max_cycles},
           "roofline": {"bound": "hbm", "kernel": "gmres_step_level0", "achieved": achieved,
                        "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                        "frac": achieved / peak,
                        "traffic": stored_traffic(w["name"], args.precision, "gmres_step_level0"),
                        "bytes_per_point": bpp, "launch_ms": {"gmres_step_level0": step_ms}}}
    mg.close()
    return rec


def cpu_baseline(w, args, cycles_hint):
    """The FP64 oracle on this host: time a bounded number of V-cycles of the
    same workload and scale to one complete solve with the oracle's own cycle
    count (from its committed golden fixture when present)."""
    import numpy as np

    import oracle as O
    n, dim = w["n"], w["dim"]
    pts = (n - 1) ** dim
    t0 = time.perf_counter()
    H = O.build_hierarchy(n, dim, w["k2"], layers=w["layers"], smoother=args.smoother)
    f = w["rhs"][0]
    u = np.zeros_like(f)
    t1 = time.perf_counter()
    ncyc = 0
    while True:
        u = O.vcycle(H, 0, u, f)
        O.residual_norm(H, u, f)
        ncyc += 1
        el = time.perf_counter() - t1
        if el > args.cpu_seconds or ncyc >= 200:
            break
    s_per_cycle = el / ncyc
    suffix = "_gmres" if args.smoother == "gmres" else ""
    gold = ROOT / "tests" / "golden" / f"{w['name']}{suffix}.json"
    if gold.exists():
        cycles = json.loads(gold.read_text())["cycles"]
        src = "oracle cycle count from its golden fixture"
    else:
        cycles = cycles_hint
        src = "cycle count of this run's solve"
    return {"value": pts / (s_per_cycle * cycles) / 1e6, "unit": "MDOF/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{ncyc} V-cycles of {w['name']} ({s_per_cycle:.3f} s/cycle, numpy FP64, "
                      f"1 thread) scaled to {cycles} cycles ({src}); setup {t1 - t0:.1f} s"}


def cpu_baseline_fgmres(w, args, iters_hint):
    """The FP64 oracle's FGMRES with the same preconditioning cycle on this
    host: a bounded number of iterations (one restart cycle, about
    --cpu-seconds) timed and scaled to one complete solve with the oracle's own
    iteration count (its golden fixture when present)."""
    import numpy as np

    import oracle as O
    n, dim = w["n"], w["dim"]
    pts = (n - 1) ** dim
    H = O.build_hierarchy(n, dim, w["k2"], layers=w["layers"], smoother=args.smoother)
    f = w["rhs"][0]
    per_cycle = []
    u = np.zeros_like(f)
    t1 = time.perf_counter()
    while time.perf_counter() - t1 < args.cpu_seconds / 2 and len(per_cycle) < 50:
        t = time.perf_counter()
        u = O.vcycle(H, 0, np.zeros_like(f), f)
        per_cycle.append(time.perf_counter() - t)
    k = max(2, min(args.fgmres_restart, int(args.cpu_seconds / max(min(per_cycle), 1e-6))))
    t = time.perf_counter()
    O.fgmres(H, f, tol=1e-300, m=k, max_iter=k, strict=False)
    s_per_iter = (time.perf_counter() - t) / k
    gold = ROOT / "tests" / "golden" / f"{w['name']}_fgmres{args.fgmres_restart}_{args.smoother}.json"
    if gold.exists():
        iters = json.loads(gold.read_text())["iterations"]
        src = "oracle iteration count from its golden fixture"
    else:
        iters = iters_hint
        src = "iteration count of this run's solve"
    return {"value": pts / (s_per_iter * iters) / 1e6, "unit": "MDOF/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{k} FGMRES iterations of {w['name']} ({s_per_iter:.3f} s/iteration, "
                      f"numpy FP64, 1 thread) scaled to {iters} iterations ({src})"}


def _oracle_cycles_worker(task):
    """One host core: build the oracle hierarchy of the workload and time
    V-cycles for about `seconds` (a process of a spawn pool)."""
    name, wargs, seconds, smoother = task
    import numpy as np

    import oracle as O
    from paper_1211_4752_gb300 import workloads as W
    w = getattr(W, name)(*wargs)
    H = O.build_hierarchy(w["n"], w["dim"], w["k2"], layers=w["layers"], smoother=smoother)
    f = w["rhs"][0]
    u = np.zeros_like(f)
    t1 = time.perf_counter()
    ncyc = 0
    while True:
        u = O.vcycle(H, 0, u, f)
        O.residual_norm(H, u, f)
        ncyc += 1
        el = time.perf_counter() - t1
        if el > seconds or ncyc >= 200:
            return ncyc, el


def cpu_baseline_all_cores(w, args, cycles):
    """The oracle on every host core at once: one independent solve per core
    (a spawn pool, one numpy thread each), each timed on a bounded sample of
    V-cycles and scaled to `cycles`; the value is their summed throughput."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(ncores) as pool:
            res = pool.map(_oracle_cycles_worker,
                           [(args.workload, tuple(args.workload_arg), args.cpu_seconds,
                             args.smoother)] * ncores)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    pts = (w["n"] - 1) ** w["dim"]
    value = sum(pts / (el / nc * cycles) / 1e6 for nc, el in res)
    per = sum(el / nc for nc, el in res) / len(res)
    return {"value": value, "unit": "MDOF/s", "cores": ncores, "kind": "oracle",
            "sample": f"{ncores} processes x {min(nc for nc, _ in res)}+ V-cycles of {w['name']} "
                      f"({per:.3f} s/cycle per core, numpy FP64, 1 thread each), one independent "
                      f"solve per core scaled to {cycles} cycles, throughputs summed"}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    from paper_1211_4752_gb300 import workloads as W
    w = getattr(W, args.workload)(*args.workload_arg)
    import numpy as np

    import oracle as O
    n, dim = w["n"], w["dim"]
    pts = (n - 1) ** dim
    H = O.build_hierarchy(n, dim, w["k2"], layers=w["layers"], smoother=args.smoother)
    f = w["rhs"][0]
    suffix = "_gmres" if args.smoother == "gmres" else ""
    gold = ROOT / "tests" / "golden" / f"{w['name']}{suffix}.json"
    cycles = json.loads(gold.read_text())["cycles"] if gold.exists() else None
    per = max(1, int(args.cpu_cycles))
    u = np.zeros_like(f)
    for _ in range(args.warmup):
        u = O.vcycle(H, 0, u, f)
    t = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per):
            u = O.vcycle(H, 0, u, f)
            O.residual_norm(H, u, f)
        t += time.perf_counter() - t0
    s_per_cycle = t / (args.steps * per)
    ncyc = cycles if cycles else per
    value = pts / (s_per_cycle * ncyc) / 1e6
    line = {"impl": "reference", "metric": "finest-grid MDOF/s solved to 1e-6 rel. residual",
            "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": s_per_cycle * ncyc * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128", "data": "synthetic (seeded point sources; " + ("k^2 field" if isinstance(w["k2"], np.ndarray) else "constant k") + ")",
            "config": {"workload": w["name"], "n": n, "interior": n - 1, "dim": dim,
                       "precision": "fp64 oracle", "tol": args.tol,
                       "smoother": "GMRES(3)" if args.smoother == "gmres" else "Jacobi 0.8"},
            "cpu_baseline": {"value": value, "unit": "MDOF/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per} V-cycles per step, scaled to {ncyc} cycles"},
            "e2e": {"value": value, "unit": "MDOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def group_record(args, steps, warmup, stand_alone=False):
    """The many-source workload over uneven grid sizes (64 point sources over
    255^2, 511^2 and 1023^2 grids, 22/21/21 right-hand sides) solved by one
    group call per step (hh_solve_group).  Returns MDOF/s (finest-grid points
    of all right-hand sides / time), e2e (pinned host buffers in and out every
    step), the same batches solved one after another, and the stated
    comparison with 64 sequential plain complex128 solves: one plain solve
    per grid size timed and scaled by that size's count (a projection)."""
    import torch
    from paper_1211_4752_gb300 import HelmholtzMG, solve_group, workloads as W
    groups = W.batch_sources()
    probs, pts = [], 0
    for g in groups:
        B = g["rhs"].shape[0]
        mg = HelmholtzMG(g["n"], k2=g["k2"], layers=g["layers"], precision=args.precision,
                         max_batch=B, smoother=args.smoother)
        probs.append((mg, torch.from_numpy(g["rhs"]).cuda()))
        pts += B * (g["n"] - 1) ** 2
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(fn):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    for _ in range(warmup):
        solve_group(probs, tol=args.tol)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if stand_alone else None
    if sampler:
        sampler.start()
    times, ok, launches = [], True, 0
    for _ in range(steps):
        t, res = timed(lambda: solve_group(probs, tol=args.tol))
        times.append(t)
        ok = ok and all(i["status"] == "OK" for _, info in res for i in info)
        launches += sum(mg.solve_kernels for mg, _ in probs)
    clocks = sampler.stop() if sampler else None
    total = sum(times)
    t_seq, _ = timed(lambda: [mg.solve(f, tol=args.tol) for mg, f in probs])
    # the same problems as one work-list group (one launch chain per cycle)
    from paper_1211_4752_gb300 import HelmholtzGroup
    grp = HelmholtzGroup([mg for mg, _ in probs], [f.shape[0] for _, f in probs])
    rhs = [f for _, f in probs]
    for _ in range(max(1, warmup)):
        grp.solve(rhs, tol=args.tol)
    wl_times, wl_ok, wl_launches = [], True, 0
    for _ in range(steps):
        t, res = timed(lambda: grp.solve(rhs, tol=args.tol))
        wl_times.append(t)
        wl_ok = wl_ok and all(i["status"] == "OK" for _, info in res for i in info)
        wl_launches += grp.kernels
    grp.close()
    worklist = {"value": pts * steps / sum(wl_times) / 1e6, "unit": "MDOF/s",
                "ms_per_step": sum(wl_times) / steps * 1e3, "all_ok": wl_ok,
                "gpu_launches": wl_launches,
                "kind": "hh_group_solve: one launch per level size over every problem's tiles"}
    streams = {"value": pts * steps / total / 1e6, "unit": "MDOF/s",
               "ms_per_step": total / steps * 1e3, "all_ok": ok, "gpu_launches": launches,
               "kind": "hh_solve_group: each problem's launch chain on its own stream"}
    # end to end: pinned host right-hand sides in, solutions out, every step
    hosts = [torch.from_numpy(g["rhs"].copy()).pin_memory() for g in groups]
    outs = [torch.empty_like(h).pin_memory() for h in hosts]

    def e2e():
        dev = [(mg, h.to("cuda", non_blocking=True)) for (mg, _), h in zip(probs, hosts)]
        res = solve_group(dev, tol=args.tol)
        for o, (u, _) in zip(outs, res):
            o.copy_(u, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e_times = [timed(e2e)[0] for _ in range(steps)]
    nbytes = sum(h.numel() * 16 for h in hosts)
    for mg, _ in probs:
        mg.close()
    # 64 sequential plain complex128 solves, projected from one per grid size
    plain, t_plain = [], 0.0
    for g in groups:
        mg = HelmholtzMG(g["n"], k2=g["k2"], layers=g["layers"], precision="fp64", max_batch=1,
                         smoother=args.smoother)
        f1 = torch.from_numpy(g["rhs"][:1].copy()).cuda()
        mg.solve(f1, tol=0.5)                  # captures the cycle graph
        t1, (_, i1) = timed(lambda: mg.solve(f1, tol=args.tol))
        cnt = int(g["rhs"].shape[0])
        plain.append({"grid": g["n"] - 1, "ms_per_solve": t1 * 1e3, "cycles": i1[0]["cycles"],
                      "count": cnt, "status": i1[0]["status"]})
        t_plain += t1 * cnt
        mg.close()
    best = worklist if worklist["value"] >= streams["value"] else streams
    return {
        "value": best["value"], "unit": "MDOF/s",
        "ms_per_step": best["ms_per_step"], "steps": steps, "warmup": warmup,
        "path": "worklist" if best is worklist else "streams",
        "worklist": worklist, "streams": streams,
        "workload": "batch_sources_64rhs_255_511_1023", "rhs": 64,
        "grids": [g["n"] - 1 for g in groups],
        "rhs_per_grid": [int(g["rhs"].shape[0]) for g in groups],
        "precision": args.precision, "all_ok": best["all_ok"],
        "sequential_batches": {"value": pts / t_seq / 1e6, "unit": "MDOF/s", "ms": t_seq * 1e3},
        "sequential_plain_c128": {"value": pts / t_plain / 1e6, "unit": "MDOF/s",
                                  "ms": t_plain * 1e3, "per_grid": plain,
                                  "kind": "projection: one plain complex128 solve per grid "
                                          "size, timed, times that size's count"},
        "e2e": {"value": pts * steps / sum(e_times) / 1e6, "unit": "MDOF/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": best["gpu_launches"], "clocks": clocks,
    }


def run_group(args):
    """--workload batch_sources: the group record as the bench line."""
    import torch
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    r = group_record(args, args.steps, args.warmup, stand_alone=True)
    line = {
        "metric": "finest-grid MDOF/s solved to 1e-6 rel. residual",
        "value": r["value"], "unit": "MDOF/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64+f64" if args.precision == "mixed" else "c128",
        "data": "synthetic (64 seeded point sources, constant k per grid)",
        "config": {"workload": r["workload"], "rhs": 64, "grids": r["grids"],
                   "rhs_per_grid": r["rhs_per_grid"], "precision": args.precision,
                   "tol": args.tol, "parallelism": "replicas1",
                   "l2": "flushed between steps (256 MB write)"},
        "all_ok": r["all_ok"],
        "path": r["path"], "worklist": r["worklist"], "streams": r["streams"],
        "sequential": r["sequential_batches"],
        "sequential_plain_c128": r["sequential_plain_c128"],
        "e2e": r["e2e"], "roofline": None, "cpu_baseline": None,
        "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)


def profile_cycles(args):
    """Run --profile-cycles V-cycles of the workload through hh_cycles (every
    kernel launched directly on the stream, no graph) and exit: the target of
    launch-list captures of one cycle's kernels."""
    import numpy as np
    import torch
    from paper_1211_4752_gb300 import HelmholtzMG, workloads as W
    w = getattr(W, args.workload)(*args.workload_arg)
    k2 = w["k2"]
    k2_t = torch.from_numpy(k2).cuda() if isinstance(k2, np.ndarray) else float(k2)
    mg = HelmholtzMG(w["n"], dim=w["dim"], k2=k2_t, layers=w["layers"],
                     precision=args.precision, max_batch=1, smoother=args.smoother,
                     tuner_cache=args.tuner_cache)
    f = torch.from_numpy(w["rhs"][:1].copy()).cuda()
    u = mg.cycles(f, torch.zeros_like(f), args.profile_cycles)
    torch.cuda.synchronize()
    print(json.dumps({"kernel": "cycles", "workload": w["name"], "cycles": args.profile_cycles,
                      "smoother": args.smoother, "precision": args.precision,
                      "kernels_per_cycle": mg.cycle_kernels,
                      "unorm": float(u.abs().pow(2).sum().sqrt())}))
    mg.close()


def profile_fgmres(args):
    """One FGMRES(restart) solve of the workload capped at --fgmres-iterations
    iterations, then exit: the target of launch-list captures of the Krylov
    kernels (run with HH_LOOP=host so that ncu sees the iteration kernels)."""
    import numpy as np
    import torch
    from paper_1211_4752_gb300 import HelmholtzMG, workloads as W
    w = getattr(W, args.workload)(*args.workload_arg)
    k2 = w["k2"]
    k2_t = torch.from_numpy(k2).cuda() if isinstance(k2, np.ndarray) else float(k2)
    mg = HelmholtzMG(w["n"], dim=w["dim"], k2=k2_t, layers=w["layers"],
                     precision=args.precision, max_batch=1, smoother=args.smoother)
    f = torch.from_numpy(w["rhs"][:1].copy()).cuda()
    _, info = mg.fgmres(f, tol=args.tol, restart=args.fgmres_restart,
                        max_iter=args.fgmres_iterations)
    torch.cuda.synchronize()
    print(json.dumps({"kernel": "fgmres", "workload": w["name"], "restart": args.fgmres_restart,
                      "info": info[0], "kernels": mg.solve_kernels}))
    mg.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="ecs_const")
    ap.add_argument("--workload-arg", type=int, nargs="*", default=[],
                    help="positional arguments of the workload (e.g. k0 of ionization)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--smoother", choices=["jacobi", "gmres"], default="jacobi",
                    help="jacobi: the benchmarked configuration; gmres: the paper's GMRES(3)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--large-n", type=int, default=4096,
                    help="also time the level-0 kernels on an (n-1)^2 grid beyond L2 (0: skip)")
    ap.add_argument("--fgmres-restart", type=int, default=32,
                    help="also time FGMRES(m) with the cycle as preconditioner (0: skip)")
    ap.add_argument("--solver", choices=["cycle", "fgmres"], default="cycle",
                    help="cycle: V-cycles as the solver (the metric's method); fgmres: FGMRES("
                         "--fgmres-restart) with one cycle per iteration as the preconditioner")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 64-source group record (255^2/511^2/1023^2) of the default line")
    ap.add_argument("--no-gmres", dest="gmres_record", action="store_false",
                    help="skip the GMRES(3)-smoothed cycle record of the default line")
    ap.add_argument("--gmres-max-cycles", type=int, default=400,
                    help="cycle cap of the GMRES record's solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", dest="cpu_all_cores", action="store_false",
                    help="skip the oracle timed on every host core at once")
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cpu-cycles", type=int, default=4)
    ap.add_argument("--profile-cycles", type=int, default=4,
                    help="V-cycles run by --kernel cycles")
    ap.add_argument("--tuner-cache", default=None,
                    help="tuner cache file of --kernel cycles (a second run with the same file "
                         "launches no tuning kernels)")
    ap.add_argument("--kernel", choices=sorted(KERNELS.values()) + sorted(KERNELS3.values()) +
                    ["gmres_step", "fgmres", "cycles"],
                    help="launch one level-0 kernel of the workload (or one capped FGMRES "
                         "solve) and exit (for ncu)")
    ap.add_argument("--kernel-n", type=int, default=0,
                    help="grid size n of the workload for --kernel (0: the workload's own)")
    ap.add_argument("--fgmres-iterations", type=int, default=40,
                    help="iteration cap of --kernel fgmres")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch_sources":
        run_group(args)
    elif args.kernel == "fgmres":
        profile_fgmres(args)
    elif args.kernel == "cycles":
        profile_cycles(args)
    elif args.kernel:
        profile_one(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
