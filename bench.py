"""Benchmark of the implicit Rykov iteration on GB300.

One step = one full implicit iteration (Steps 2-6: reconstruction, interface
collision and fluxes, macro PR-SGS prediction, micro PR-SGS, compensated update)
over every (cell, velocity) pair of the workload.  The default workload is the
scale case: a Mach-8 sphere-cone at Kn 0.005, ~500k seeded Delaunay tetrahedra x
~8,000-point unstructured velocity space from the paper's DVS criterion, in mixed
precision (FP32 distributions and per-velocity arithmetic, compensated sums, FP64
macro PR-SGS and compensation).  Metric: cell-velocity updates/s (N*K / time per
iteration); the wall time to residual 1e-6 is reported beside it (from the sphere
case, ~62k tetrahedra x ~3,000 velocities, which converges in about a hundred
iterations; the sphere's throughput, its FP64 form and the adjoint are extra keys).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload scale|sphere]
                  [--precision mixed|fp64] [--impl reference]

--impl reference times the FP64 CPU oracle (the test oracle, as it stands) on the
host cores on a bounded sample of the same workload (the full mesh with every S-th
velocity; the same sample as the cpu_baseline key of the GPU arm).  Under torchrun
every rank runs an independent replica (the path has no data-path collective);
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-velocity updates/s per implicit sweep; wall time to residual 1e-6"
UNIT = "cell-velocity updates/s"
START_ITERS = 10          # start-up iterations (first order, CFL ramp), untimed
# velocity stride of the oracle's bounded sample, per workload: the full mesh with
# every S-th velocity (weights x S), used by the cpu_baseline key and the reference arm
CPU_STRIDE = {"scale": 50, "sphere": 30}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the kernels
# as they stand, mixed precision, from one full-size ncu capture of one second-order
# iteration of each workload (one pass; the micro sweeps: the 16 launches' total / 16);
# a kernel changed since the capture has no entry
NCU_TRAFFIC = {"scale": {"k_micro_sweep": 36.20e9, "k_recon": 110.84e9, "k_face_interior": 189.67e9},
               "sphere": {"k_micro_sweep": 1.694e9, "k_face_interior": 6.791e9}}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
        sm, smax, reasons, n = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            n += 1
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": n}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Max of a per-rank scalar over all ranks (identity for one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput of `world` independent replicas timed by the slowest."""
    return world * units_per_rank / (ms_max * 1e-3)


def workload(name: str):
    from paper_2303_10846_gb300 import inputs as I
    return {"scale": I.cone_scale_workload, "sphere": I.sphere_workload}[name]()


def dvs_sample(wl, stride):
    """Every stride-th velocity of the workload's DVS (weights scaled by stride):
    the bounded CPU sample of the same workload."""
    import copy
    from paper_2303_10846_gb300 import inputs as I
    if stride <= 1:
        return wl
    w2 = copy.copy(wl)
    w2.dvs = I.DVS(u=wl.dvs.u[::stride].copy(), w=wl.dvs.w[::stride] * stride,
                   name=f"{wl.dvs.name}/every{stride}")
    w2.name = f"{wl.name}/every{stride}thvelocity_K{w2.dvs.K}"
    return w2


def _cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def oracle_rate(wl, iters, warmup=0):
    """FP64 oracle (C, OpenMP over the cells of a colour and over faces) on the host
    cores: updates/s over `iters` implicit iterations after `warmup` more."""
    import oracle as O
    o = O.Oracle(wl)
    if warmup:
        o.iterate(warmup)
    t0 = time.perf_counter()
    o.iterate(iters)
    dt = time.perf_counter() - t0
    o.close()
    return wl.mesh.n_cell * wl.dvs.K * iters / dt, dt


def oracle_sample_rate(name, stride, iters, warmup, threads=None):
    """The oracle on the bounded sample of workload `name` (every stride-th velocity)
    in a fresh child process (no CUDA context, no torch thread pool beside OpenMP):
    the same start-up iterations as the GPU arm (first order, CFL ramp), `warmup`
    more, then `iters` timed iterations of the limited second-order scheme.
    Returns (updates/s of the sample, seconds per iteration, sample K, start-up)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "wl = bench.dvs_sample(bench.workload(sys.argv[1]), int(sys.argv[2])); "
            "start = max(bench.START_ITERS, wl.params.first_order_iters + 2); "
            "v, dt = bench.oracle_rate(wl, int(sys.argv[3]), start + int(sys.argv[4])); "
            "print(json.dumps({'v': v, 'dt': dt, 'K': wl.dvs.K, 'start': start}))" % ROOT)
    env = dict(os.environ)
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    r = subprocess.run([sys.executable, "-c", code, name, str(stride), str(iters), str(warmup)],
                       capture_output=True, text=True, env=env, timeout=1800)
    line = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not line:
        raise RuntimeError("oracle sample failed: " + r.stderr[-500:])
    d = json.loads(line[-1])
    return d["v"], d["dt"] / iters, d["K"], d["start"]


def cpu_sample_desc(wl, sample_k, stride, what):
    return (f"{what} of the full mesh (N={wl.mesh.n_cell}) with every {stride}th velocity "
            f"(K={sample_k} of {wl.dvs.K}, weights x{stride}), in a child process")


def oracle_table(steps=2):
    """The oracle's timing table: its time per iteration on one core and
    on all cores for the cavity (512 cells x 512 velocities, whole case) and the
    sphere (every 10th velocity), and on all cores for the capsule (every 20th
    velocity, 5 timed iterations), each in a child process with OMP_NUM_THREADS set."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "from paper_2303_10846_gb300 import inputs as I; "
            "c, n = sys.argv[1], int(sys.argv[2]); "
            "wl = I.cavity_workload() if c == 'cavity' else "
            "bench.dvs_sample(I.sphere_workload(), 10) if c == 'sphere' else "
            "bench.dvs_sample(I.capsule_workload(), 20); "
            "v, dt = bench.oracle_rate(wl, n, 1); "
            "print(json.dumps({'updates_per_s': v, 's_per_iteration': dt / n, "
            "'iterations': n, 'N': wl.mesh.n_cell, 'K': wl.dvs.K}))" % ROOT)
    out = {}
    for case, threads, n in (("cavity", 1, steps), ("cavity", _cores(), steps), ("sphere", 1, steps),
                             ("sphere", _cores(), steps), ("capsule", _cores(), 5)):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        r = subprocess.run([sys.executable, "-c", code, case, str(n)], capture_output=True, text=True,
                           env=env, timeout=900)
        line = [l for l in r.stdout.splitlines() if l.startswith("{")]
        out[f"{case}_threads{threads}"] = json.loads(line[-1]) if line else {"error": r.stderr[-300:]}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    wl = workload(args.workload)
    stride = CPU_STRIDE[args.workload]
    v, dt, sk, start = oracle_sample_rate(args.workload, stride, args.steps, args.warmup)
    cores = _cores()
    out = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": wl.name, "N": wl.mesh.n_cell, "K": wl.dvs.K,
                      "sample_K": sk, "precision": "fp64", "l2": "n/a (CPU)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": cpu_sample_desc(
                                wl, sk, stride, f"{start} start-up + {args.warmup} warm-up + "
                                f"{args.steps} timed oracle iterations")},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if not args.no_oracle_table:
        out["oracle_table"] = oracle_table()
    return out


# algorithmic words per unit and step of the per-velocity kernels (each input element
# read once, each output written once): micro sweeps 10 (first: phi, F, neighbour dphi;
# Res, dphi) + 6 per middle sweep (Res, neighbour dphi; dphi) + 10 (last: Res,
# neighbour dphi, phi; phi, dphi) per (cell, k); recon 2 per (cell, k) + 2 per (face,
# k); interior faces 4 per (interior face, k)
def algorithmic_bytes(wl, Tsz, n_micro=2):
    N, K = wl.mesh.n_cell, wl.dvs.K
    F = wl.mesh.n_face
    Fi = int((wl.mesh.face_cell[:, 1] >= 0).sum())
    nsw = 2 * n_micro
    return {"k_micro_sweep": (10 + 6 * (nsw - 2) + 10) * N * K * Tsz,
            "k_recon": (2 * N * K + 2 * F * K) * Tsz,
            "k_face_interior": 4 * Fi * K * Tsz}


KERNEL_CLASSES = {"k_recon": ("recon",), "k_face_interior": ("face_interior",),
                  "k_face_boundary": ("face_boundary",), "k_micro_flux + macro fluxes": ("fluxes",),
                  "k_macro (prep + PR-SGS + finish)": ("macro_sgs",),
                  "k_micro_sweep": ("micro_sweep_first", "micro_sweep_mid", "micro_sweep_last")}


class Case:
    """One solver on one workload: start-up, warm-up, timed graph iterations, a
    profiled pass with CUDA events around every kernel class."""

    def __init__(self, wl, precision, macro32=False):
        from paper_2303_10846_gb300.rykov import Solver
        self.wl = wl
        self.precision = precision
        self.s = Solver(wl, precision, macro32=macro32)
        self.N, self.K = wl.mesh.n_cell, wl.dvs.K
        self.Tsz = 4 if precision == "mixed" else 8

    def timed(self, steps, warmup, start, barrier, clocks=None):
        import torch
        s = self.s
        s.iterate(start)
        s.iterate(warmup)
        barrier()
        if clocks:
            clocks.start()
        _, l0 = s.profile_get()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        t0 = time.perf_counter()
        e0.record(s.stream)
        rc, done, res = s.iterate(steps)
        e1.record(s.stream)
        torch.cuda.synchronize()
        self.wall = time.perf_counter() - t0
        self.clocks = clocks.stop() if clocks else None
        self.ms = e0.elapsed_time(e1) / steps
        _, l1 = s.profile_get()
        self.launches = l1 - l0
        self.res = res
        return self.ms

    def profiled(self, steps):
        import torch
        s = self.s
        s.profile(True)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(s.stream)
        s.iterate(steps)
        p1.record(s.stream)
        torch.cuda.synchronize()
        self.ms_profiled = p0.elapsed_time(p1) / steps
        prof, _ = s.profile_get()
        s.profile(False)
        self.prof_steps = steps
        self.kern = {k: tuple(map(sum, zip(*[prof[c] for c in cls]))) for k, cls in KERNEL_CLASSES.items()}
        return self.kern

    def roofline(self, peak, peak_kind, traffic=None):
        """Dominant kernel class: algorithmic bytes per launch / CUDA-event duration."""
        algo = algorithmic_bytes(self.wl, self.Tsz)
        name, (tms, cnt) = max(self.kern.items(), key=lambda kv: kv[1][0])
        if name not in algo or not cnt:
            return {"kernel": name, "bound": "hbm", "achieved": None, "peak": peak}
        lps = cnt / self.prof_steps
        bl = algo[name] / lps
        ach = bl / (tms / cnt * 1e-3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": peak,
                "unit": "GB/s", "frac": round(ach / peak, 4),
                "traffic": (traffic or {}).get(name), "peak_kind": peak_kind,
                "launches_per_step": lps, "algorithmic_bytes_per_launch": int(bl),
                "share_of_step": round(tms / (self.ms_profiled * self.prof_steps), 4),
                "timing": "CUDA events around every launch of the kernel class on the solver "
                          "stream, in a profiled pass right after the timed (graph) region"}

    def kernel_table(self, peak):
        algo = algorithmic_bytes(self.wl, self.Tsz)
        out = {}
        for k, (tms, cnt) in self.kern.items():
            ms = tms / self.prof_steps
            d = {"ms_per_step": round(ms, 4), "launches_per_step": cnt / self.prof_steps}
            if k in algo and ms > 0:
                d["hbm_frac"] = round(algo[k] / (ms * 1e-3) / 1e9 / peak, 4)
            out[k] = d
        return out

    def iteration_roofline(self, peak):
        b = 52 * self.Tsz * self.N * self.K
        a = b / (self.ms * 1e-3) / 1e9
        return {"model_bytes_per_cell_velocity": 52 * self.Tsz, "achieved": round(a, 1),
                "peak": peak, "frac": round(a / peak, 4)}

    def converge(self, cap, tol=1e-6):
        import numpy as np
        import torch
        s = self.s
        s.set_state_prim(self.wl.prim0)
        torch.cuda.synchronize()
        tc = time.perf_counter()
        rc, n, res = s.iterate(cap, tol=tol)
        torch.cuda.synchronize()
        t = time.perf_counter() - tc
        return {"tol": tol, "iterations": n, "wall_s": round(t, 4),
                "reached": bool(rc == 0 and float(np.max(res)) < tol),
                "final_residual": float(np.max(res))}

    def end_to_end(self, steps, world, dev, barrier):
        """Through the public API with host buffers: a restart from a host checkpoint
        (W, q and the distributions in pinned host memory, uploaded by rk_set_state),
        `steps` second-order iterations with the residual read back to the host every
        iteration, then W and q read back."""
        import dataclasses
        import torch
        from paper_2303_10846_gb300.rykov import _ptr
        s, N = self.s, self.N
        s.set_params(dataclasses.replace(self.wl.params, first_order_iters=0))
        s.iterate(1)                                   # capture the graph for these params
        Wh = torch.empty((N, 6), dtype=torch.float64).pin_memory()
        qh = torch.empty((N, 6), dtype=torch.float64).pin_memory()
        s._check(s.L.rk_moments(s.h, _ptr(Wh), _ptr(qh), None, 0))
        dg = s.get_distribution()
        dist = torch.empty(dg.shape, dtype=dg.dtype).pin_memory()
        dist.copy_(dg)
        del dg
        torch.cuda.empty_cache()
        barrier()
        t1 = time.perf_counter()
        s._check(s.L.rk_set_state(s.h, _ptr(Wh), _ptr(qh), _ptr(dist), 0))
        rc2, done2, _ = s.iterate(steps, tol=1e-300)
        s._check(s.L.rk_moments(s.h, _ptr(Wh), _ptr(qh), None, 0))
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t1, world, dev)
        up = (Wh.numel() + qh.numel()) * 8 + dist.numel() * dist.element_size()
        s.set_params(self.wl.params)
        return {"value": job_value(self.N * self.K * done2, world, e2e_s * 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(up / done2),
                "d2h_bytes_per_step": int(6 * 8 + (Wh.numel() + qh.numel()) * 8 / done2),
                "what": f"restart from a pinned host checkpoint ({up / 1e9:.2f} GB), {done2} "
                        f"iterations with the residual read back each iteration, W and q read back"}

    def adjoint(self, dev, iters, krylov):
        import torch
        s = self.s
        s.bind_adjoint(krylov)
        gen = torch.Generator(device=dev).manual_seed(1)
        v = torch.randn(s.state_len, dtype=torch.float64, device=dev, generator=gen)
        s.vjp(v)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        a0.record(s.stream)
        for _ in range(reps):
            s.vjp(v)
        a1.record(s.stream)
        torch.cuda.synchronize()
        vjp_ms = a0.elapsed_time(a1) / reps
        tk = time.perf_counter()
        it, rel, J, dJdp = s.adjoint_solve("heat", max_iter=iters, tol=0.0)
        torch.cuda.synchronize()
        tk = time.perf_counter() - tk
        return {"vjp_ms": round(vjp_ms, 3), "vjp_cell_velocity_per_s": self.N * self.K / (vjp_ms * 1e-3),
                "gmres_krylov_dim": krylov, "gmres_iterations": it,
                "s_per_gmres_iteration": round(tk / max(it, 1), 4),
                "relative_residual_after": rel,
                "arithmetic": "f32+f64" if self.precision == "mixed" and
                os.environ.get("RYKOV_ADJ_FP64", "0") in ("", "0") else "f64"}

    def close(self):
        import torch
        self.s.close()
        del self.s
        torch.cuda.empty_cache()


def fp64_peak():
    """DFMA throughput of this GPU (TFLOP/s), measured by the library's peak kernel."""
    from paper_2303_10846_gb300 import rykov as RK
    try:
        return RK.peak_tflops("fp64")
    except Exception as e:           # an older library without the entry point
        return None


def sphere_extras(args, dev, peak, peak_kind):
    """The sphere case beside the headline: mixed throughput (FP64 and FP32 macro
    solve), time to residual 1e-6, the FP64 form against min(HBM, FP64) and the
    adjoint."""
    wl = workload("sphere")
    out = {"workload": wl.name, "N": wl.mesh.n_cell, "K": wl.dvs.K}
    noop = lambda: None
    start = max(START_ITERS, wl.params.first_order_iters + 2)
    c = Case(wl, "mixed")
    c.timed(args.steps, args.warmup, start, noop)
    c.profiled(min(args.steps, 5))
    out["mixed"] = {"ms_per_step": round(c.ms, 4), "value": wl.mesh.n_cell * wl.dvs.K / (c.ms * 1e-3),
                    "roofline": c.roofline(peak, peak_kind, NCU_TRAFFIC["sphere"]),
                    "iteration_roofline": c.iteration_roofline(peak),
                    "kernels": c.kernel_table(peak)}
    if args.converge > 0:
        out["time_to_residual"] = c.converge(args.converge)
    if args.adj_iters > 0:
        c.s.iterate(args.steps)
        out["adjoint"] = c.adjoint(dev, args.adj_iters, args.adj_krylov)
        out["adjoint"]["state"] = "mixed context at the residual 1e-6 state"
    c.close()
    c = Case(wl, "mixed", macro32=True)
    c.timed(args.steps, args.warmup, start, noop)
    out["mixed_macro_fp32"] = {"ms_per_step": round(c.ms, 4),
                               "value": wl.mesh.n_cell * wl.dvs.K / (c.ms * 1e-3)}
    c.close()
    if not args.no_fp64:
        c = Case(wl, "fp64")
        n64 = max(2, min(args.steps, 5))
        c.timed(n64, 3, start, noop)
        c.profiled(2)
        pk = fp64_peak()
        d = {"ms_per_step": round(c.ms, 3), "value": wl.mesh.n_cell * wl.dvs.K / (c.ms * 1e-3),
             "iteration_roofline_hbm": c.iteration_roofline(peak),
             "kernels": c.kernel_table(peak), "fp64_peak_tflops_measured": pk}
        if pk and FP64_FLOPS_PER_CELL_VELOCITY:
            fl = FP64_FLOPS_PER_CELL_VELOCITY * wl.mesh.n_cell * wl.dvs.K
            d["fp64_flops_per_cell_velocity"] = FP64_FLOPS_PER_CELL_VELOCITY
            d["fp64_achieved_tflops"] = round(fl / (c.ms * 1e-3) / 1e12, 4)
            d["fp64_alu_frac"] = round(fl / (c.ms * 1e-3) / 1e12 / pk, 4)
        d["mixed_over_fp64_speedup"] = round(c.ms / out["mixed"]["ms_per_step"], 2)
        out["fp64"] = d
        c.close()
    return out


def config_table(args):
    """The other configurations beside the headline: the 8^3 cavity in FP64 (its run of
    200 implicit iterations from rest, and the throughput of single iterations) and the
    capsule in mixed precision (throughput over second-order iterations, then the wall
    time to residual 1e-6 from the free-stream start, capped at --capsule-cap)."""
    from paper_2303_10846_gb300 import inputs as I
    noop = lambda: None
    out = {}
    wl = I.cavity_workload()
    c = Case(wl, "fp64")
    run = c.converge(200, tol=0.0)
    c.timed(args.steps, args.warmup, max(START_ITERS, wl.params.first_order_iters + 2), noop)
    out["cavity_fp64"] = {"workload": wl.name, "N": wl.mesh.n_cell, "K": wl.dvs.K,
                          "ms_per_step": round(c.ms, 4),
                          "value": wl.mesh.n_cell * wl.dvs.K / (c.ms * 1e-3),
                          "run_200_iterations": {"wall_s": run["wall_s"],
                                                 "final_residual": run["final_residual"]}}
    c.close()
    if args.capsule_cap > 0:
        wl = I.capsule_workload()
        c = Case(wl, "mixed")
        c.timed(args.steps, args.warmup, max(START_ITERS, wl.params.first_order_iters + 2), noop)
        out["capsule_mixed"] = {"workload": wl.name, "N": wl.mesh.n_cell, "K": wl.dvs.K,
                                "ms_per_step": round(c.ms, 4),
                                "value": wl.mesh.n_cell * wl.dvs.K / (c.ms * 1e-3),
                                "time_to_residual": c.converge(args.capsule_cap)}
        c.close()
    return out


# FP64 operations per (cell, velocity) per iteration of the FP64 form: 2 x DFMA + DADD +
# DMUL summed over the per-velocity kernels (reconstruction, faces, micro flux, the 16
# micro sweeps, cell update) by ncu's instruction counters on the sphere mesh with every
# 10th velocity (K = 304), divided by N*K (the macro solve, O(N), is left out)
FP64_FLOPS_PER_CELL_VELOCITY = 1120.9


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = workload(args.workload)
    if args.kstride > 1:
        wl = dvs_sample(wl, args.kstride)
    N, K = wl.mesh.n_cell, wl.dvs.K

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    c = Case(wl, args.precision)
    clk = Clocks(local_rank)
    # the timed iterations are second-order ones: the start-up runs past the
    # workload's first-order iterations
    start = max(args.start, wl.params.first_order_iters + 2)
    c.timed(args.steps, args.warmup, start, barrier, clk)
    ms = max_over_ranks(c.ms, world, dev)
    value = job_value(N * K, world, ms)
    c.profiled(min(args.steps, 5))
    conv = c.converge(args.converge_main) if args.converge_main > 0 else None
    e2e = c.end_to_end(args.steps, world, dev, barrier)
    peak, peak_kind = _peaks()
    roof = c.roofline(peak, peak_kind, NCU_TRAFFIC.get(args.workload) if
                      (args.precision == "mixed" and args.kstride == 1) else None)
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "N": N, "K": K, "faces": wl.mesh.n_face,
                       "precision": args.precision,
                       "macro_solve": "fp64",
                       "l2": f"inputs larger than L2 (distributions {2 * N * K * c.Tsz / 1e9:.2f} GB)",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e,
            "gpu_launches": int(c.launches),
            "clocks": c.clocks,
            "roofline": roof,
            "iteration_roofline": c.iteration_roofline(peak),
            "kernels": c.kernel_table(peak),
            "ms_per_step_profiled": round(c.ms_profiled, 3),
            "time_to_residual": conv,
            "residual_after": float(np.max(c.res)),
            "wall_s_timed": c.wall,
        }
    c.close()
    if rank == 0:
        if not args.no_cpu:
            stride = CPU_STRIDE[args.workload]
            full = workload(args.workload) if args.kstride > 1 else wl
            # the iterations the GPU arm times: the same start-up and warm-up, then
            # --steps timed iterations (the oracle's time per iteration falls over the
            # first second-order iterations, so a shorter run would not compare)
            v, dt, sk, start = oracle_sample_rate(args.workload, stride, args.steps, args.warmup)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                                   "sample": cpu_sample_desc(
                                       full, sk, stride, f"{start} start-up + {args.warmup} warm-up + "
                                       f"{args.steps} timed oracle iterations")}
        else:
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle",
                                   "sample": "skipped"}
        if not args.no_extras and args.workload == "scale":
            out["sphere"] = sphere_extras(args, dev, peak, peak_kind)
            if not args.no_configs:
                out["configs"] = config_table(args)
            if conv is None:
                out["time_to_residual"] = dict(out["sphere"].get("time_to_residual") or {},
                                               workload=out["sphere"]["workload"])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="scale", choices=["scale", "sphere"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sphere case (throughput, time to residual, FP64 form, adjoint)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the sphere's FP64 form")
    ap.add_argument("--no-oracle-table", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the cavity (FP64) and capsule (mixed) rows")
    ap.add_argument("--capsule-cap", type=int, default=400,
                    help="iteration cap of the capsule's time-to-residual-1e-6 run (0: skip the capsule)")
    ap.add_argument("--start", type=int, default=START_ITERS)
    ap.add_argument("--converge", type=int, default=600,
                    help="iteration cap of the sphere's time-to-residual-1e-6 run (0: skip)")
    ap.add_argument("--converge-main", type=int, default=0,
                    help="iteration cap of a time-to-residual run on the main workload (0: skip)")
    ap.add_argument("--adj-iters", type=int, default=8,
                    help="GMRES iterations of the timed adjoint solve on the sphere (0: skip)")
    ap.add_argument("--adj-krylov", type=int, default=4)
    ap.add_argument("--kstride", type=int, default=1,
                    help="keep every S-th velocity (weights x S): the smaller case that "
                         "profiler captures of single kernels run on; not a bench line")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        out = run_gpu(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
