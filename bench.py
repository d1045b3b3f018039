"""Benchmark of the implicit Rykov iteration on GB300.

One step = one full implicit iteration (Steps 2-6: reconstruction, interface
collision and fluxes, macro PR-SGS prediction, micro PR-SGS, compensated update)
over every (cell, velocity) pair of the sphere workload: Mach 5, Kn 0.1 on the
diameter, ~62k seeded Delaunay tetrahedra in a 10R box, ~3,000-point unstructured
velocity space from the paper's DVS criterion.  Metric: cell-velocity updates/s
(N*K / time per iteration); the wall time to residual 1e-6 is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--impl reference]

--impl reference times the FP64 CPU oracle (the test oracle, as it stands) on the
host cores on a bounded sample of the same workload.  Under torchrun every rank
runs an independent replica (the path has no data-path collective); rank 0 prints
one JSON line.
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
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the kernels
# as they stand, mixed precision, full sphere workload: one ncu capture on the same mesh
# with every 5th velocity (K = 607), scaled by 3033/607 (traffic is proportional to K)
NCU_TRAFFIC_MIXED = {"k_recon": 4.731e9, "k_face_interior": 5.668e9, "k_micro_sweep": 1.706e9,
                     "k_micro_flux": 4.563e9}


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


def workload():
    from paper_2303_10846_gb300 import inputs as I
    return I.sphere_workload()


def dvs_sample(wl, stride):
    """Every stride-th velocity of the workload's DVS (weights scaled by stride):
    the bounded CPU sample of the same workload."""
    import copy
    from paper_2303_10846_gb300 import inputs as I
    w2 = copy.copy(wl)
    w2.dvs = I.DVS(u=wl.dvs.u[::stride].copy(), w=wl.dvs.w[::stride] * stride,
                   name=f"{wl.dvs.name}/every{stride}")
    w2.name = f"{wl.name}/every{stride}thvelocity_K{w2.dvs.K}"
    return w2


def cpu_oracle_rate(wl, iters=4, stride=2):
    """Oracle (FP64 C, OpenMP over cells/faces) on the host cores: updates/s on a
    DVS sample of the workload, the first `iters` implicit iterations."""
    import oracle as O
    w2 = dvs_sample(wl, stride)
    o = O.Oracle(w2)
    t0 = time.perf_counter()
    o.iterate(iters)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return (w2.mesh.n_cell * w2.dvs.K * iters / dt, cores,
            f"{iters} oracle iteration(s) of the full mesh (N={w2.mesh.n_cell}) with every "
            f"{stride}th velocity (K={w2.dvs.K} of {wl.dvs.K}), {dt:.1f} s")


def run_reference(args, rank, world):
    out = {"metric": METRIC, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic"}
    if rank != 0:
        return None
    import oracle as O
    wl = workload()
    stride = 30
    w2 = dvs_sample(wl, stride)
    o = O.Oracle(w2)
    for _ in range(args.warmup):
        o.iterate(1)
    t0 = time.perf_counter()
    o.iterate(args.steps)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = w2.mesh.n_cell * w2.dvs.K * args.steps / dt
    out.update(value=v, ms_per_step=1e3 * dt / args.steps,
               config={"workload": wl.name, "N": wl.mesh.n_cell, "K": wl.dvs.K,
                       "sample_K": w2.dvs.K, "precision": "fp64", "l2": "n/a (CPU)"},
               cpu_baseline={"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"full mesh, every {stride}th velocity (K={w2.dvs.K}), "
                                       f"{args.warmup} warm-up + {args.steps} timed iterations"},
               e2e={"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    return out


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2303_10846_gb300.rykov import Solver

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = workload()
    if args.kstride > 1:
        wl = dvs_sample(wl, args.kstride)
    N, K = wl.mesh.n_cell, wl.dvs.K
    s = Solver(wl, args.precision)
    stream = s.stream

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # start-up (first-order iterations and the CFL ramp), then warm-up
    s.iterate(args.start)
    s.iterate(args.warmup)
    barrier()
    clk = Clocks(local_rank)
    clk.start()
    _, launches0 = s.profile_get()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    t0 = time.perf_counter()
    e0.record(stream)
    rc, done, res = s.iterate(args.steps)          # CUDA-graph path
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    _, launches1 = s.profile_get()
    gpu_launches = launches1 - launches0
    # per-kernel CUDA-event durations: the same number of steps right after, with
    # every kernel class bracketed by events on the solver's stream (direct launches)
    s.profile(True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    s.iterate(args.steps)
    p1.record(stream)
    torch.cuda.synchronize()
    ms_profiled = p0.elapsed_time(p1) / args.steps
    prof, _ = s.profile_get()
    s.profile(False)
    ms = max_over_ranks(ms, world, dev)
    value = job_value(N * K, world, ms)

    # wall time to residual 1e-6 from the initial field (graph path; the residual
    # is read back every iteration to test convergence)
    conv = None
    if args.converge > 0:
        s.set_state_prim(wl.prim0)
        barrier()
        tc = time.perf_counter()
        rc3, n3, res3 = s.iterate(args.converge, tol=1e-6)
        torch.cuda.synchronize()
        tconv = time.perf_counter() - tc
        conv = {"tol": 1e-6, "iterations": n3, "wall_s": round(tconv, 4),
                "reached": bool(rc3 == 0 and float(np.max(res3)) < 1e-6),
                "final_residual": float(np.max(res3))}

    # end to end through the public API with host buffers: a restart from a host
    # checkpoint (W, q and the distributions in pinned host memory, uploaded by
    # rk_set_state), the same second-order iterations as the timed region with the
    # residual read back to the host every iteration, then W and q read back
    from paper_2303_10846_gb300.rykov import _ptr
    import dataclasses
    s.set_params(dataclasses.replace(wl.params, first_order_iters=0))
    s.iterate(1)                                   # capture the graph for these params
    Wh = torch.empty((N, 6), dtype=torch.float64).pin_memory()
    qh = torch.empty((N, 6), dtype=torch.float64).pin_memory()
    s._check(s.L.rk_moments(s.h, _ptr(Wh), _ptr(qh), None, 0))
    dist = s.get_distribution().cpu().pin_memory()
    barrier()
    t1 = time.perf_counter()
    s._check(s.L.rk_set_state(s.h, _ptr(Wh), _ptr(qh), _ptr(dist), 0))
    rc2, done2, _ = s.iterate(args.steps, tol=1e-300)
    s._check(s.L.rk_moments(s.h, _ptr(Wh), _ptr(qh), None, 0))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t1
    e2e_s = max_over_ranks(e2e_s, world, dev)
    up = (Wh.numel() + qh.numel()) * 8 + dist.numel() * dist.element_size()
    e2e = {"value": job_value(N * K * done2, world, e2e_s * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(up / done2),
           "d2h_bytes_per_step": int(6 * 8 + (Wh.numel() + qh.numel()) * 8 / done2)}
    s.set_params(wl.params)

    # adjoint of the steady residual at the context's state (FP32 per-velocity
    # arithmetic with compensated sums in a mixed context, FP64 in an FP64 one): one
    # vector-Jacobian product, and a fixed number of GMRES iterations of the adjoint solve
    adj = None
    if args.adj_iters > 0:
        s.bind_adjoint(args.adj_krylov)
        gen = torch.Generator(device=dev).manual_seed(1)
        v = torch.randn(s.state_len, dtype=torch.float64, device=dev, generator=gen)
        s.vjp(v)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        a0.record(stream)
        for _ in range(reps):
            s.vjp(v)
        a1.record(stream)
        torch.cuda.synchronize()
        vjp_ms = a0.elapsed_time(a1) / reps
        tk = time.perf_counter()
        it, rel, J, dJdp = s.adjoint_solve("heat", max_iter=args.adj_iters, tol=0.0)
        torch.cuda.synchronize()
        tk = time.perf_counter() - tk
        adj = {"vjp_ms": round(vjp_ms, 3),
               "vjp_cell_velocity_per_s": N * K / (vjp_ms * 1e-3),
               "gmres_krylov_dim": args.adj_krylov, "gmres_iterations": it,
               "s_per_gmres_iteration": round(tk / max(it, 1), 4),
               "relative_residual_after": rel,
               "arithmetic": "f32+f64" if args.precision == "mixed" and
               os.environ.get("RYKOV_ADJ_FP64", "0") in ("", "0") else "f64",
               "state": f"{args.precision} context after {args.steps} end-to-end iterations"}

    out = None
    if rank == 0:
        peak, peak_kind = _peaks()
        Tsz = 4 if args.precision == "mixed" else 8
        # dominant kernel class and its roofline (algorithmic bytes per launch from the
        # per-unit word counts below)
        F, Fi = wl.mesh.n_face, int((wl.mesh.face_cell[:, 1] >= 0).sum())
        nnz = 2 * Fi + (F - Fi)
        # kernels (the micro sweep's first / middle / last launches are one kernel)
        kern = {
            "k_recon": prof["recon"], "k_face_interior": prof["face_interior"],
            "k_face_boundary": prof["face_boundary"], "k_macro (prep + PR-SGS + finish)": prof["macro_sgs"],
            "k_micro_sweep": tuple(map(sum, zip(prof["micro_sweep_first"], prof["micro_sweep_mid"],
                                                prof["micro_sweep_last"]))),
        }
        nsw = 2 * 2                                     # 2 x (forward + backward)
        # algorithmic words per unit per step (each input element read once, each output
        # written once): micro sweeps 10 (first: phi, F, neighbour dphi; Res, dphi) +
        # 6 per middle sweep (Res, neighbour dphi; dphi) + 10 (last: Res, neighbour dphi,
        # phi; phi, dphi) per (cell, k); recon 2 per (cell, k) + 2 per (face, k); faces 4
        # per (face, k)
        algo_step = {
            "k_micro_sweep": (10 + 6 * (nsw - 2) + 10) * N * K * Tsz,
            "k_recon": (2 * N * K + 2 * F * K) * Tsz,
            "k_face_interior": 4 * Fi * K * Tsz,
        }
        name, (tms, cnt) = max(kern.items(), key=lambda kv: kv[1][0])
        roof = None
        if name in algo_step and cnt:
            launches_per_step = cnt / args.steps
            bytes_launch = algo_step[name] / launches_per_step
            ach = bytes_launch / (tms / cnt * 1e-3) / 1e9
            roof = {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(ach / peak, 4),
                    "traffic": (NCU_TRAFFIC_MIXED.get(name) if args.precision == "mixed"
                                and args.kstride == 1 else None),
                    "peak_kind": peak_kind, "launches_per_step": launches_per_step,
                    "algorithmic_bytes_per_launch": int(bytes_launch),
                    "share_of_step": round(tms / (ms_profiled * args.steps), 4),
                    "timing": "CUDA events around every launch of the kernel on the solver "
                              "stream, in a profiled pass of the same number of steps run "
                              "right after the timed (graph) region"}
        # whole iteration against the 52-word per (cell, velocity) model
        iter_bytes = 52 * Tsz * N * K
        cpu_v, cores, sample = cpu_oracle_rate(wl) if not args.no_cpu else (None, 0, "skipped")
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "N": N, "K": K, "faces": F,
                       "precision": args.precision,
                       "l2": f"inputs larger than L2 (distributions {2 * N * K * Tsz / 1e9:.2f} GB)",
                       "parallelism": f"replicas x{world}"},
            "e2e": e2e,
            "gpu_launches": int(gpu_launches),
            "clocks": clocks,
            "roofline": roof,
            "iteration_roofline": {"model_bytes_per_cell_velocity": 52 * Tsz,
                                   "achieved": round(iter_bytes / (ms * 1e-3) / 1e9, 1),
                                   "peak": peak, "frac": round(iter_bytes / (ms * 1e-3) / 1e9 / peak, 4)},
            "kernel_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items()},
            "ms_per_step_profiled": round(ms_profiled, 3),
            "time_to_residual": conv,
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "residual_after": float(np.max(res)),
            "adjoint": adj,
            "wall_s_timed": wall,
        }
    s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--start", type=int, default=START_ITERS)
    ap.add_argument("--converge", type=int, default=600,
                    help="iteration cap of the time-to-residual-1e-6 run (0: skip)")
    ap.add_argument("--adj-iters", type=int, default=8,
                    help="GMRES iterations of the timed adjoint solve (0: skip the adjoint)")
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
