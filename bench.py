#!/usr/bin/env python
"""GenEO-PCG throughput on one GB300: PCG DOF-iterations/s at 1e-10 relative residual.

Workload (default): the curved corner-unfolding laminate, 90-degree arc of
5 mm inner radius with 50 mm limbs, 12 plies [0/90/+45/-45/0/90]s of 0.25 mm
with 0.02 mm resin interfaces, 4 Q2 elements through every layer, 100
elements on the arc + 10 per limb, 30 across a 15 mm width: 120 x 30 x 92
triquadratic hexahedra, 8,159,055 DOF, a Gaussian fibre-misalignment field of
10 degrees amplitude and 4 mm width at mid-arc, limb 1 clamped and a rigid
opening rotation of the limb-2 end.  128 overlapping subdomains (32 x 4
in-plane, full thickness, overlap 1), 10 GenEO eigenvectors each, FP64.

A step = one full PCG solve (to ||r||/||f|| <= 1e-10) of K u = f with the
device-resident load vector, followed by the stress recovery; the setup
(geometry, factorisations, GenEO coarse space) runs once before the warm-up
and is reported as setup_s.  value = free DOFs x PCG iterations / solve time.

Other configurations (--config): corner_small (a 32x8x23 dry-run case),
corner_wide / corner_mixed (the 120x45x92 corner, 12,171,705 DOF, in FP64 or
with FP32 local factors; --compare-fp64 adds the FP64 solve of the same
laminate and reports the differences), batch (96 flat laminates solved
together, autotuned decompositions) and adjoint (the gradient of the resin
stress p-norm with respect to every element's misalignment angle) and
paper_corner (the paper's 39-ply wrinkle-study geometry with its sech^2
wrinkle, 13,559,865 DOF, mixed precision).

--impl reference times the CPU oracle (oracle/), as it stands, on a bounded
sample of the same laminate family on the host cores.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG DOF-iterations/s at 1e-10 rel. residual; K*u HBM GB/s vs peak"
# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one FP64
# local-solve application per algorithmic byte, measured over the 20 launches
# of one application on the 151,011-DOF 32x8x23 corner; every panel is read
# once, so it scales with the panels to the full-size workload.
FP64_LOCAL_TRAFFIC_PER_ALG_BYTE = 1.076
UNIT = "DOF-iterations/s"
FP64_FMA_PER_SM_CLK = 2        # nominal FP64 FMA rate per SM and clock of this part (context only)


def fp64_peak(device):
    """FP64 peak measured in this run by the library's FMA probe (no memory
    traffic, 8 independent chains per thread, 8 blocks of 256 per SM), with the
    SM clocks sampled meanwhile; the nominal rate n_SM x 2 FMA/clk x 2 flop x
    max clock is reported beside it."""
    from paper_1707_04228_gb300 import lib
    with ClockSampler(device) as clk:
        flops, n_sm, ms = lib.fp64_peak_probe(device, iters=8192, reps=40)
    c = clk.summary()
    mx = c["sm_max_mhz"] or 2070.0
    return {"tflops": flops / 1e12, "n_sm": n_sm, "ms": ms, "clocks": c,
            "nominal_tflops": n_sm * FP64_FMA_PER_SM_CLK * 2 * mx * 1e6 / 1e12}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(name):
    from paper_1707_04228_gb300 import inputs
    if name == "corner":
        lam = inputs.corner_c1()
        lam.px, lam.py, lam.pz, lam.nev = 32, 4, 1, 10
        desc = ("curved_corner_120x30x92_q2: 8,159,055 DOF, 128 subdomains (32x4x1 in-plane, overlap 1), "
                "10 GenEO eigenvectors each, FP64, tol 1e-10")
    elif name in ("corner_wide", "corner_mixed"):
        lam = inputs.curved_corner(n_width=45, width=22.5, name="curved_corner_120x45x92")
        lam.px, lam.py, lam.pz, lam.nev = 32, 4, 1, 10
        mixed = name == "corner_mixed"
        lam.precision = 1 if mixed else 0
        lam.tol = 1e-8 if mixed else 1e-10
        desc = ("curved_corner_120x45x92_q2: 12,171,705 DOF, 128 subdomains (32x4x1), 10 eigenvectors, "
                + ("mixed (FP32 local factors and sweeps, FP64 CG/K*u/coarse), tol 1e-8" if mixed
                   else "FP64, tol 1e-10"))
    elif name == "paper_corner":
        lam = inputs.paper_corner()
        lam.precision = 1
        lam.tol = 1e-8
        desc = ("paper_corner_120x60x77_q2: the 39-ply wrinkle-study geometry (R 22 mm, 10 mm limbs, 52 mm width, "
                "0.24/0.015 mm plies/resin, sech^2 wrinkle of 0.62 mm), 13,559,865 DOF, 128 subdomains (32x4x1), "
                "10 eigenvectors, mixed (FP32 local factors and sweeps), tol 1e-8")
    elif name == "paper_corner_periodic":
        lam = inputs.paper_corner(nsub=(32, 1, 1), periodic=True)
        lam.precision = 1
        lam.tol = 1e-8
        desc = ("paper_corner_120x60x77_q2 with periodic width conditions (the 39-ply wrinkle study: R 22 mm, 10 mm "
                "limbs, 52 mm width, sech^2 wrinkle of 0.62 mm), 13,559,865 DOF, 32 subdomains spanning the width, "
                "10 eigenvectors, mixed (FP32 local factors and sweeps), tol 1e-8")
    elif name in ("corner_small", "corner_small_mixed"):
        lam = inputs.curved_corner(n_arc=24, n_limb=4, n_width=8, nel_layer=1, name="curved_corner_small",
                                   nsub=(8, 2, 1), nev=10)
        mixed = name == "corner_small_mixed"
        lam.precision = 1 if mixed else 0
        lam.tol = 1e-8 if mixed else 1e-10
        desc = ("curved_corner_32x8x23_q2 (small dry-run case), 16 subdomains, 10 eigenvectors, "
                + ("mixed, tol 1e-8" if mixed else "FP64, tol 1e-10"))
    else:
        raise SystemExit(f"unknown config {name}")
    return lam, desc


def oracle_sample():
    """Bounded CPU sample of the same family: a 16x3x23 curved corner (12 plies,
    1 element per layer), 8 in-plane subdomains, 10 eigenvectors."""
    from paper_1707_04228_gb300 import inputs
    lam = inputs.curved_corner(n_arc=12, n_limb=2, n_width=3, nel_layer=1, width=3.0, limb_L=5.0,
                               name="curved_corner_16x3x23", nsub=(8, 1, 1), nev=10, wrinkle_w=1.0)
    return lam


def run_oracle(steps, warmup, max_seconds=None):
    """Times the oracle's PCG solve (setup excluded); returns dict."""
    from oracle import fem, geneo
    lam = oracle_sample()
    sysm = fem.System(fem.Mesh(lam))
    dec = geneo.Decomposition(sysm, lam.px, lam.py, lam.pz, lam.overlap)
    P = geneo.GenEO(dec, lam.nev)
    nfree = sysm.free.size
    for _ in range(warmup):
        geneo.pcg(sysm.Kff, sysm.ff, P.apply, tol=lam.tol)
    t_tot, it_tot, done, cpu_tot = 0.0, 0, 0, 0.0
    for _ in range(steps):
        t0, c0 = time.perf_counter(), time.process_time()
        _, it, _ = geneo.pcg(sysm.Kff, sysm.ff, P.apply, tol=lam.tol)
        t_tot += time.perf_counter() - t0
        cpu_tot += time.process_time() - c0
        it_tot += it
        done += 1
        if max_seconds and t_tot > max_seconds:
            break
    return {"value": nfree * it_tot / t_tot, "unit": UNIT, "cores": max(1, round(cpu_tot / t_tot)), "kind": "oracle",
            "sample": f"{lam.name}: {nfree} free DOF, {lam.px}x{lam.py}x{lam.pz} subdomains, nev {lam.nev}, "
                      f"{done} PCG solve(s) of {it_tot // max(done, 1)} iterations, setup excluded; "
                      f"SciPy SuperLU/sparse; cores = process CPU time / wall time over the timed solves",
            "ms_per_step": 1e3 * t_tot / done}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def shard_worklist(costs, world):
    """Static split of independent laminates over `world` replicas: largest
    first, each to the least loaded rank (ties to the lower rank).  Returns
    one sorted index list per rank; every index appears exactly once."""
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(o) for o in out]


def run_batch(args, rank=0, local_rank=0, world=1):
    """96 flat laminates of 40k-800k DOF solved together (one launch per phase,
    graph-replayed iterations, autotuned decompositions, FP64 CG with FP32
    local factors); value = sum of free DOFs x iterations over all laminates
    per second of the batched solve.  With N replicas the laminates are split
    by shard_worklist (by DOF) and each rank solves its share as one batch; the
    whole-job value is the sum of all ranks' work over the slowest rank's time."""
    import torch
    from paper_1707_04228_gb300 import inputs, lib
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    all_lams = inputs.batch_plates(count=args.count, nev=8)
    mine = shard_worklist([l.n_dof for l in all_lams], world)[rank]
    lams = [all_lams[i] for i in mine]
    t0 = time.perf_counter()
    b = lib.Batch(lams, device=local_rank)
    b.setup(px=0, py=0, nev=8, tol=1e-8, precision=lib.GL_PREC_MIXED, max_iter=3000)
    setup_s = time.perf_counter() - t0
    outs = [torch.empty(l.n_dof, dtype=torch.float64, device=dev) for l in lams]
    for _ in range(args.warmup):
        _, infos = b.solve(outs)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    units, ms = 0, 0.0
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            t1 = time.perf_counter()
            _, infos = b.solve(outs)
            torch.cuda.synchronize()
            ms += 1e3 * (time.perf_counter() - t1)
            units += sum(i["n_free"] * i["iters"] for i in infos)
    if world > 1:
        dist.barrier()
    t_max, units = aggregate_ranks(ms, units, world, dev)
    grid = b.grid().tolist()
    if rank == 0:
        line = {"metric": METRIC, "value": units / (t_max / 1e3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / max(args.steps, 1),
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64+f32",
                "data": "synthetic",
                "config": {"workload": f"batch of {len(all_lams)} flat laminates, "
                                       f"{sum(l.n_dof for l in all_lams):,} DOF in total, autotuned in-plane grids, "
                                       f"8 eigenvectors, mixed, tol 1e-8",
                           "parallelism": "replicas (laminates split by DOF)" if world > 1 else "single GPU"},
                "setup_s": setup_s, "iters": [i["iters"] for i in infos],
                "rel_resid_true_max": max(i["rel_resid_true"] for i in infos), "grids": grid,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    b.close()
    if world > 1:
        dist.destroy_process_group()


def run_adjoint(args):
    """Adjoint gradient on the curved corner (8,159,055 DOF): J = ||s33||_8 over the
    resin elements of the arc, differentiated through torch.autograd with respect
    to every element's misalignment angle (one forward and one adjoint PCG solve
    per gradient).  value = free DOFs x (forward + adjoint iterations) per second;
    gradient_s = the time of one gradient.  --fd N compares N patch components
    drawn with seed 4228 with central differences (h = 1e-6 rad), each
    perturbed state reached by an increment solve from u(theta0)."""
    import torch
    from paper_1707_04228_gb300 import inputs, lib
    from paper_1707_04228_gb300.autograd import pnorm, stress_of_theta
    lam, _ = workload("corner")
    t0 = time.perf_counter()
    s = lib.Solver.from_laminate(lam, max_iter=5000)
    setup_s = time.perf_counter() - t0
    dev = torch.device("cuda", 0)
    f = torch.empty(s.n_dof, dtype=torch.float64, device=dev)
    s.rhs(out=f)
    mask = torch.tensor(inputs.arc_resin_mask(lam), device=dev)
    patch = inputs.wrinkle_patch_mask(lam)
    theta0 = torch.tensor(np.ascontiguousarray(lam.theta).reshape(-1), dtype=torch.float64, device=dev)

    def gradient():
        th = theta0.clone().requires_grad_(True)
        J = pnorm(stress_of_theta(th, s, f), mask, 8)
        J.backward()
        return J, th.grad, s.last_info["iters"] + s.last_adjoint_info["iters"]

    for _ in range(args.warmup):
        gradient()
    torch.cuda.synchronize()
    units, its = 0, []
    with ClockSampler(0) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            J, g, it = gradient()
            units += s.last_info["n_free"] * it
            its.append(it)
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    gfull = g.cpu().numpy()
    gp = gfull[patch]
    fd = []
    if args.fd > 0:
        # args.fd patch parameters drawn with seed 4228; J(theta0 +- h e_k) by increment solves from u(theta0)
        from paper_1707_04228_gb300.autograd import theta_central_differences
        elems = np.random.default_rng(4228).choice(np.flatnonzero(patch), args.fd, replace=False)
        t_fd = time.perf_counter()
        vals = theta_central_differences(s, lam.nx, lam.ny, theta0, elems, mask, 8, 1e-6, f)
        fd_s = time.perf_counter() - t_fd
        for e, d in zip(elems, vals):
            fd.append({"elem": int(e), "adjoint": float(gfull[e]), "fd": d,
                       "rel_diff": abs(d - gfull[e]) / abs(gfull[e])})
        rd = [x["rel_diff"] for x in fd]
        fd = {"n": len(fd), "h": 1e-6, "seed": 4228, "max_rel_diff": max(rd), "median_rel_diff": float(np.median(rd)),
              "time_s": fd_s, "samples": fd}
    line = {"metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "adjoint gradient dJ/dtheta, J = ||s33||_8 over the arc resin elements of "
                                   "curved_corner_120x30x92_q2 (8,159,055 DOF, 32x4x1 subdomains, nev 10, FP64, "
                                   "tol 1e-10); one forward + one adjoint PCG solve per step",
                       "n_params_patch": int(patch.sum())},
            "gradient_s": ms / 1e3 / max(args.steps, 1), "setup_s": setup_s, "iters_per_gradient": its,
            "J": J.item(), "grad_patch_norm": float(np.linalg.norm(gp)), "fd_check": fd,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def aggregate_ranks(ms, units, world, device):
    """Whole-job figures of independent replicas: the slowest rank's time and the
    sum of the work units of all ranks (no collective touches the solve itself)."""
    if world <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms, float(units)], dtype=torch.float64, device=device)
    mx = tt.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return mx[0].item(), tt[1].item()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="corner")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--count", type=int, default=96, help="laminates in --config batch")
    ap.add_argument("--fd", type=int, default=0, help="central-difference checks in --config adjoint")
    ap.add_argument("--fp32-update", type=int, default=0, choices=[0, 1],
                    help="mixed precision: trailing updates of the FP32 factors on the tensor cores (0) or the "
                         "FP32 CUDA cores (1)")
    ap.add_argument("--sweep-overlap", type=int, default=0,
                    help="local solves: overlap the sweeps of two halves of the subdomains, their top N levels "
                         "on a high-priority stream (0: the library default, -1: sequential)")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="after a mixed-precision run, solve the same laminate in FP64 and report the differences")
    args = ap.parse_args()
    rank, local_rank, world = dist_env()
    if args.config == "batch" and args.impl == "ours":
        run_batch(args, rank, local_rank, world)
        return
    if args.config == "adjoint" and args.impl == "ours":
        if rank == 0:
            run_adjoint(args)
        return

    if args.impl == "reference":
        if rank != 0:
            return
        lam, desc = workload(args.config)
        r = run_oracle(args.steps, min(args.warmup, 1), max_seconds=150)
        line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": desc, "reference_sample": r["sample"]},
                "cpu_baseline": {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_1707_04228_gb300 import lib

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    lam, desc = workload(args.config)
    t0 = time.perf_counter()
    prec = getattr(lam, "precision", 0)
    s = lib.Solver.from_laminate(lam, device=local_rank, precision=prec, max_iter=5000,
                                 fp32_update=args.fp32_update, sweep_overlap=args.sweep_overlap)
    setup_s = time.perf_counter() - t0
    N, NE = s.n_dof, s.n_elem
    dev = torch.device("cuda", local_rank)
    f = torch.empty(N, dtype=torch.float64, device=dev)
    s.rhs(out=f)
    u = torch.empty(N, dtype=torch.float64, device=dev)
    s33 = torch.empty(NE, dtype=torch.float64, device=dev)
    t13 = torch.empty(NE, dtype=torch.float64, device=dev)
    info = None
    for _ in range(args.warmup):
        _, info = s.solve(f, out=u)
        s.stress(u, s33, t13)
    torch.cuda.synchronize()
    probe = fp64_peak(local_rank)
    FP64_PEAK_TFLOPS = probe["tflops"]

    def barrier():
        if world > 1:
            dist.barrier()

    launches0 = s.kernel_launches()
    iters = 0
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            _, info = s.solve(f, out=u)
            s.stress(u, s33, t13)
            iters += info["iters"]
        ev1.record()
        torch.cuda.synchronize()
        barrier()
    launches = s.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    t_max, units = aggregate_ranks(ms, info["n_free"] * iters, world, dev)
    value = units / (t_max / 1e3)

    # end to end through the public API with host buffers (pinned f in, u out)
    f_h = torch.empty(N, dtype=torch.float64).pin_memory()
    f_h.copy_(f.cpu())
    u_h = torch.empty(N, dtype=torch.float64).pin_memory()
    f_np, u_np = f_h.numpy(), u_h.numpy()
    t1 = time.perf_counter()
    e_iters = 0
    for _ in range(max(1, args.steps)):
        _, inf2 = s.solve(f_np, out=u_np)
        e_iters += inf2["iters"]
    e2e_s = time.perf_counter() - t1
    e2e = {"value": info["n_free"] * e_iters / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * N,
           "d2h_bytes_per_step": 8 * N}

    # phase timing pass (separate from the timed steps)
    s.profile(1)                 # phases in the solve's own schedule
    s.solve(f, out=u)
    prof = s.profile_read()
    s.profile(2)                 # and every dissection level, the levels one after another
    s.solve(f, out=u)
    prof_seq = s.profile_read()
    lv = s.profile_levels()
    s.profile(False)
    hbm, hbm_src = peaks()
    # algorithmic work of one local-solve phase: every nonzero of the lower-triangular
    # factors is read once per sweep and used in one FMA per sweep (2 sweeps)
    fe, bpe = prof["factor_nonzeros"], prof["factor_bytes_per_entry"]
    loc_bytes = 2 * fe * bpe + 6 * prof["local_dofs"] * 8          # factors read twice + local vectors
    loc_flops = 4 * fe
    loc_ms = prof["ms_local"] / max(prof["n_local"], 1)
    ku_bytes = 16 * N + NE * (36 + 270) * 8                         # x in, y out, C_e and Gauss-point J^-1, w|J|
    ku_flops = NE * (2 * 5346 + 162)                                # collocation sum factorisation: FMA, MUL
    ku_ms = prof["ms_ku"] / max(prof["n_ku"], 1)
    per_iter = {"ku_ms": ku_ms, "local_ms": loc_ms, "coarse_ms": prof["ms_coarse"] / max(prof["n_coarse"], 1),
                "local_ms_levels_in_sequence": prof_seq["ms_local"] / max(prof_seq["n_local"], 1)}
    loc_tf = loc_flops / (loc_ms / 1e3) / 1e12
    fp64 = bpe == 8
    if fp64:
        roof = {"bound": "alu", "achieved": loc_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": loc_tf / FP64_PEAK_TFLOPS, "traffic": FP64_LOCAL_TRAFFIC_PER_ALG_BYTE * loc_bytes,
                "traffic_note": "bytes per application: the ratio of DRAM to algorithmic bytes measured by ncu "
                                "on the 32x8x23 corner times this workload's algorithmic bytes",
                "kernel": "local forward/backward supernodal sweeps (all levels) + gather/scatter",
                "hbm_gbs": loc_bytes / (loc_ms / 1e3) / 1e9, "hbm_frac": loc_bytes / (loc_ms / 1e3) / 1e9 / hbm,
                "peak_note": f"FP64 peak measured in this run by the FMA probe ({probe['n_sm']} SMs, nominal "
                             f"{probe['nominal_tflops']:.3f} TFLOP/s); HBM {hbm} GB/s {hbm_src}"}
    else:
        gbs = loc_bytes / (loc_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                "kernel": "local forward/backward supernodal sweeps (all levels) + gather/scatter",
                "peak_note": f"HBM {hbm_src}"}
    # per dissection level: sweep times per application and their rate (FP64: FMA pipe; FP32: HBM)
    nc = max(lv["calls"], 1)
    levels = {"fronts": lv["fronts"].tolist(), "nonzeros": lv["nonzeros"].tolist(),
              "padded_entries": lv["padded"].tolist(), "max_front": lv["max_front"].tolist(),
              "fwd_us": [round(1e3 * t / nc, 1) for t in lv["fwd_ms"]],
              "bwd_us": [round(1e3 * t / nc, 1) for t in lv["bwd_ms"]]}
    for k in ("fwd", "bwd"):
        ms_k = lv[k + "_ms"] / nc
        if fp64:
            rate = [2 * z / (t / 1e3) / 1e12 / FP64_PEAK_TFLOPS if t > 0 else 0.0
                    for z, t in zip(lv["nonzeros"], ms_k)]
        else:
            rate = [z * bpe / (t / 1e3) / 1e9 / hbm if t > 0 else 0.0 for z, t in zip(lv["nonzeros"], ms_k)]
        levels[k + "_frac"] = [round(r, 3) for r in rate]
    levels["frac_of"] = "measured FP64 FMA peak" if fp64 else "measured HBM copy bandwidth"
    ku = {"hbm_gbs": ku_bytes / (ku_ms / 1e3) / 1e9, "hbm_frac": ku_bytes / (ku_ms / 1e3) / 1e9 / hbm,
          "fp64_tflops": ku_flops / (ku_ms / 1e3) / 1e12,
          "fp64_frac": ku_flops / (ku_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS, "ms": ku_ms,
          "bytes_per_launch": ku_bytes, "flops_per_launch": ku_flops}

    # mixed precision against the plain FP64 form on the same laminate (after the timing)
    vs_fp64 = None
    if args.compare_fp64 and prec == 1:
        _, peak_m = s.stress(u, s33, t13)[::2]
        u_m = u.cpu().numpy()
        it_m = info["iters"]
        s.close()
        t2 = time.perf_counter()
        s64 = lib.Solver.from_laminate(lam, device=local_rank, precision=0, tol=1e-10, max_iter=5000)
        setup64 = time.perf_counter() - t2
        _, info64 = s64.solve(f, out=u)
        _, peak64 = s64.stress(u, s33, t13)[::2]
        u64 = u.cpu().numpy()
        vs_fp64 = {"rel_l2_u": float(np.linalg.norm(u_m - u64) / np.linalg.norm(u64)),
                   "rel_peak_s33": float(abs(peak_m - peak64) / abs(peak64)),
                   "iters_mixed": it_m, "iters_fp64_1e-10": info64["iters"], "setup_fp64_s": setup64,
                   "rel_resid_true_fp64": info64["rel_resid_true"]}
        s64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = run_oracle(3, 1, max_seconds=40)
        cpu = {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max / max(args.steps, 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f64+f32",
                "data": "synthetic",
                "config": {"workload": desc, "l2": "inputs larger than L2 (local factors of "
                           f"{fe * bpe / 1e9:.1f} GB stream every iteration)",
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "stop": ("recurrence residual ||r||/||f|| <= tol; the FP64 true residual "
                                    "||f - K u||/||f|| is reported as rel_resid_true" if prec == 0 else
                                    "FP64 true residual ||f - K u||/||f|| <= tol")},
                "roofline": roof, "ku": ku, "per_iteration": per_iter, "levels": levels, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk.summary(), "fp64_probe": probe, "gpu_launches": launches, "setup_s": setup_s,
                "iters_per_solve": iters / max(args.steps, 1), "rel_resid_true": info["rel_resid_true"],
                "n_free": info["n_free"], "factor_nonzeros": fe, "n_coarse": info["n_coarse"]}
        if prec == 1:
            line["config"]["fp32_update"] = ("tensor cores (tcgen05 kind::tf32, 3xTF32 split, rank-128 panels)"
                                             if args.fp32_update == 0 else "FP32 CUDA cores (rank-32)")
        if vs_fp64 is not None:
            line["vs_fp64"] = vs_fp64
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
