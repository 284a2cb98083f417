#!/usr/bin/env python
"""Benchmark of the BRAS-PCG mass solve on one B300 (or N replicas under torchrun).

Workload (the H1 configuration of the headline metric): unit cube, 48^3 cells x 6 Kuhn
tetrahedra = 663,552 cells, interior vertices jittered by U(-0.15h, 0.15h) (seed 0), H1
Lagrange p = 1, 2, 3, 4 at the GLL-based nodes of the paper's nodal variant (117,649 / 912,673
/ 3,048,625 / 7,189,057 dofs), right-hand side
N(0, 1) (seed 1), u_0 = 0, stop at ||r||/||b|| <= 1e-10 (Sec. 3).  One step = one solve for
each of the four orders with the library's fast path: BRAS-preconditioned CG in FP32 (FP64
dot products and scalars) inside FP64 iterative refinement, the TRUE FP64 residual tested.
The metric is conforming dofs solved per second (sum of n over the step / step time).
Setup (tables, element inverses) is excluded, as in the paper.

Every timed answer is checked afterwards by its true FP64 residual from the FP64 mass apply
(`true_relres_fp64`, must be <= 1e-10).  Also in the same JSON line: plain FP64 BRAS-PCG and
FP64 Jacobi-PCG on the same GPU (top level, `fp64_bras_pcg`, `fp64_jacobi_pcg`); comparison
rows (mixed Jacobi-PCG; 32 right-hand sides at p = 2, 4; 64 right-hand sides on H(curl) k = 1..3,
mixed vs FP64 BRAS vs FP64 Jacobi; the FP64 damped fixed point and Chebyshev iterations of Sec. 3;
the Bernstein basis with BRAS vs Jacobi; the batched H(div) solves RT k = 1..3 over 256 meshes;
the differentiable weighted solve, forward and backward; kappa_hat by CG-Lanczos; the mixed
Poisson Schur apply), the end-to-end number through host buffers, live CUDA-event timings of
the apply kernels (H1 p = 1..4 and the streamed N1curl k = 3 inverses on 40^3 x 6 tets), the
roofline of the dominant kernel and of the streamed path, and the FP64 CPU oracle baselines
(one thread, and one independent solve per host core).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BRAS-PCG mass-solve DOF/s to 1e-10 rel. residual vs Jacobi-PCG; bras_apply GB/s vs HBM peak"
WORKLOAD = ("H1 Lagrange (GLL-based nodes) p=1,2,3,4 on 48^3x6 Kuhn tets (663,552), jitter 0.15h, 1 RHS N(0,1), "
            "rtol 1e-10")
SPACE = "h1g"   # Lagrange at the GLL-based nodes of Sec. 3 (equal to the equispaced basis for p <= 2)
N_CELLS = 48
JITTER = 0.15


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--orders", default="1,2,3,4")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched multi-mesh rows")
    ap.add_argument("--no-c3", action="store_true", help="skip the 64-RHS H(curl) rows")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t: float, ws: int, device="cpu") -> float:
    """The slowest rank's time: every rank gets the same value (identity on one rank)."""
    if ws <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(units_per_rank: float, t_max: float, ws: int) -> float:
    """Replicas: every rank solves the same fixed workload, so the job rate is the units of all
    ranks over the slowest rank's time (weak scaling)."""
    return ws * units_per_rank / t_max


# ---- CPU oracle timing (the baseline leg; the only place bench.py runs the oracle) ----------
def oracle_solve_rate(orders=(1, 2), repeats=3):
    """FP64 oracle BRAS-PCG (assembled CSR M and BRAS, scipy) on the same inputs; setup
    excluded; mean of `repeats` solves per order (Sec. 3 reports means of 3)."""
    from oracle.assembly import Problem
    from oracle.solvers import pcg
    from paper_2607_12138_b300 import meshgen as mg
    mesh = mg.unit_cube_mesh(N_CELLS, jitter=JITTER, seed=0)
    tot_n, tot_t, detail = 0, 0.0, []
    for p in orders:
        n, l2g, s = mg.dof_map(mesh, SPACE, p)
        pr = Problem(mesh, SPACE, p, l2g, s, n)
        b = mg.rhs(n, 1, seed=1)
        ts = []
        for _ in range(repeats):
            t0 = time.perf_counter()
            _, its, hist = pcg(pr.mass_apply, b, pr.bras_apply, rtol=1e-10)
            ts.append(time.perf_counter() - t0)
        t = float(np.mean(ts))
        tot_n += n
        tot_t += t
        detail.append({"p": p, "n": n, "its": its, "s": round(t, 4)})
    return tot_n / tot_t, detail


def _oracle_worker(args):
    """One process of the all-cores leg: build the oracle problem of order p (its own RHS
    seed), wait for the others, then time one solve."""
    p, seed, barrier = args
    from oracle.assembly import Problem
    from oracle.solvers import pcg
    from paper_2607_12138_b300 import meshgen as mg
    mesh = mg.unit_cube_mesh(N_CELLS, jitter=JITTER, seed=0)
    n, l2g, s = mg.dof_map(mesh, SPACE, p)
    pr = Problem(mesh, SPACE, p, l2g, s, n)
    b = mg.rhs(n, 1, seed=seed)
    barrier.wait()
    t0 = time.perf_counter()
    pcg(pr.mass_apply, b, pr.bras_apply, rtol=1e-10)
    return n, time.perf_counter() - t0


def oracle_all_cores_rate(p=2, max_procs=16):
    """Throughput of the FP64 oracle on all host cores: one independent single-threaded
    BRAS-PCG solve per process (order p, one right-hand side each, started together after
    their setups); rate = all processes' dofs / the slowest solve."""
    import multiprocessing as mp
    procs = max(1, min(os.cpu_count() or 1, max_procs))
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        barrier = man.Barrier(procs)
        with ctx.Pool(procs) as pool:
            res = pool.map(_oracle_worker, [(p, 1 + i, barrier) for i in range(procs)])
    tot_n = sum(r[0] for r in res)
    t_max = max(r[1] for r in res)
    return tot_n / t_max, procs, t_max


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    orders = (1, 2)
    for _ in range(a.warmup):
        oracle_solve_rate(orders, repeats=1)
    vals, t_all = [], []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        v, detail = oracle_solve_rate(orders, repeats=1)
        t_all.append(time.perf_counter() - t0)
        vals.append(v)
    value = float(np.mean(vals))
    sample = "oracle FP64 BRAS-PCG (scipy CSR, 1 thread) on the same 48^3x6 mesh at p=1,2 (sample of p=1..4)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * float(np.mean(t_all)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "p=1,2 only", "detail": detail},
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- ncu DRAM traffic of a kernel, if the committed capture matches the current source ---------
KERNEL_SOURCES = ["paper_2607_12138_b300/csrc/apply_kernels.cuh", "paper_2607_12138_b300/csrc/tc_kernels.cuh",
                  "paper_2607_12138_b300/csrc/packet.h", "paper_2607_12138_b300/csrc/tables.cpp"]


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(key, alg_bytes):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from profiles/dram_traffic.json, or None
    when that capture was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        rec = json.load(open(path))[key]
    except Exception:
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    return rec["dram_bytes_per_launch"]


# ---- clocks ------------------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = os.path.join(tempfile.gettempdir(), f"bras_clocks_{os.getpid()}.csv")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in open(self.path):
            c = [x.strip() for x in row.split(",")]
            if len(c) < 9:
                continue
            try:
                mhz.append(float(c[1]))
                mx = max(mx, float(c[2]))
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(mhz)}


# ---- our arm --------------------------------------------------------------------------------------
def run_ours(a):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2607_12138_b300 import bras as B
    from paper_2607_12138_b300 import meshgen as mg

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    orders = [int(p) for p in a.orders.split(",")]
    mesh = mg.unit_cube_mesh(N_CELLS, jitter=JITTER, seed=0)
    probs = []
    for p in orders:
        n, l2g, s = mg.dof_map(mesh, SPACE, p)
        ctx = B.Context(mesh.coords, mesh.cells, SPACE, p, n, l2g, s, autotune=True)   # setup: untimed
        b = torch.as_tensor(mg.rhs(n, 1, seed=1), device="cuda")
        x = torch.empty_like(b)
        bh = b.cpu().pin_memory()
        xh = torch.empty_like(bh).pin_memory()
        probs.append({"p": p, "n": n, "ctx": ctx, "b": b, "x": x, "bh": bh, "xh": xh, "l2g": l2g})
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > L2
    st = torch.cuda.current_stream()

    order_ms = {}

    def step(mode=B.SOLVE_MIXED, pc=B.PC_BRAS, host=False):
        out = []
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(probs) + 1)]
        evs[0].record(st)
        for i, pr in enumerate(probs):
            b, x = (pr["bh"], pr["xh"]) if host else (pr["b"], pr["x"])
            _, its, rel, status = pr["ctx"].pcg_solve(b, pc=pc, mode=mode, inner_precision=B.FP32, rtol=1e-10, out=x)
            evs[i + 1].record(st)
            out.append((int(its[0]), float(rel[0]), status))
        torch.cuda.synchronize()
        order_ms[(mode, pc, host)] = [evs[i].elapsed_time(evs[i + 1]) for i in range(len(probs))]
        return out

    def timed(fn, steps, collective=True):
        # collective: every rank runs this loop (barriers around each step); rank 0's comparison
        # rows run after the other ranks have left and time locally
        ts = []
        res = None
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            if collective:
                barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            res = fn()
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        if collective:
            barrier()
        return ts, res

    for _ in range(a.warmup):
        step()
    total_n = sum(pr["n"] for pr in probs)
    clocks = Clocks(local)
    launches0, graphs0 = B.kernel_launches(), B.graph_launches()
    ts, res = timed(step, a.steps)
    launches = B.kernel_launches() - launches0
    graphs = B.graph_launches() - graphs0
    clk = clocks.stop()
    t_step = float(np.mean(ts))
    t_max = max_over_ranks(t_step, ws, "cuda")
    value = whole_job_rate(total_n, t_max, ws)
    for its, rel, status in res:
        if status != 0 or rel > 1e-10:
            raise RuntimeError(f"solve did not reach 1e-10: {res}")
    # independent check of the 1e-10 target: the true residual ||b - M x|| / ||b|| of every
    # answer of the last timed step from the FP64 mass apply (the FP64 block kernel, parity-
    # tested at full size; not the float-float apply the refinement loop itself uses), untimed
    true_relres = []
    for pr in probs:
        r = pr["b"] - pr["ctx"].mass_apply(pr["x"], B.FP64)
        true_relres.append(float(torch.linalg.norm(r) / torch.linalg.norm(pr["b"])))
    if max(true_relres) > 1e-10:
        raise RuntimeError(f"true FP64 residual above 1e-10: {true_relres}")

    # end to end through host buffers (H2D of b and D2H of x inside the call)
    for _ in range(1):
        step(host=True)
    ts_e2e = []
    for _ in range(a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(host=True)
        ts_e2e.append(time.perf_counter() - t0)
    t_e2e = max_over_ranks(float(np.mean(ts_e2e)), ws, "cuda")
    e2e = {"value": whole_job_rate(total_n, t_e2e, ws), "unit": "DOF/s",
           "h2d_bytes_per_step": 8 * total_n, "d2h_bytes_per_step": 8 * total_n}

    if ws > 1:
        barrier()
        torch.distributed.destroy_process_group()   # no collective follows: rank 0 reports alone
    if rank != 0:
        return 0

    # per-order detail, comparison rows and per-kernel live timings
    detail = []
    compare = {}
    last_ms = order_ms.get((B.SOLVE_MIXED, B.PC_BRAS, False), [None] * len(probs))
    for i, pr in enumerate(probs):
        its, rel, _ = res[i]
        detail.append({"p": pr["p"], "n": pr["n"], "mixed_bras_its": its, "relres": rel,
                       "true_relres_fp64": true_relres[i], "solve_ms": last_ms[i],
                       "block_elems": pr["ctx"].block_tuning[0]})
    if not a.no_compare:
        for name, mode, pc in (("fp64_bras", B.SOLVE_FP64, B.PC_BRAS), ("fp64_jacobi", B.SOLVE_FP64, B.PC_JACOBI),
                               ("mixed_jacobi", B.SOLVE_MIXED, B.PC_JACOBI)):
            step(mode, pc)
            tsc, rc = timed(lambda: step(mode, pc), 1, collective=False)
            compare[name] = {"dof_per_s": total_n / tsc[0], "ms": 1e3 * tsc[0], "its": [r[0] for r in rc],
                             "solve_ms": order_ms.get((mode, pc, False))}
        compare["mixed_bras"] = {"dof_per_s": value / ws, "ms": 1e3 * t_step, "its": [r[0] for r in res]}

    # multi-RHS rows: 32 right-hand sides per solve, one context per order (p = 2, 4)
    if not a.no_compare:
        for pr in probs:
            if pr["p"] not in (2, 4):
                continue
            R = 32
            n = pr["n"]
            ctxR = B.Context(mesh.coords, mesh.cells, SPACE, pr["p"], n, pr["l2g"], None, max_nrhs=R)
            bR = torch.as_tensor(mg.rhs(n, R, seed=1), device="cuda")
            xR = torch.empty_like(bR)
            ctxR.pcg_solve(bR, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, rtol=1e-10, out=xR)
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _, itsR, relR, stR = ctxR.pcg_solve(bR, pc=B.PC_BRAS, mode=B.SOLVE_MIXED, rtol=1e-10, out=xR)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            compare[f"mixed_bras_r32_p{pr['p']}"] = {"dof_per_s": n * R / (ms / 1e3), "ms": ms,
                                                   "its_max": int(max(itsR)), "relres_max": float(max(relR)),
                                                   "status": int(stR)}
            del ctxR, bR, xR

    # stationary iterations (Sec. 3), FP64: damped fixed point with omega = 2 / (1 + lambda_max)
    # and Chebyshev on [1, lambda_max] with BRAS; fixed point with omega = 1 / lambda_max with
    # Jacobi for p <= 2 (its count grows like kappa).  lambda_max from 100 power-iteration steps,
    # outside the timed region, as in the paper's tables.
    if not a.no_compare:
        stat = {}
        for pr in probs:
            ctx, n = pr["ctx"], pr["n"]
            v0 = torch.as_tensor(mg.rhs(n, 1, seed=4), device="cuda")
            lb = float(ctx.lambda_max(v0, B.PC_BRAS, iters=100)[0])
            runs = [("bras_fixed_point", lambda: ctx.fixed_point_solve(pr["b"], 2.0 / (1.0 + lb), B.PC_BRAS, out=pr["x"])),
                    ("bras_chebyshev", lambda: ctx.chebyshev_solve(pr["b"], 1.0, lb, B.PC_BRAS, out=pr["x"]))]
            row = {"lambda_max_bras": lb}
            if pr["p"] <= 2:
                ld = float(ctx.lambda_max(v0, B.PC_JACOBI, iters=100)[0])
                row["lambda_max_jacobi"] = ld
                runs.append(("jacobi_fixed_point",
                             lambda: ctx.fixed_point_solve(pr["b"], 1.0 / ld, B.PC_JACOBI, out=pr["x"])))
            for name, fn in runs:
                fn()
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                _, its_s, rel_s, st_s = fn()
                e1.record(st)
                torch.cuda.synchronize()
                row[name] = {"its": int(its_s[0]), "relres": float(rel_s[0]), "status": int(st_s),
                             "ms": e0.elapsed_time(e1)}
            stat[f"p{pr['p']}"] = row
        compare["fp64_stationary"] = stat

    # Bernstein basis (Table 1's second H1 family) on the same mesh: mixed BRAS-PCG against
    # mixed Jacobi-PCG, p = 2..4
    if not a.no_compare:
        bern = {}
        for pr in probs:
            if pr["p"] < 2:
                continue
            cb = B.Context(mesh.coords, mesh.cells, "h1b", pr["p"], pr["n"], pr["l2g"], None)
            row = {}
            for name, pc in (("mixed_bras", B.PC_BRAS), ("mixed_jacobi", B.PC_JACOBI)):
                cb.pcg_solve(pr["b"], pc=pc, mode=B.SOLVE_MIXED, rtol=1e-10, out=pr["x"])
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                _, its_b, rel_b, st_b = cb.pcg_solve(pr["b"], pc=pc, mode=B.SOLVE_MIXED, rtol=1e-10, out=pr["x"])
                e1.record(st)
                torch.cuda.synchronize()
                row[name] = {"its": int(its_b[0]), "relres": float(rel_b[0]), "status": int(st_b),
                             "ms": e0.elapsed_time(e1)}
            bern[f"p{pr['p']}"] = row
            del cb
        compare["bernstein"] = bern

    # Batched multi-mesh solve (the H(div) batch configuration): jittered boxes with target tet
    # counts log-uniform in [2e3, 2e5], one N(0,1) right-hand side each, all meshes in one
    # context and one solve (per-mesh scalars and stopping tests).  RT k = 1, 2, 3 on the whole
    # batch of 256 meshes; the contexts keep FP32 inverses only (the mixed solve's inner
    # precision; FP64 cell mass matrices for the refinement residual are always kept).
    if not a.no_compare and not a.no_batch:
        sizes = mg.batch_mesh_sizes(256, seed=0)
        batch = {}
        for k, count in ((1, 256), (2, 256), (3, 256)):
            t0 = time.perf_counter()
            meshes, rhs = [], []
            for i, (nx, nz) in enumerate(sizes[:count]):
                m = mg.unit_cube_mesh(nx, jitter=JITTER, seed=100 + i, nz=nz)
                nk, lk, sk = mg.dof_map(m, "hdiv", k)
                meshes.append((m.coords, m.cells, nk, lk, sk))
                rhs.append(mg.rhs(nk, 1, seed=1000 + i))
            cb = B.Context.batched(meshes, "hdiv", k, precisions=2)
            t_setup = time.perf_counter() - t0
            bt = torch.as_tensor(np.concatenate(rhs), device="cuda")
            xb = torch.empty_like(bt)
            row = {"meshes": count, "cells": int(cb.n_cell), "dofs": int(cb.n_dof), "setup_s": t_setup,
                   "block_elems": cb.block_tuning[0]}
            for name, pc in (("mixed_bras", B.PC_BRAS), ("mixed_jacobi", B.PC_JACOBI)):
                cb.pcg_solve(bt, pc=pc, mode=B.SOLVE_MIXED, rtol=1e-10, out=xb)
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                _, its_b, rel_b, st_b = cb.pcg_solve(bt, pc=pc, mode=B.SOLVE_MIXED, rtol=1e-10, out=xb)
                e1.record(st)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                row[name] = {"ms": ms, "dof_per_s": cb.n_dof / (ms / 1e3), "its_min": int(its_b.min()),
                             "its_max": int(its_b.max()), "relres_max": float(rel_b.max()), "status": int(st_b)}
            batch[f"rt{k}"] = row
            del cb, bt, xb
            torch.cuda.empty_cache()
        compare["batched_hdiv"] = batch

    # 64 right-hand sides, H(curl) Nedelec k = 1..3 on 40^3 x 6 tets: mixed BRAS-PCG (FP32 inner,
    # FP64 refinement) against plain FP64 BRAS-PCG and FP64 Jacobi-PCG, one solve each
    if not a.no_compare and not a.no_c3:
        c3rows = {}
        m40c = mg.unit_cube_mesh(40, jitter=JITTER, seed=0)
        R = 64
        for k in (1, 2, 3):
            nk, lk, sk = mg.dof_map(m40c, "hcurl", k)
            cc = B.Context(m40c.coords, m40c.cells, "hcurl", k, nk, lk, sk, max_nrhs=R, precisions=3)
            bR = torch.as_tensor(mg.rhs(nk, R, seed=1), device="cuda")
            xR = torch.empty_like(bR)
            row = {"dofs": nk, "nrhs": R}
            for name, mode, pc in (("mixed_bras", B.SOLVE_MIXED, B.PC_BRAS), ("fp64_bras", B.SOLVE_FP64, B.PC_BRAS),
                                   ("fp64_jacobi", B.SOLVE_FP64, B.PC_JACOBI)):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                _, itsR, relR, stR = cc.pcg_solve(bR, pc=pc, mode=mode, rtol=1e-10, out=xR)
                e1.record(st)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                r = bR - cc.mass_apply(xR, B.FP64)
                true_rel = float((torch.linalg.norm(r, dim=0) / torch.linalg.norm(bR, dim=0)).max())
                row[name] = {"ms": ms, "dof_per_s": nk * R / (ms / 1e3), "its_max": int(max(itsR)),
                             "relres_max": float(max(relR)), "true_relres_fp64_max": true_rel, "status": int(stR)}
            c3rows[f"n1curl_k{k}"] = row
            del cc, bR, xR
            torch.cuda.empty_cache()
        compare["hcurl_64rhs"] = c3rows

    # differentiable weighted mass solve (H1 p = 3 on 32^3 x 6 tets, rho = exp(z), z ~ N(0, 0.5^2)):
    # forward x = M(rho)^{-1} b and backward (second solve, fused element gradient) timed
    if not a.no_compare:
        from paper_2607_12138_b300.autograd import WeightedMassSolver
        m32 = mg.unit_cube_mesh(32, jitter=JITTER, seed=0)
        n5, l5, _ = mg.dof_map(m32, SPACE, 3)
        zt = torch.as_tensor(np.random.default_rng(2).normal(0, 0.5, m32.n_cell), device="cuda")
        b5 = torch.as_tensor(mg.rhs(n5, 1, seed=1), device="cuda")
        xs5 = torch.as_tensor(mg.rhs(n5, 1, seed=3), device="cuda")
        grad_rows = {"dofs": n5, "cells": int(m32.n_cell)}
        for name, mode, rtol in (("mixed_rtol1e-10", B.SOLVE_MIXED, 1e-10), ("fp64_rtol1e-12", B.SOLVE_FP64, 1e-12)):
            solver = WeightedMassSolver(m32.coords, m32.cells, 3, n5, l5, rtol=rtol, mode=mode, space=SPACE)
            fwd, bwd = [], []
            for rep in range(3):
                z = zt.clone().requires_grad_(True)
                bb = b5.clone().requires_grad_(True)
                torch.cuda.synchronize()
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(st)
                x5 = solver(z, bb)
                loss = 0.5 * torch.sum((x5 - xs5) ** 2)
                e1.record(st)
                loss.backward()
                e2.record(st)
                torch.cuda.synchronize()
                if rep:
                    fwd.append(e0.elapsed_time(e1))
                    bwd.append(e1.elapsed_time(e2))
            grad_rows[name] = {"forward_ms": float(np.mean(fwd)), "backward_ms": float(np.mean(bwd)),
                               "its_last_solve": solver.last[0]}
            del solver
        compare["weighted_solve_grad"] = grad_rows

    # kappa_hat = lambda_max / lambda_min of Mt^{-1} M by CG-Lanczos (FP64) on ~1e6-dof meshes:
    # uniform meshes beside the values the paper prints (Tables 1-3, diagonal / BRAS, ~5e3 dofs;
    # kappa_hat of a mass matrix barely depends on the mesh size), and the jittered bench mesh
    if not a.no_compare:
        kap = {}
        def lanczos_pair(ctx, n):
            b0 = torch.as_tensor(mg.rhs(n, 1, seed=1), device="cuda")
            out = {}
            for name, pc, steps in (("diag", B.PC_JACOBI, 400), ("bras", B.PC_BRAS, 150)):
                lo, hi, k = ctx.cg_lanczos(b0, pc, steps=steps)
                out[name] = {"kappa": hi / lo, "lambda_min": lo, "lambda_max": hi, "steps": k}
            return out
        cases = (("h1_3d_p1", "h1", 1, 96, (5.0, 1.8), "Table 1, 3D, p=1, Lagrange"),
                 ("h1_3d_p2", "h1", 2, 48, (17, 3.0), "Table 1, 3D, p=2, Lagrange"),
                 ("h1g_3d_p3", "h1g", 3, 32, (13, 2.9), "Table 1, 3D, p=3, Lagrange (GLL-based nodes)"),
                 ("h1g_3d_p4", "h1g", 4, 24, (22, 3.5), "Table 1, 3D, p=4, Lagrange (GLL-based nodes)"),
                 ("h1b_3d_p2", "h1b", 2, 48, (24, 4.9), "Table 1, 3D, p=2, Bernstein"),
                 ("h1b_3d_p3", "h1b", 3, 32, (98, 7.8), "Table 1, 3D, p=3, Bernstein"),
                 ("h1b_3d_p4", "h1b", 4, 24, (420, 11), "Table 1, 3D, p=4, Bernstein"),
                 ("hcurl_3d_k1", "hcurl", 1, 56, (6.0, 1.8), "Table 2, 3D, p=1, N1curl"),
                 ("hdiv_3d_k1", "hdiv", 1, 64, (4.0, 1.6), "Table 3, 3D, p=1, RT"),
                 ("n2curl_3d_k1", "n2curl", 1, 40, (36, 7.4), "Table 2, 3D, p=1, N2curl"),
                 ("n2curl_3d_k2", "n2curl", 2, 26, (170, 10), "Table 2, 3D, p=2, N2curl"),
                 ("bdm_3d_k1", "bdm", 1, 28, (39, 7.1), "Table 3, 3D, p=1, BDM"),
                 ("bdm_3d_k2", "bdm", 2, 21, (32, 5.4), "Table 3, 3D, p=2, BDM"))
        for key, space, order, cells, printed, where in cases:
            mu = mg.unit_cube_mesh(cells, jitter=0.0, seed=0)
            nk, lk, sk = mg.dof_map(mu, space, order)
            cu = B.Context(mu.coords, mu.cells, space, order, nk, lk, sk)
            row = lanczos_pair(cu, nk)
            row.update({"mesh": f"uniform {cells}^3x6", "dofs": nk, "paper": {"diag": printed[0], "bras": printed[1]},
                        "paper_where": where})
            kap[key] = row
            del cu
        for pr in probs:
            row = lanczos_pair(pr["ctx"], pr["n"])
            row.update({"mesh": "jittered 48^3x6 (bench workload)", "dofs": pr["n"]})
            kap[f"h1_bench_p{pr['p']}"] = row
        compare["kappa_cg_lanczos"] = kap

    # mixed Poisson Schur complement apply -S~ x = B M_bras^{-1} B^T x (RT_k or BDM_k / DG_{k-1},
    # FP32) on 40^3 x 6 tets, beside the BRAS apply it contains
    if not a.no_compare:
        sch = {}
        m40s = mg.unit_cube_mesh(40, jitter=JITTER, seed=0)
        for fam, k in (("hdiv", 1), ("hdiv", 2), ("hdiv", 3), ("bdm", 1), ("bdm", 2), ("bdm", 3)):
            nk, lk, sk = mg.dof_map(m40s, fam, k)
            cs = B.Context(m40s.coords, m40s.cells, fam, k, nk, lk, sk, precisions=2)
            nq = k * (k + 1) * (k + 2) // 6
            xq = torch.as_tensor(mg.rhs(m40s.n_cell * nq, 1, seed=1), device="cuda").float()
            yq = torch.empty_like(xq)
            xb = torch.as_tensor(mg.rhs(nk, 1, seed=1), device="cuda").float()
            yb = torch.empty_like(xb)
            row = {"cells": m40s.n_cell, "hdiv_dofs": nk, "dg_dofs": m40s.n_cell * nq}
            for name, fn in (("schur_apply_us", lambda: cs.schur_apply(xq, B.FP32, out=yq)),
                             ("bras_apply_us", lambda: cs.bras_apply(xb, B.FP32, out=yb))):
                for _ in range(3):
                    fn()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(st)
                for _ in range(10):
                    fn()
                e1.record(st)
                torch.cuda.synchronize()
                row[name] = e0.elapsed_time(e1) * 1e3 / 10
            sch[f"{'rt' if fam == 'hdiv' else 'bdm'}{k}"] = row
            del cs
        compare["schur_mixed_poisson"] = sch

    # live per-kernel timings on the launching stream: FP32 BRAS / mass apply and FP64 mass apply
    kern = {}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    for pr in probs:
        ctx = pr["ctx"]
        x32 = pr["b"].float()
        y32 = torch.empty_like(x32)
        for name, fn, prec, xx, yy in (("bras_f32", ctx.bras_apply, B.FP32, x32, y32),
                                       ("mass_f32", ctx.mass_apply, B.FP32, x32, y32),
                                       ("mass_f64", ctx.mass_apply, B.FP64, pr["b"], pr["x"])):
            for _ in range(3):
                fn(xx, prec, out=yy)
            reps = 20
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(reps):
                fn(xx, prec, out=yy)
            e1.record(st)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / reps
            by = ctx.algorithmic_bytes(prec, 1, name.startswith("bras"))
            kern[f"{name}_p{pr['p']}"] = {"us": us, "alg_bytes": by, "gbs": by / us / 1e3}
    # dominant FP32 kernel by time per solve: bras apply and mass apply run once per inner iteration
    top = max(probs, key=lambda pr: kern[f"bras_f32_p{pr['p']}"]["us"])
    kb = kern[f"bras_f32_p{top['p']}"]
    roofline = {"bound": "hbm", "achieved": kb["gbs"], "peak": hbm_peak, "unit": "GB/s",
                "frac": kb["gbs"] / hbm_peak, "traffic": _traffic("h1_p4_bras_f32", kb["alg_bytes"]),
                "kernel": f"bras_apply FP32 (tcgen05 block kernel + group combine), H1 p={top['p']}",
                "alg_bytes_per_launch": kb["alg_bytes"], "launch_us": kb["us"], "peak_source": "measured"}

    # streamed path: H(curl) Nedelec k=3 on 40^3 x 6 tets, per-cell inverses FP32 / bf16
    streamed = None
    if not a.no_compare:
        m40 = mg.unit_cube_mesh(40, jitter=JITTER, seed=0)
        n3, l3, s3 = mg.dof_map(m40, "hcurl", 3)
        c3 = B.Context(m40.coords, m40.cells, "hcurl", 3, n3, l3, s3)
        x3 = torch.as_tensor(mg.rhs(n3, 1, seed=1), device="cuda").float()
        y3 = torch.empty_like(x3)
        for name, fn, prec in (("bras_f32_hcurl3", c3.bras_apply, B.FP32), ("bras_bf16_hcurl3", c3.bras_apply, B.BF16),
                               ("mass_f32_hcurl3", c3.mass_apply, B.FP32)):
            for _ in range(3):
                fn(x3, prec, out=y3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(10):
                fn(x3, prec, out=y3)
            e1.record(st)
            torch.cuda.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / 10
            by = c3.algorithmic_bytes(prec, 1, name.startswith("bras"))
            kern[name] = {"us": us, "alg_bytes": by, "gbs": by / us / 1e3}
        ks = kern["bras_f32_hcurl3"]
        streamed = {"bound": "hbm", "achieved": ks["gbs"], "peak": hbm_peak, "unit": "GB/s",
                    "frac": ks["gbs"] / hbm_peak, "traffic": _traffic("hcurl3_bras_f32", ks["alg_bytes"]),
                    "kernel": "bras_apply FP32 streamed per-cell inverses, N1curl k=3, 40^3x6 tets",
                    "alg_bytes_per_launch": ks["alg_bytes"], "launch_us": ks["us"], "peak_source": "measured"}
        del c3

    cpu = None
    cpu_all = None
    if not a.no_cpu_baseline:
        rate, cdetail = oracle_solve_rate((1, 2), repeats=3)
        cpu = {"value": rate, "unit": "DOF/s", "cores": 1, "kind": "oracle",
               "sample": "FP64 oracle BRAS-PCG (scipy CSR, single thread) on the same mesh at p=1,2, mean of 3",
               "detail": cdetail}
        try:
            rate_all, procs, t_all = oracle_all_cores_rate(2)
            cpu_all = {"value": rate_all, "unit": "DOF/s", "cores": procs, "nproc": os.cpu_count(), "kind": "oracle",
                       "sample": f"{procs} concurrent single-threaded FP64 oracle BRAS-PCG solves of the p=2 problem "
                                 f"(one process per core, own RHS seeds), dofs of all / slowest solve ({t_all:.2f} s)"}
        except Exception as ex:   # a host without spawn support: report why, keep the line
            cpu_all = {"unavailable": str(ex)[:200]}

    line = {"metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * t_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner / f64 refinement", "data": "synthetic",
            "config": {"workload": WORKLOAD, "orders": orders, "cells": int(mesh.n_cell), "dofs_per_step": total_n,
                       "solver": "mixed: FP32 BRAS-PCG (FP64 dots) in FP64 refinement",
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{ws}",
                       "detail": detail},
            "roofline": roofline, "roofline_streamed": streamed, "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
            "true_relres_fp64": true_relres,
            "fp64_bras_pcg": compare.get("fp64_bras"), "fp64_jacobi_pcg": compare.get("fp64_jacobi"),
            "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / a.steps,
            "solve_graph_launches_per_step": graphs / a.steps, "solves_per_step": len(probs),
            "clocks": clk, "compare": compare, "kernels": kern}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
