#!/usr/bin/env python
"""Benchmark of the CLAIR AMG hot path on one GB300 (or N independent replicas).

One step = the whole hot path on the 1024x1024 2D upwind advection-diffusion workload
(velocity angle pi/6, eps = 1e-2, pattern degree m = 2, B = 1): CLAIR setup (strength,
splitting, weight, mode smoothing, patterns, batched local solves, constraint projection,
Galerkin products over all levels) and the V(1,1)-preconditioned FGMRES solve to a 1e-8
relative true residual.  Inputs are resident in HBM before the timed region; the L2 is
flushed (256 MiB write) before every timed step, outside the step's CUDA events.

value = R rows built per step / seconds per step (MIXED precision: FP32 local solves and
V-cycle, FP64 FGMRES); the FP64 path is timed beside it ("fp64").  `e2e` repeats the step
from pinned host buffers with the host->device copies of A, B, f and the device->host copy
of u inside the timed region.  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "R rows/s in setup; time-to-1e-8 rel residual, mixed vs FP64 path, 1 GB300"
UNIT = "R rows/s"
PEAK_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# DRAM bytes (read + write, ncu dram__bytes_read.sum + dram__bytes_write.sum) of one step's
# local-solve launches on the default workload, keyed by the SHA-256 of the source they were
# measured on: reported only while that source is unchanged, null otherwise.
MEASURED_TRAFFIC = {
    "local_solve": {
        # 80.8 MB read + ~0 written (the writes stay in L2) per setup on the 512^2 case by
        # every local-solve launch (lsolve_persist and lsolve_cta), scaled by the ratio of
        # algorithmic bytes (530.9 MB / 132.1 MB = 4.02) to 1024^2
        "bytes": 80.8e6 * (530854884.0 / 132096084.0),
        "source_sha256": "43e1cdca0215f17a021f9d87110d9d0100555a966049681d0b97a1d8ae609757",
        "capture": "ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum "
                   "--clock-control none -k regex:lsolve_ python bench.py --nside 512 --steps 1 "
                   "--warmup 1 --fp64-steps 0 --no-e2e --no-cpu-baseline --no-errors "
                   "(second setup's launches), scaled to 1024^2 by algorithmic bytes",
    },
}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 flop x max clock
FP64_PEAK_TFLOPS = 1.19                               # measured FMA loop (dependent chains)


def source_sha256(name):
    import hashlib
    path = os.path.join(ROOT, "paper_2307_00229_gb300", "csrc", name)
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()


def measured_traffic(phase, source):
    m = MEASURED_TRAFFIC.get(phase)
    if not m or m.get("source_sha256") != source_sha256(source):
        return None
    return m["bytes"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["clair", "reference"], default="clair")
    ap.add_argument("--nside", type=int, default=1024)
    ap.add_argument("--eps", type=float, default=1e-2)
    ap.add_argument("--degree", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed FP64 steps (0: skip that arm)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-errors", action="store_true",
                    help="skip the MIXED-vs-FP64 result comparison (profiling runs)")
    ap.add_argument("--cpu-nside", type=int, default=192)
    ap.add_argument("--workload", choices=["advdiff1024", "batch64", "adjoint512", "recirc3d"],
                    default="advdiff1024",
                    help="advdiff1024: the headline line (default).  The others time the "
                         "many-instance batch (64 instances, sides 64-512), the adjoint "
                         "gradient (512^2 variable eps, 8 RHS) and the 128^3 recirculating "
                         "aggregation setup, each on its own JSON line")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return dict(PEAK_FALLBACK), "fallback"


def workload(args):
    import workloads
    return workloads.config2(eps=args.eps, degree=args.degree, nside=args.nside)


# ----------------------------------------------------------------------------------------
# Clocks during the timed region
# ----------------------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------------------
# Algorithmic traffic of one V(1,1) cycle (MIXED: 4-byte values and vectors)
# ----------------------------------------------------------------------------------------
def vcycle_bytes(levels, s=4):
    """Bytes one V(1,1) cycle must move, level by level: each Jacobi sweep reads the rows
    of its subset (s+4 bytes per entry), the row pointers, cf, dinv, b and the incoming
    x and writes x; residual, restriction and interpolation are SpMVs; the coarsest
    level is a dense n^2 product."""
    total = 0.0
    for L in levels:
        n, nnz = L["n"], L["nnz"]
        if L["nc"] == 0:
            total += s * n * n + 2 * s * n
            continue
        nc, nnzR, nnzP, nnzF, nF = L["nc"], L["nnz_R"], L["nnz_P"], L["nnz_F"], L["n"] - L["nc"]
        nnzC = nnz - nnzF
        sweep = lambda nnzX, nX: (s + 4) * nnzX + 4 * (n + 1) + n + 2 * s * nX + 2 * s * n
        total += (2 * s + 1) * n + s * n                        # first C sweep from x = 0
        total += 2 * sweep(nnzF, nF)                           # two F sweeps
        total += (s + 4) * nnz + 4 * (n + 1) + 3 * s * n       # residual
        total += (s + 4) * nnzR + 4 * (nc + 1) + s * n + s * nc  # restriction
        total += (s + 4) * nnzP + 4 * (n + 1) + s * nc + 2 * s * n  # interpolation
        total += 2 * sweep(nnzF, nF) + sweep(nnzC, nc)         # F, F, C post sweeps
        total += 2 * s * n                                      # copy
    return total


def phase_bytes(levels, arnoldi_steps=15, sweeps=5):
    """Algorithmic bytes per setup phase, summed over the levels that have transfers (FP64
    data: 8-byte values, 4-byte indices).  Each is the data the phase must read and write
    at least once: transpose, row maxima, the coarsening- and interpolation-strength masks
    of A and A^T (one pass over each, two masks written), one pass of the independent-set
    selection (split); the two pattern CSRs (pattern); the Arnoldi steps, each an SpMV of D^-1 A plus the classical
    Gram-Schmidt passes over the basis, twice (weight); CFF sweeps on both mode vectors
    (smooth); R, A, P read once and A_c written once (galerkin)."""
    b = {"split": 0.0, "pattern": 0.0, "weight": 0.0, "smooth": 0.0, "galerkin": 0.0}
    for k, L in enumerate(levels):
        if not L.get("nc"):
            continue
        n, nnz = L["n"], L["nnz"]
        nnzR, nnzP = L["nnz_R"], L["nnz_P"]
        nnzAc = levels[k + 1]["nnz"] if k + 1 < len(levels) else 0
        csr = 12 * nnz + 4 * (n + 1)
        b["split"] += 2 * csr + 2 * (12 * nnz + 8 * n) + 2 * (csr + 16 * n + 2 * nnz) + 2 * (4 * nnz + nnz) + n
        b["pattern"] += 8 * nnz + 4 * (nnzR + nnzP) + 8 * (L["nc"] + n)
        for j in range(arnoldi_steps):
            b["weight"] += csr + 24 * n + 2 * (8 * n * (j + 1) + 8 * n) + 2 * (8 * n * (j + 1) + 16 * n) + 24 * n
        sweep = csr + n + 4 * 8 * n
        b["smooth"] += 2 * sweeps * 3 * sweep
        b["galerkin"] += 12 * (nnzR + nnz + nnzP + nnzAc) + 4 * (L["nc"] + 1)
    return b


def level_summary(cl, h):
    import torch
    st = cl.clair_stats(h)
    out = []
    for k in range(st.levels):
        v = cl.clair_level_view(h, k)
        d = {"n": v["n"], "nc": v["nc"], "nnz": int(v["A_col"].numel())}
        if v["nc"]:
            cf = v["cf"].to(torch.int32)
            rl = (v["A_rowptr"][1:] - v["A_rowptr"][:-1])
            d["nnz_F"] = int(rl[cf == 0].sum().item())
            d["nnz_R"] = int(v["R_col"].numel())
            d["nnz_P"] = int(v["P_col"].numel())
        out.append(d)
    return out


# ----------------------------------------------------------------------------------------
# Several GPUs: independent replicas (the path does not shard across GPUs on this system);
# every rank runs the same workload, the job's time is the slowest rank's.
# ----------------------------------------------------------------------------------------
def slowest_rank_ms(ms, dist=None, device=None):
    """Max over ranks of the per-step time (all-reduce MAX; the local value alone at N=1)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rows_per_s(rows_per_rank, world, ms):
    """Whole-job throughput: every rank builds `rows_per_rank` R rows in `ms` (weak scaling)."""
    return world * rows_per_rank / (ms / 1e3)


# ----------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------
def run_clair(args):
    import numpy as np
    import torch

    from paper_2307_00229_gb300 import clair as cl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cl.load()
    prob = workload(args)
    A = prob.A
    dev = torch.device("cuda", local)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    rowptr, col, val = t(A.rowptr, torch.int32), t(A.col, torch.int32), t(A.val, torch.float64)
    B, f = t(prob.B, torch.float64), t(prob.f, torch.float64)
    u = torch.zeros_like(f)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def params(precision):
        p = cl.clair_params_default()
        p.degree = args.degree
        p.precision = precision
        return p

    def step(p):
        h = cl.clair_setup(rowptr, col, val, B, p)
        u.zero_()
        st, its, rel = cl.clair_solve(h, f, u, raise_not_converged=False)
        return h, st, its, rel

    def timed(precision, steps, warmup, e2e=False):
        p = params(precision)
        host = None
        if e2e:
            host = {k: v.cpu().pin_memory() for k, v in
                    (("rowptr", rowptr), ("col", col), ("val", val), ("B", B), ("f", f))}
            u_host = torch.empty(u.shape, dtype=torch.float64).pin_memory()
        for _ in range(warmup):
            h, *_ = step(p)
            cl.clair_free(h)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        times, its_l, rel_l, stats = [], [], [], None
        launches0 = cl.clair_kernel_launches()
        wall0 = time.perf_counter()
        gc.collect()
        gc.disable()  # no collector pauses inside the timed steps (the host drives every step)
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if e2e:
                for name, dst in (("rowptr", rowptr), ("col", col), ("val", val), ("B", B), ("f", f)):
                    dst.copy_(host[name], non_blocking=True)
            h, st, its, rel = step(p)
            if e2e:
                u_host.copy_(u, non_blocking=True)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            its_l.append(its)
            rel_l.append(rel)
            stats = (cl.clair_stats(h), level_summary(cl, h))
            cl.clair_free(h)
        torch.cuda.synchronize()
        gc.enable()
        wall = time.perf_counter() - wall0
        launches = cl.clair_kernel_launches() - launches0
        if dist:
            dist.barrier()
        ms = slowest_rank_ms(statistics.mean(times), dist, dev)
        bytes_h2d = sum(x.numel() * x.element_size() for x in host.values()) if e2e else 0
        return {"ms": ms, "times": times, "its": its_l, "rel": rel_l, "stats": stats[0],
                "levels": stats[1], "wall": wall, "launches": launches // max(steps, 1),
                "h2d": bytes_h2d, "d2h": u.numel() * 8 if e2e else 0}

    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            gpu_index = int(vis.split(",")[local])
        except ValueError:
            pass
    sampler = ClockSampler(gpu_index)
    mixed = timed(cl.CLAIR_MIXED, args.steps, args.warmup)
    clocks = sampler.stop()
    fp64 = timed(cl.CLAIR_FP64, args.fp64_steps, 1) if args.fp64_steps > 0 else None
    e2e = None if args.no_e2e else timed(cl.CLAIR_MIXED, max(1, min(args.steps, 3)), 1, e2e=True)

    # error of every MIXED result against the FP64 path (which matches the FP64 oracle to
    # 1e-12 per row in the parity tests): level-0 R and P weights per row, the solution
    def results(precision):
        h, st_, its_, rel_ = step(params(precision))
        v = cl.clair_level_view(h, 0)
        out = {k_: v[k_].cpu().numpy() for k_ in ("R_val", "P_val", "R_rowptr", "P_rowptr")}
        out["u"] = u.cpu().numpy()
        cl.clair_free(h)
        return out

    def rowwise(a, ref, rp):
        worst = 0.0
        for lo, hi in zip(rp[:-1], rp[1:]):
            if hi > lo:
                m_ = np.abs(ref[lo:hi]).max()
                if m_ > 0:
                    worst = max(worst, float(np.abs(a[lo:hi] - ref[lo:hi]).max() / m_))
        return worst
    errors = None
    if not args.no_errors:
        rm, r64 = results(cl.CLAIR_MIXED), results(cl.CLAIR_FP64)
        errors = {"R_rowwise_max_rel": rowwise(rm["R_val"], r64["R_val"], r64["R_rowptr"]),
                  "P_rowwise_max_rel": rowwise(rm["P_val"], r64["P_val"], r64["P_rowptr"]),
                  "u_rel": float(np.linalg.norm(rm["u"] - r64["u"]) / np.linalg.norm(r64["u"])),
                  "against": "the FP64 GPU path of the same workload (level 0 weights, solution)"}

    st = mixed["stats"]
    rows = int(st.r_rows)
    value = job_rows_per_s(rows, world, mixed["ms"])
    pk, pk_kind = peaks()
    phases = {name: st.phase_ms[i] for i, name in enumerate(cl.PHASES[:8])}
    phases.update({name: st.solve_phase_ms[i] for i, name in enumerate(cl.PHASES) if i >= 8})
    its = mixed["its"][-1]
    # roofline of the dominant phase
    vb = vcycle_bytes(mixed["levels"])
    vcycle_ms = phases["vcycle"] / max(its, 1)
    lsolve = {"bound": "alu", "achieved": st.lsolve_flops / (phases["local_solve"] * 1e-3) / 1e12,
              "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
              "traffic": measured_traffic("local_solve", "local_solve.cu"),
              "traffic_scope": "per step, all local-solve launches (ncu DRAM read + write), "
                               "measured at 512^2 and scaled by algorithmic bytes",
              "algorithmic_bytes": st.lsolve_min_bytes,
              "kernel": "lsolve_persist / lsolve_cta / lsolve_blk (FP32 batched local LU)",
              "share_of_step": phases["local_solve"] / mixed["ms"]}
    lsolve["frac"] = lsolve["achieved"] / lsolve["peak"]
    hbm = pk.get("hbm_gbs", PEAK_FALLBACK["hbm_gbs"])
    # the other setup phases against HBM (algorithmic bytes per phase_bytes)
    pb = phase_bytes(mixed["levels"])
    roofline_phases = {}
    for name, nbytes in pb.items():
        ms_ = phases[name]
        if ms_ > 0:
            gbs = nbytes / (ms_ * 1e-3) / 1e9
            roofline_phases[name] = {"bound": "hbm", "ms": ms_, "algorithmic_bytes": nbytes,
                                     "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                     "frac": gbs / hbm, "share_of_step": ms_ / mixed["ms"],
                                     "stream": "side" if name in ("weight", "smooth") else "main"}
    vcyc = {"bound": "hbm", "achieved": vb / (vcycle_ms * 1e-3) / 1e9 if vcycle_ms > 0 else None,
            "peak": hbm, "unit": "GB/s", "traffic": None, "bytes_per_cycle": vb,
            "kernel": "V(1,1) cycle kernels (jacobi/spmv, FP32)",
            "share_of_step": phases["vcycle"] / mixed["ms"]}
    vcyc["frac"] = vcyc["achieved"] / vcyc["peak"] if vcyc["achieved"] else None
    dominant, other = (lsolve, vcyc) if lsolve["share_of_step"] >= vcyc["share_of_step"] else (vcyc, lsolve)
    dominant["peak_source"] = ("derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
                               if dominant["unit"] == "TFLOP/s" else f"{pk_kind} hbm_gbs")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mixed["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": prob.name, "n": A.n, "nnz": A.nnz, "eps": args.eps,
                   "velocity_angle": "pi/6", "degree": args.degree, "coarsen": "FC",
                   "precision": "mixed (FP32 local solves and V-cycle, FP64 FGMRES)",
                   "parallelism": f"replicas x{world}", "l2": "flushed (256 MiB write) before each step"},
        "time_to_1e8_ms": mixed["ms"], "iterations": its, "relres": mixed["rel"][-1],
        "setup_ms": st.setup_ms, "r_rows": rows, "levels": st.levels,
        "operator_complexity": st.operator_complexity,
        "setup_rows_per_s": rows / (st.setup_ms / 1e3),
        "phases_ms": phases,
        "levels_ms": [{"n": L["n"], "span": round(st.level_span_ms[k], 3),
                       **{name: round(st.level_phase_ms[k][i], 3) for i, name in enumerate(cl.PHASES[:8])}}
                      for k, L in enumerate(mixed["levels"])],
        "fp64": None if fp64 is None else {
            "ms_per_step": fp64["ms"], "iterations": fp64["its"][-1], "relres": fp64["rel"][-1],
            "setup_ms": fp64["stats"].setup_ms, "value": job_rows_per_s(rows, world, fp64["ms"]),
            "local_solve_ms": fp64["stats"].phase_ms[4]},
        "mixed_speedup_vs_fp64": None if fp64 is None else fp64["ms"] / mixed["ms"],
        "e2e": None if e2e is None else {
            "value": job_rows_per_s(rows, world, e2e["ms"]), "unit": UNIT,
            "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"],
            "ms_per_step": e2e["ms"]},
        "roofline": dominant, "roofline_other": other, "roofline_phases": roofline_phases,
        "error_vs_fp64": errors,
        "gpu_launches": mixed["launches"],
        "tuning": {"lsolve_kind_b1": st.lsolve_kind_b1, "lsolve_kind_b3": st.lsolve_kind_b3,
                   "lsolve_blocks_per_sm": st.lsolve_blocks_per_sm,
                   "lsolve_tuned": st.lsolve_tuned, "cycle_short_lanes": st.cycle_short_lanes},
        "clocks": clocks,
        "step_times_ms": mixed["times"], "wall_s": mixed["wall"],
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ----------------------------------------------------------------------------------------
def oracle_step(nside, eps, degree):
    import numpy as np

    import oracle as O
    import workloads
    prob = workloads.constdir_2d(nside, math.pi / 6, eps, seed=1, degree=degree)
    p = O.Params(degree=degree)
    t0 = time.perf_counter()
    c0 = time.process_time()
    H, x, its, hist = O.solve(prob.A, prob.f, prob.B, p)
    dt = time.perf_counter() - t0
    cpu = time.process_time() - c0
    rows = sum(int(l.cf.sum()) for l in H.levels if l.cf is not None)
    return rows, dt, cpu, its


def cpu_baseline(args):
    rows, dt, cpu, its = oracle_step(args.cpu_nside, args.eps, args.degree)
    return {"value": rows / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "threads_busy": round(cpu / dt, 2),
            "sample": f"oracle setup + FGMRES solve of the same problem family at {args.cpu_nside}^2 "
                      f"(eps={args.eps}, angle pi/6, m={args.degree}): {rows} R rows in {dt:.1f} s, "
                      f"{its} iterations; numpy/scipy on the host's {os.cpu_count()} cores "
                      f"(CPU time / wall time {cpu / dt:.2f})"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    nside = max(32, args.cpu_nside * 3 // 4)
    for _ in range(args.warmup):
        oracle_step(nside, args.eps, args.degree)
    times, rows, cpus = [], 0, []
    for _ in range(args.steps):
        rows, dt, cpu, its = oracle_step(nside, args.eps, args.degree)
        times.append(dt)
        cpus.append(cpu)
    ms = 1e3 * statistics.mean(times)
    value = rows / (ms / 1e3)
    cores = os.cpu_count()
    sample = (f"oracle setup + FGMRES solve per step on the same problem family at {nside}^2 "
              f"(eps={args.eps}, angle pi/6, m={args.degree}), {rows} R rows per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"constdir2d_{nside}_eps{args.eps:g}_m{args.degree}",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------------------
# Other workloads (one JSON line each; not the headline)
# ----------------------------------------------------------------------------------------
def _events_ms(fn, steps, warmup, flush):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    times, out = [], None
    gc.collect()
    gc.disable()
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    gc.enable()
    return statistics.mean(times), times, out


def _line(metric, value, unit, hib, ms, times, args, workload, extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": hib, "scaling": "weak",
         "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
         "config": dict(workload, l2="flushed (256 MiB write) before each step")}
    d.update(extra)
    d["step_times_ms"] = times
    print(json.dumps(d), flush=True)


def run_batch(args):
    import numpy as np
    import torch

    import workloads
    from paper_2307_00229_gb300 import clair as cl
    cl.load()
    probs = workloads.config4()
    A, offs = workloads.block_diagonal([pr.A for pr in probs])
    f = np.concatenate([pr.f for pr in probs])
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    rowptr, col, val = t(A.rowptr, torch.int32), t(A.col, torch.int32), t(A.val, torch.float64)
    B, fd = t(np.ones(A.n), torch.float64), t(f, torch.float64)
    u = torch.zeros_like(fd)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    res = {}
    for name, prec, steps in (("mixed", cl.CLAIR_MIXED, args.steps), ("fp64", cl.CLAIR_FP64, max(1, args.fp64_steps))):
        p = cl.clair_params_default()
        p.precision = prec

        def step():
            h = cl.clair_setup_batched(offs.tolist(), rowptr, col, val, B, p)
            u.zero_()
            st, its, rel = cl.clair_solve(h, fd, u, raise_not_converged=False)
            s_ = cl.clair_stats(h)
            cl.clair_free(h)
            return st, its, rel, s_
        l0 = cl.clair_kernel_launches()
        ms, times, (st, its, rel, sts) = _events_ms(step, steps, args.warmup, flush)
        res[name] = {"ms": ms, "times": times, "its": its, "rel": rel, "status": st,
                     "setup_ms": sts.setup_ms, "rows": int(sts.r_rows), "levels": sts.levels,
                     "cycle64_from": sts.cycle64_from, "fp64_cycle_from": int(sts.fp64_cycle_from),
                     "launches": (cl.clair_kernel_launches() - l0) // (steps + args.warmup),
                     "phases_ms": {n_: sts.phase_ms[i] for i, n_ in enumerate(cl.PHASES[:8])},
                     "solve_phases_ms": {n_: sts.solve_phase_ms[i] for i, n_ in enumerate(cl.PHASES) if i >= 8}}
    # the same instances one after another (setup + solve each), for comparison
    p = cl.clair_params_default()
    p.precision = cl.CLAIR_MIXED
    flush.fill_(1.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    seq_rows = 0
    for i, pr in enumerate(probs):
        lo, hi = int(offs[i]), int(offs[i + 1])
        h = cl.clair_setup(t(pr.A.rowptr, torch.int32), t(pr.A.col, torch.int32),
                           t(pr.A.val, torch.float64), B[lo:hi].contiguous(), p)
        ui = torch.zeros(hi - lo, dtype=torch.float64, device="cuda")
        cl.clair_solve(h, fd[lo:hi].contiguous(), ui, raise_not_converged=False)
        seq_rows += int(cl.clair_stats(h).r_rows)
        cl.clair_free(h)
    e1.record()
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    m = res["mixed"]
    _line("R rows/s in setup; time-to-1e-8 rel residual of all instances (one batched setup + solve)",
          m["rows"] / (m["ms"] / 1e3), "R rows/s", True, m["ms"], m["times"], args,
          {"workload": "batch64_advdiff2d", "instances": len(probs), "n_total": A.n, "nnz_total": A.nnz,
           "sides": [pr.meta["nside"] for pr in probs], "coarsen": "FC", "degree": 2,
           "precision": "mixed (FP32 local solves and V-cycle, FP64 FGMRES)"},
          {"iterations": m["its"], "worst_instance_relres": m["rel"], "status": m["status"],
           "cycle64_from": m["cycle64_from"], "fp64_cycle_from": m["fp64_cycle_from"],
           "setup_ms": m["setup_ms"], "r_rows": m["rows"], "levels": m["levels"],
           "phases_ms": m["phases_ms"], "solve_phases_ms": m["solve_phases_ms"],
           "gpu_launches": m["launches"],
           "fp64": {k: res["fp64"][k] for k in ("ms", "its", "rel", "setup_ms", "status")},
           "sequential_instances_ms": seq_ms, "sequential_r_rows": seq_rows})


def run_adjoint(args):
    import numpy as np
    import torch

    import workloads
    from paper_2307_00229_gb300 import clair as cl
    cl.load()
    prob = workloads.config5()
    A, m = prob.A, prob.meta
    nside = m["nside"]
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    rowptr, col, val0 = t(A.rowptr, torch.int32), t(A.col, torch.int32), t(A.val, torch.float64)
    F0, T = t(prob.f, torch.float64), t(m["u_target"], torch.float64)
    eps, vx, vy = t(m["eps_field"], torch.float64), t(m["vx"], torch.float64), t(m["vy"], torch.float64)
    B = t(np.ones(A.n), torch.float64)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    out = {}
    for name, prec in (("mixed", cl.CLAIR_MIXED), ("fp64", cl.CLAIR_FP64)):
        p = cl.clair_params_default()
        p.precision = prec

        def step():
            val = val0.clone().requires_grad_(True)
            U = cl.ClairSolve.apply(val, F0, rowptr, col, B, p)
            loss = ((U - T) ** 2).sum()
            loss.backward()
            return cl.clair_advdiff2d_param_grad(nside, 1.0 / (nside + 1), eps, vx, vy, rowptr, col, val.grad)
        ms, times, g = _events_ms(step, args.steps if name == "mixed" else max(1, args.fp64_steps),
                                  args.warmup, flush)
        out[name] = {"ms": ms, "times": times}
    _line("adjoint gradient time: forward setup + 8 solves, adjoint setup + 8 solves, "
          "sampled outer product, field chain rule", out["mixed"]["ms"], "ms", False,
          out["mixed"]["ms"], out["mixed"]["times"], args,
          {"workload": f"varcoef2d_{nside}_8rhs", "n": A.n, "nnz": A.nnz, "nrhs": 8,
           "precision": "mixed (FP32 local solves and V-cycle, FP64 FGMRES)"},
          {"fp64": out["fp64"]})


def run_recirc3d(args):
    import numpy as np
    import torch

    import workloads
    from paper_2307_00229_gb300 import clair as cl
    cl.load()
    prob = workloads.config3()
    A = prob.A
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    args_ = (t(A.rowptr, torch.int32), t(A.col, torch.int32), t(A.val, torch.float64),
             t(prob.B, torch.float64))
    f = t(prob.f, torch.float64)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    p = cl.clair_params_default()
    p.precision = cl.CLAIR_MIXED
    p.coarsen = cl.CLAIR_COARSEN_AGG

    def setup_only():
        h = cl.clair_setup(*args_, p)
        s_ = cl.clair_stats(h)
        cl.clair_free(h)
        return s_
    ms, times, sts = _events_ms(setup_only, args.steps, args.warmup, flush)
    h = cl.clair_setup(*args_, p)
    u = torch.zeros_like(f)
    st, its, rel = cl.clair_solve(h, f, u, raise_not_converged=False)
    cl.clair_free(h)
    # the documented fallback: C/F splitting (FC) on the same operator, one setup + solve
    pf = cl.clair_params_default()
    pf.precision = cl.CLAIR_MIXED
    pf.coarsen = cl.CLAIR_COARSEN_FC

    def fc_step():
        hf = cl.clair_setup(*args_, pf)
        uf = torch.zeros_like(f)
        out = cl.clair_solve(hf, f, uf, raise_not_converged=False)
        sf = cl.clair_stats(hf)
        cl.clair_free(hf)
        return out, sf
    fc_ms, _, ((fst, fits, frel), fsts) = _events_ms(fc_step, 1, 0, flush)
    _line("R rows/s in setup (aggregation coarsening)", int(sts.r_rows) / (ms / 1e3), "R rows/s", True,
          ms, times, args, {"workload": "recirc3d_128", "n": A.n, "nnz": A.nnz, "coarsen": "AGG",
                            "degree": 2, "eps": 1e-3, "precision": "mixed"},
          {"r_rows": int(sts.r_rows), "levels": sts.levels, "operator_complexity": sts.operator_complexity,
           "phases_ms": {n_: sts.phase_ms[i] for i, n_ in enumerate(cl.PHASES[:8])},
           "t_hist": list(sts.t_hist)[:7],
           "levels_ms": [{"n": int(sts.n[k]), "span": round(sts.level_span_ms[k], 2),
                          "local_solve": round(sts.level_phase_ms[k][4], 2)}
                         for k in range(sts.levels)],
           "solve": {"status": st, "iterations": its, "relres": rel,
                     "note": "the paper's aggregation variant did not converge at alpha <= 1e-3 either"},
           "fc_fallback": {"time_to_1e8_ms": fc_ms, "setup_ms": fsts.setup_ms, "status": fst,
                           "t_hist": list(fsts.t_hist)[:7],
                           "phases_ms": {n_: fsts.phase_ms[i] for i, n_ in enumerate(cl.PHASES[:8])},
                           "iterations": fits, "relres": frel, "levels": fsts.levels,
                           "operator_complexity": fsts.operator_complexity,
                           "r_rows": int(fsts.r_rows)}})


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload == "adjoint512":
        run_adjoint(args)
    elif args.workload == "recirc3d":
        run_recirc3d(args)
    else:
        run_clair(args)


if __name__ == "__main__":
    main()
