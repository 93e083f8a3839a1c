#!/usr/bin/env python3
"""Benchmark of the GB300 isogeometric EFIE library.

Workload: plane-wave scattering by the unit sphere as 6 exact rational NURBS patches,
div-conforming B-splines of degree p = 2 on 32 x 32 elements per patch (13 068 complex
DOFs), wavenumber kappa = 10, interpolation degree q = 8, eta = 1.6, GMRES(1500) to a
relative residual of 1e-6, one plane wave along +z polarised in x.

One step = one pass of the whole hot path: device setup from the device-resident geometry
(geometry at the interpolation nodes, Sauter-Schwab near field, trees), right-hand side,
device GMRES solve (FMM matrix-vector products) and the far field in 64 directions.
value = solves per second (steps per second, whole job).  The mixed-precision form (FP32
phase-split M2L, FP64 near field, geometry and GMRES) is the timed form; its
matrix-vector product is checked against the FP64 form in the same run.

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.

Other workloads (--workload):
  multi    64 plane waves on the torus (16 patches, p = 3, 64x64 elements per patch, 139 392
           DOFs, kappa = 20, q = 10): matvec/s of the batched product on the tensor cores
           (--check-fp64 adds the error of two right-hand sides against the FP64 form);
  serving  32 Poisson-arriving scattering requests through the serving loop: solves/s and
           p50/p99 latency;
  batch    256 independent solves of a seeded mix of spheres, cubes and tori through the
           serving loop: solves/s.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import geometry as G  # noqa: E402

WORKLOAD = {
    "workload": "sphere6_nurbs_p2_n32_kappa10_q8_eta1.6_gmres1e-6",
    "geometry": "unit sphere, 6 exact rational Bezier patches (bidegree 4)",
    "p": 2, "elements_per_patch": "32x32", "level_m": 5, "kappa": 10.0, "q": 8, "eta": 1.6,
    "gmres_tol": 1e-6, "gmres_restart": 1500, "incident": "dir +z, pol x", "far_field_directions": 64,
    "l2": "working set > L2 (near-field blocks 0.68 GB, Krylov basis up to 0.31 GB)",
}
MAXIT = 3000
METRIC = ("FMM-EFIE solves/s (plane-wave scattering solve incl. setup) at GMRES 1e-6, "
          "mixed-precision matvec <=1e-5 rel err vs FP64")
# GMRES iterations of this workload (deterministic: 604 with the mixed and with the FP64
# operator); the oracle's solve estimate uses the same count
WORKLOAD_ITERATIONS = 604
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")


def peaks():
    try:
        with open(MEASURED) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev=0):
        self.dev = dev
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def far_dirs(n=64):
    # Fibonacci directions on the sphere (deterministic)
    k = np.arange(n) + 0.5
    z = 1 - 2 * k / n
    ph = math.pi * (1 + 5 ** 0.5) * k
    r = np.sqrt(1 - z * z)
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)


def max_over_ranks(ms, device="cpu"):
    """Slowest rank's time: every replica runs the same workload, the job is done when the
    last one is (no data-path collective; this is the only exchange)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, ms):
    """Whole-job solves/s of `world` replicas that each finish one solve per `ms`."""
    return world * 1000.0 / ms


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------- CPU oracle
def oracle_sample(seconds_hint=15.0, its=None):
    """Oracle cost of one solve of the workload (serial, one core), from a bounded sample:
    * setup = problem creation + (near pairs) x (time of one near block, timed on the near
      pairs of 3 sampled elements);
    * product = direct moments (timed) + (far blocks) x (time of one far block), the latter
      timed on the far-field part of 48 sampled rows: a far pair whose target cluster is on
      level l is applied once for each of the 4^(m-l) elements under it, which gives the
      number of far blocks the sampled rows process on average;
    the near-field apply with the stored blocks (< 0.5 % of the product) is not counted.
    Returns (solves/s, details)."""
    import oracle as O

    geo = G.sphere()
    w = WORKLOAD
    t0 = time.perf_counter()
    r = O.Problem(geo, p=w["p"], m=w["level_m"], kappa=w["kappa"], q=w["q"], eta=w["eta"])
    t_create = time.perf_counter() - t0
    rng = np.random.default_rng(5)
    xs = rng.standard_normal(r.nsup) + 1j * rng.standard_normal(r.nsup)
    nE = r.nE
    e_all = rng.permutation(nE)
    t = time.perf_counter()
    r.fmm_rows_far(xs, e_all[:0])
    t_mom = time.perf_counter() - t
    nrow = 48
    t = time.perf_counter()
    r.fmm_rows_far(xs, e_all[:nrow])
    t_rows = max(time.perf_counter() - t - t_mom, 1e-9)
    far = np.asarray(r.far_pairs())
    m = w["level_m"]
    blocks_per_row = float(np.sum(4.0 ** (m - far[:, 0]))) / nE
    t_block = t_rows / (nrow * blocks_per_row)
    apply_ = t_mom + len(far) * t_block
    near = r.near_pairs()
    pick = set(e_all[:3].tolist())
    sel = [k for k, (a, _) in enumerate(near) if a in pick]
    t = time.perf_counter()
    for k in sel:
        r.pair_block(int(near[k][0]), int(near[k][1]))
    t_pair = (time.perf_counter() - t) / max(len(sel), 1)
    setup = t_create + len(near) * t_pair
    its = its or 1
    solve = setup + its * apply_
    return 1.0 / solve, {"oracle_setup_s_est": setup, "oracle_matvec_s_est": apply_, "iterations": its,
                         "far_block_us": t_block * 1e6, "near_block_ms": t_pair * 1e3,
                         "sample": f"oracle far field of {nrow} of {nE} element rows (far blocks per row from the "
                                   f"block tree), direct moments, and near blocks of {len(sel)} pairs; scaled to "
                                   f"{len(far)} far blocks and {len(near)} near pairs; solve = setup + {its} x "
                                   f"product; serial, one core"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    its = args.ref_iterations
    vals = []
    det = None
    for _ in range(args.warmup + args.steps):
        v, det = oracle_sample(its=its)
        vals.append(v)
    vals = vals[args.warmup:]
    val = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC,
            "value": val, "unit": "solves/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / val, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, precision=args.precision, parallelism="single"),
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": det["sample"]},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "details": det}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------- GPU
def run_gpu(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1807_03097_gb300 import Solver
    from workloads.geometry import flatten

    w = WORKLOAD
    geo = G.sphere()
    stream = torch.cuda.current_stream()
    kw = dict(p=w["p"], level_m=w["level_m"], kappa=w["kappa"], q=w["q"], eta=w["eta"], gmres_tol=w["gmres_tol"],
              gmres_restart=w["gmres_restart"], gmres_maxit=args.maxit, m2l_store=args.m2l_store)
    prec = 1 if args.precision == "mixed" else 0
    s = Solver(geo, stream=stream.cuda_stream, precision=prec, **kw)
    N = s.ndof
    dirs = far_dirs(64)
    d_inc, p_inc = np.array([[0, 0, 1.0]]), np.array([[1.0, 0, 0]])
    wdev = torch.zeros((1, N), dtype=torch.complex128, device="cuda")
    edev = torch.zeros((1, 64, 3), dtype=torch.complex128, device="cuda")

    def step():
        s.setup()
        _, info, st = s.solve_plane_waves(d_inc, p_inc, out=wdev)
        s.far_field(wdev[0], dirs, out=edev)
        return info, st

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = s.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    its = []
    conv = []
    for _ in range(args.steps):
        info, st = step()
        its.append(info.iterations)
        conv.append(bool(info.converged))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    launches = s.launch_count() - l0
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms, "cuda")
    value = replica_value(world, ms)
    if args.only_steps:
        if rank == 0:
            print(json.dumps({"metric": "steps only", "value": value, "unit": "solves/s", "ms_per_step": ms,
                              "gmres_iterations": int(np.median(its)), "gpu_launches": int(launches)}))
        s.close()
        return 0

    # matrix-vector products: mixed vs FP64 form, per-phase device times (CUDA events on
    # the library's stream), roofline of the dominant kernel
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.standard_normal(N) + 1j * rng.standard_normal(N)).cuda()
    y = torch.empty_like(x)
    ph = []
    for i in range(23):
        s.matvec(x, out=y)
        if i >= 3:
            ph.append(s.last_timings())
    mv = {k: statistics.median([p[k] for p in ph]) for k in ph[0]}
    y_mixed = y.clone()
    s64 = Solver(geo, stream=stream.cuda_stream, precision=0, **kw)
    y64 = torch.empty_like(x)
    ph64 = []
    for i in range(3):
        s64.matvec(x, out=y64)
        if i >= 1:
            ph64.append(s64.last_timings())
    mv64 = {k: statistics.median([p[k] for p in ph64]) for k in ph64[0]}
    err_vs_fp64 = float(torch.linalg.norm(y_mixed - y64) / torch.linalg.norm(y64))
    # far-field error of the mixed solution vs the FP64 operator applied in the same solve
    pk = peaks()
    n_eval = s.nfar * (w["q"] + 1) ** 4
    # 4 complex MACs on the folded fields (32) + kernel generation counted as 16: distance 9,
    # phase 2, 1/r 1, rotation 4, with sqrt / rcp / sin / cos weighted 1 each
    flops_per_eval = 48.0
    m2l_ms = mv["m2l"]
    achieved = n_eval * flops_per_eval / (m2l_ms * 1e-3) / 1e12
    fp32_peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    roof = {"kernel": "k_m2l_f32w", "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": None,
            "peak_note": "FP32 SIMT: 152 SMs x 128 lanes x 2 flop x max SM clock (derived, not measured)",
            "work": f"{n_eval:.3e} kernel entries x {flops_per_eval:.0f} flop per matvec", "m2l_ms": m2l_ms}
    near_bytes = s.nnear * s.nb * s.nb * (8 if prec else 16) + 2 * s.nsup * 16
    near_roof = {"kernel": "k_near_apply", "bound": "hbm", "achieved": near_bytes / (mv["near"] * 1e-3) / 1e9,
                 "peak": pk.get("hbm_gbs"), "unit": "GB/s", "near_ms": mv["near"], "bytes": near_bytes}
    near_roof["frac"] = near_roof["achieved"] / near_roof["peak"]

    # end to end through the C ABI with host buffers (copies inside the timed region)
    deg, ncp, knots, cp, wgt = flatten(geo)
    h2d = sum(a.nbytes for a in (deg, ncp, knots, cp, wgt, d_inc, p_inc, dirs))
    d2h = N * 16 + 64 * 3 * 16
    s_e2e = Solver(None, stream=stream.cuda_stream, precision=prec, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        s_e2e.set_geometry(geo)
        s_e2e.setup()
        wh, _, _ = s_e2e.solve_plane_waves(d_inc, p_inc)
        s_e2e.far_field(wh[0], dirs)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / max(1, args.e2e_steps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, det = oracle_sample(its=int(np.median(its)))
        cpu = {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": det["sample"],
               "oracle_matvec_s_est": det["oracle_matvec_s_est"], "oracle_setup_s_est": det["oracle_setup_s_est"]}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-m2l/f64" if prec else "f64", "data": "synthetic",
            "config": dict(WORKLOAD, precision=args.precision, parallelism="replicas" if world > 1 else "single"),
            "gmres_iterations": int(np.median(its)), "converged": all(conv),
            "matvec_per_s": 1000.0 / mv["total"], "matvec_ms_phases": mv,
            "matvec_per_s_fp64": 1000.0 / mv64["total"], "matvec_ms_phases_fp64": mv64,
            "matvec_rel_err_vs_fp64": err_vs_fp64,
            "roofline": roof, "roofline_near": near_roof,
            "cpu_baseline": cpu,
            "e2e": {"value": 1000.0 / e2e_ms, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(line))
    s.close()
    s64.close()
    s_e2e.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------- many right-hand sides
MULTI = {
    "workload": "torus16_nurbs_p3_n64_kappa20_q10_eta1.6_64rhs",
    "geometry": "torus R=2, r=0.5, 16 rational biquadratic patches",
    "p": 3, "elements_per_patch": "64x64", "level_m": 6, "kappa": 20.0, "q": 10, "eta": 1.6,
    "rhs": 64, "directions": "plane waves, directions normalised Gaussian, polarisation random unit vector "
                             "orthogonal to the direction, seed 1807",
    "precision": "mixed: M2L split-TF32 on the tensor cores with FP32 accumulation, near field FP32 blocks "
                 "from FP64 quadrature, geometry FP64",
    "l2": "working set > L2 (near-field blocks 19 GB FP32, 64 x 2.1e6 superspace vectors)",
}


def run_multi(args):
    """One step = one matrix-vector product of all 64 right-hand sides (a batched GMRES
    iteration's product); value = right-hand-side products per second."""
    import torch

    torch.cuda.set_device(0)
    from paper_1807_03097_gb300 import Solver

    w = MULTI
    geo = G.torus(R=2.0, r=0.5)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    s = Solver(geo, stream=stream.cuda_stream, p=w["p"], level_m=w["level_m"], kappa=w["kappa"], q=w["q"],
               eta=w["eta"], precision=1, m2l_batch=0)
    setup_s = time.time() - t0
    N, R = s.ndof, w["rhs"]
    d, pol = G.plane_waves(R, seed=1807)
    b = s.rhs(d, pol)                                    # [R][N] right-hand sides (host)
    x = torch.from_numpy(b).cuda()
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        s.matvec(x, out=y)
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    l0 = s.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ph = []
    for _ in range(args.steps):
        s.matvec(x, out=y)
        ph.append(s.last_timings())
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = s.launch_count() - l0
    ms = ev0.elapsed_time(ev1) / args.steps
    mv = {k: statistics.median([p_[k] for p_ in ph]) for k in ph[0]}
    # the batched tensor-core product against the single-vector FP32 product (CUDA cores)
    # for two right-hand sides
    y1 = torch.empty_like(x[0])
    diffs = []
    for i in (0, R - 1):
        s.matvec(x[i], out=y1)
        diffs.append(float(torch.linalg.norm(y[i] - y1) / torch.linalg.norm(y1)))
    single_ms = s.last_timings()["total"]
    fp64 = None
    if getattr(args, "check_fp64", False):
        # both mixed products against the FP64 form (coupling matrices evaluated) for the same
        # two right-hand sides; outside the timed region
        s64 = Solver(geo, stream=stream.cuda_stream, p=w["p"], level_m=w["level_m"], kappa=w["kappa"], q=w["q"],
                     eta=w["eta"], precision=0, m2l_store=1)
        y64 = torch.empty_like(x[0])
        fp64 = {"tensor_batched": [], "single_fp32": []}
        for i in (0, R - 1):
            s64.matvec(x[i], out=y64)
            s.matvec(x[i], out=y1)
            n64 = torch.linalg.norm(y64)
            fp64["tensor_batched"].append(float(torch.linalg.norm(y[i] - y64) / n64))
            fp64["single_fp32"].append(float(torch.linalg.norm(y1 - y64) / n64))
        fp64["fp64_matvec_ms"] = s64.last_timings()["total"]
        s64.close()
    # roofline of the tensor-core M2L (useful complex work; TF32 peak = measured BF16 peak x
    # the nominal TF32/BF16 ratio 1.1/2.25)
    pk = peaks()
    nI = (w["q"] + 1) ** 2
    useful = 8.0 * nI * nI * 4 * R * s.nfar
    np_ = 64 if nI <= 64 else (96 if nI <= 96 else 128)
    kp = 8 * sum(min(4, (nI - 32 * c + 7) // 8) for c in range((nI + 31) // 32))
    executed = 3 * 2.0 * 128 * (2 * np_) * kp * ((4 * R + 63) // 64) * s.nfar
    tf32_peak = pk.get("bf16_tflops", 1900.0) * 1.1 / 2.25
    m2l_s = mv["m2l"] * 1e-3
    roof = {"kernel": "k_m2l_tc", "bound": "tensor", "achieved": useful / m2l_s / 1e12, "peak": tf32_peak,
            "unit": "TFLOP/s", "frac": useful / m2l_s / 1e12 / tf32_peak, "traffic": None,
            "peak_note": "TF32 dense = measured BF16 burst peak x 1.1/2.25 (nominal ratio)",
            "work": f"useful 8 n_I^2 x 4R x far pairs = {useful:.3e} real flop per product "
                    f"(complex MACs of {4 * R} fields); executed on the tensor pipe (3 split-TF32 passes, "
                    f"padded to N={2 * np_}, K={kp}) = {executed:.3e}",
            "executed_tflops": executed / m2l_s / 1e12, "m2l_ms": mv["m2l"]}
    # end to end with host buffers
    yh = np.empty_like(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        s.matvec(b, out=yh)
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / max(1, args.e2e_steps)
    line = {"metric": "FMM-EFIE matvec/s (right-hand-side products per second, 64 right-hand sides per "
                      "batched product), mixed precision",
            "value": R * 1000.0 / ms, "unit": "matvec/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "tf32x3-m2l/f32/f64", "data": "synthetic", "config": MULTI, "ndof": int(N),
            "far_pairs": int(s.nfar), "near_pairs": int(s.nnear), "setup_s": setup_s,
            "matvec_ms_phases": mv, "single_rhs_matvec_ms": single_ms,
            "tensor_vs_single_rhs_rel_diff": diffs, "rel_err_vs_fp64": fp64, "roofline": roof, "cpu_baseline": None,
            "cpu_baseline_note": "the FP64 oracle is timed on the default workload only",
            "e2e": {"value": R * 1000.0 / e2e_ms, "unit": "matvec/s", "h2d_bytes_per_step": int(b.nbytes),
                    "d2h_bytes_per_step": int(yh.nbytes)},
            "gpu_launches": int(launches), "clocks": clocks}
    print(json.dumps(line))
    s.close()
    return 0


# ---------------------------------------------------------------------------- serving
SERVING = {
    "workload": "serving_poisson50_mixed_1e-5",
    "arrivals": "Poisson, mean 50 requests/s, seed 1809",
    "requests": 32,
    "geometries": "6-patch sphere (radius U[0.5,2]), 6-patch cube (side U[1,3]), 16-patch torus (R=2a, r=a/2)",
    "p": "U{1,2,3}", "kappa": "U[1,30], geometry scaled so that the electrical size kappa*a is U[1,6]",
    "directions": "U{1..16} seeded plane waves per request", "q": 6, "eta": 1.6, "gmres_tol": 1e-5,
    "precision": "mixed", "dofs": "1e3 .. 3e4 per request (refinement level drawn among those in range)",
}


def serving_requests(n, seed=1809):
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for i in range(n):
        t += rng.exponential(1.0 / 50.0)
        kind = rng.integers(0, 3)
        p = int(rng.integers(1, 4))
        kappa = float(rng.uniform(1.0, 30.0))
        ka = float(rng.uniform(1.0, 6.0))
        a = ka / kappa
        if kind == 0:
            geo, npch = G.sphere(radius=a), 6
        elif kind == 1:
            geo, npch = G.cube(side=2 * a), 6
        else:
            geo, npch = G.torus(R=2 * a, r=a / 2), 16
        # refinement giving 1e3 .. 3e4 DOFs
        cand = [m for m in range(1, 8) if 1000 <= 2 * npch * ((1 << m) + p - 1) ** 2 <= 30000]
        m = int(cand[int(rng.integers(0, len(cand)))])
        nd = int(rng.integers(1, 17))
        d, pol = G.plane_waves(nd, seed=seed * 1000 + i)
        reqs.append(dict(t=t, geo=geo, dirs=d, pols=pol,
                         opt=dict(p=p, level_m=m, kappa=kappa, q=6, eta=1.6, precision=1, gmres_tol=1e-5,
                                  gmres_maxit=2000)))
    return reqs


BATCH = {
    "workload": "batch256_mixed_1e-5",
    "solves": 256, "seed": 1808,
    "geometries": "6-patch sphere (radius U[0.5,2]), 6-patch bilinear cube (side 2), 16-patch torus (R=2, r=0.5)",
    "elements_per_patch": "4x4, 8x8, 16x16 or 32x32", "p": "U{1,2}", "kappa": "U[1,15]", "q": 6, "eta": 1.6,
    "incident": "one seeded plane wave per solve", "gmres_tol": 1e-5, "gmres_maxit": 1500, "precision": "mixed",
    "execution": "all 256 submitted at once to the serving loop (independent contexts, 16 slots); the "
                 "persistent fused launch across solves is not built",
}


def batch_requests(n, seed=1808):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        kind = int(rng.integers(0, 3))
        if kind == 0:
            geo = G.sphere(radius=float(rng.uniform(0.5, 2.0)))
        elif kind == 1:
            geo = G.cube()
        else:
            geo = G.torus()
        m = int(rng.integers(2, 6))
        p = int(rng.integers(1, 3))
        kappa = float(rng.uniform(1.0, 15.0))
        d, pol = G.plane_waves(1, seed=seed * 1000 + i)
        reqs.append(dict(t=0.0, geo=geo, dirs=d, pols=pol,
                         opt=dict(p=p, level_m=m, kappa=kappa, q=6, eta=1.6, precision=1, gmres_tol=1e-5,
                                  gmres_maxit=1500)))
    return reqs


def run_batch(args):
    import torch
    from paper_1807_03097_gb300.efie import Server

    torch.cuda.set_device(0)
    reqs = batch_requests(BATCH["solves"], BATCH["seed"])
    clk = ClockSampler(0)
    clk.start()
    srv = Server(hbm_budget_bytes=int(args.budget_gib) << 30, max_slots=16)
    t0 = time.perf_counter()
    tickets = [srv.submit(r["geo"], r["dirs"], r["pols"], None, **r["opt"]) for r in reqs]
    res = [srv.wait(t) for t in tickets]
    makespan = time.perf_counter() - t0
    srv.close()
    clocks = clk.stop()
    lat = np.array([x[0].latency_ms for x in res])
    its = [int(x[0].iterations) for x in res]
    ok = sum(1 for x in res if x[0].status == 0)
    line = {"metric": "batch of independent solves: solves/s (mixed precision, GMRES 1e-5)",
            "value": len(reqs) / makespan, "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "solves": len(reqs), "converged": ok, "makespan_s": makespan,
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "gmres_iterations_median": int(np.median(its)), "gmres_iterations_max": int(max(its)),
            "total_dofs": int(sum(int(x[0].ndof) for x in res)), "data": "synthetic", "config": BATCH,
            "clocks": clocks}
    print(json.dumps(line))
    return 0


def run_serving(args):
    import torch
    from paper_1807_03097_gb300.efie import Server

    torch.cuda.set_device(0)
    reqs = serving_requests(SERVING["requests"])
    srv = Server(hbm_budget_bytes=int(args.budget_gib) << 30, max_slots=args.slots)
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        now = time.perf_counter() - t0
        if r["t"] > now:
            time.sleep(r["t"] - now)
        tickets.append(srv.submit(r["geo"], r["dirs"], r["pols"], None, **r["opt"]))
    res = [srv.wait(t) for t in tickets]
    makespan = time.perf_counter() - t0
    srv.close()
    lat = np.array([x[0].latency_ms for x in res])
    nsolve = sum(len(r["dirs"]) for r in reqs)
    ok = sum(1 for x in res if x[0].status == 0)
    line = {"metric": "serving: solves/s and p50/p99 request latency (mixed precision, GMRES 1e-5)",
            "value": nsolve / makespan, "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "requests": len(reqs), "requests_converged": ok, "plane_wave_solves": nsolve,
            "makespan_s": makespan, "latency_ms_p50": float(np.percentile(lat, 50)),
            "latency_ms_p99": float(np.percentile(lat, 99)), "slots": args.slots, "budget_gib": args.budget_gib,
            "dofs": [int(x[0].ndof) for x in res], "data": "synthetic", "config": SERVING}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--maxit", type=int, default=MAXIT)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--ref-iterations", type=int, default=WORKLOAD_ITERATIONS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-steps", action="store_true", help="time the steps only (for launch-list profiling)")
    ap.add_argument("--workload", default="solve", choices=["solve", "serving", "multi", "batch"])
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--budget-gib", type=int, default=192, help="serving: device-memory budget of the admission")
    ap.add_argument("--check-fp64", action="store_true",
                    help="multi workload: also compare two right-hand sides with the FP64 form (slow)")
    ap.add_argument("--m2l-store", type=int, default=0, choices=[0, 1, 2],
                    help="M2L coupling matrices: 0 auto (kept in HBM when they fit), 1 evaluated, 2 kept")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "multi":
        return run_multi(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
