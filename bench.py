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
phase-split M2L, near field integrated in FP64 and applied from FP32 blocks, geometry and
GMRES in FP64) is the timed form.  After the timed steps, the same line carries: the
matrix-vector products of the mixed and FP64 forms and their difference; one plain FP64 solve
(solves/s) with the mixed form's far-field and current errors against it; the rooflines of the
M2L (FP32 ALU), the near-field apply (HBM) and the near-field quadrature (FP64 ALU) against
compute peaks measured on the GPU by microbench/ and the HBM copy bandwidth of
MEASURED_PEAKS.json; the end-to-end rate with host buffers; the 64-right-hand-side torus
leg (matvec/s, tensor roofline) and the serving leg (p50/p99 latency) unless --no-extras; and
the oracle's CPU baseline (an estimate from a bounded sample, one core and all cores, plus a
timed oracle solve of the 192-DOF sphere).

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.

Other workloads (--workload):
  multi    64 plane waves on the torus (16 patches, p = 3, 64x64 elements per patch, 139 392
           DOFs, kappa = 20, q = 10): matvec/s of the batched product on the tensor cores
           (--check-fp64 adds the error of two right-hand sides against the FP64 form);
  serving  32 Poisson-arriving scattering requests through the serving loop: solves/s and
           p50/p99 latency;
  batch    256 independent solves of a seeded mix of spheres, cubes and tori through the
           serving loop: solves/s;
  tesla    the paper's Tesla settings (p = 4, eta = 0.1, q = 14) on a synthetic 232-patch
           surface of revolution: setup, matvec/s, mixed-vs-FP64 error, one solve.
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
def host_cpu():
    """(model name, logical cores) of the host, from lscpu when available."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return model, os.cpu_count() or 1


def _far_rows_worker(args):
    """Process-pool worker (spawned): time the oracle's far-field part of a share of element
    rows of the workload."""
    rows, seed = args
    import oracle as O

    w = WORKLOAD
    r = O.Problem(G.sphere(), p=w["p"], m=w["level_m"], kappa=w["kappa"], q=w["q"], eta=w["eta"])
    rng = np.random.default_rng(seed)
    xs = rng.standard_normal(r.nsup) + 1j * rng.standard_normal(r.nsup)
    t = time.perf_counter()
    r.fmm_rows_far(xs, np.asarray(rows[:0], np.int32))  # direct moments alone
    t_mom = time.perf_counter() - t
    t = time.perf_counter()
    r.fmm_rows_far(xs, np.asarray(rows, np.int32))
    return max(time.perf_counter() - t - t_mom, 1e-9)


def oracle_sample(its=None, all_cores=True):
    """Estimate of the oracle's cost of one solve of the workload, from a bounded sample:
    * setup = problem creation + (near pairs) x (time of one near block, timed on the near
      pairs of 3 sampled elements);
    * product = direct moments (timed) + (far blocks) x (time of one far block), the latter
      timed on the far-field part of 48 sampled rows: a far pair whose target cluster is on
      level l is applied once for each of the 4^(m-l) elements under it, which gives the
      number of far blocks the sampled rows process on average;
    the near-field apply with the stored blocks (< 0.5 % of the product) is not counted.
    Serial (one core) and, with all_cores, the far-field rows split over one spawned process
    per core (the oracle's near-block loop uses OpenMP over pairs).
    Returns (solves/s on one core, details)."""
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
    model, ncores = host_cpu()
    det = {"kind": "estimate", "oracle_setup_s_est": setup, "oracle_matvec_s_est": apply_, "iterations": its,
           "far_block_us": t_block * 1e6, "near_block_ms": t_pair * 1e3, "cpu_model": model, "cpu_cores": ncores,
           "sample": f"estimate, not a timed solve: oracle far field of {nrow} of {nE} element rows (far blocks per "
                     f"row from the block tree), direct moments, and near blocks of {len(sel)} pairs; scaled to "
                     f"{len(far)} far blocks and {len(near)} near pairs; solve = setup + {its} x product; serial, "
                     f"one core"}
    if all_cores and ncores > 1:
        import multiprocessing as mp

        rows_per = 24
        shares = [(e_all[nrow + i * rows_per: nrow + (i + 1) * rows_per].tolist(), 100 + i) for i in range(ncores)]
        ctx = mp.get_context("spawn")
        t = time.perf_counter()
        with ctx.Pool(ncores) as pool:
            times = pool.map(_far_rows_worker, shares)
        wall = max(times)
        t_block_all = wall / (rows_per * ncores * blocks_per_row)
        apply_all = t_mom + len(far) * t_block_all
        setup_all = t_create + len(near) * t_pair / ncores
        det.update({"all_cores": ncores, "far_block_us_all_cores": t_block_all * 1e6,
                    "oracle_matvec_s_est_all_cores": apply_all,
                    "solves_per_s_all_cores": 1.0 / (setup_all + its * apply_all),
                    "all_cores_sample": f"far field of {rows_per} rows per process on {ncores} spawned processes "
                                        f"(slowest process's time), near blocks scaled by 1/{ncores}, direct "
                                        f"moments serial; pool wall {time.perf_counter() - t:.1f} s"})
    return 1.0 / solve, det


def oracle_timed_small_solve():
    """A really timed oracle solve on the host: the 192-DOF sphere (6 patches, p = 1, 4 x 4
    elements per patch, kappa = 1, q = 4, eta = 1.6), one plane wave along +z polarised in x,
    FMM operator, GMRES to 1e-8 (serial except the near-block loop)."""
    import oracle as O

    t0 = time.perf_counter()
    r = O.Problem(G.sphere(), p=1, m=2, kappa=1.0, q=4, eta=1.6)
    b = r.rhs(np.array([0, 0, 1.0]), np.array([1.0, 0, 0]))
    x, its = r.gmres(b, use_fmm=True, tol=1e-8)[:2]
    dt = time.perf_counter() - t0
    return {"workload": "sphere6_p1_n4_kappa1_q4 (192 DOFs), GMRES 1e-8", "seconds": dt, "solves_per_s": 1.0 / dt,
            "gmres_iterations": int(its)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    its = args.ref_iterations
    vals = []
    det = None
    for _ in range(args.warmup + args.steps):
        v, det = oracle_sample(its=its, all_cores=False)
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
            "note": "each step is a bounded oracle sample (about 20 s) from which the cost of one solve is "
                    "estimated; ms_per_step is that estimated solve time, not the sample's wall time",
            "details": det}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------- measured peaks
def measured_peaks():
    """Compute peaks measured on this GPU by microbench/ (FFMA, FFMA2, DFMA, MUFU, tcgen05), or
    None with the reason."""
    try:
        import microbench

        return microbench.measure(), None
    except Exception as e:  # noqa: BLE001
        return None, f"peak microbenchmark unavailable: {e}"


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
    pk_alu, pk_err = measured_peaks() if not args.only_steps else (None, "skipped")
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
    its, conv, setups = [], [], []
    for _ in range(args.steps):
        info, st = step()
        its.append(info.iterations)
        conv.append(bool(info.converged))
        setups.append(s.setup_timings())
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
    e_mixed = edev[0].cpu().numpy().copy()
    w_mixed = wdev[0].cpu().numpy().copy()

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

    fp64 = None
    if not args.no_fp64_solve:
        # the plain FP64 form: one whole step (setup, solve, far field) timed on the host clock
        # around synchronous calls, and the per-result errors of the mixed form against it
        w64 = torch.zeros((1, N), dtype=torch.complex128, device="cuda")
        e64 = torch.zeros((1, 64, 3), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64.setup()
        _, info64, _ = s64.solve_plane_waves(d_inc, p_inc, out=w64)
        s64.far_field(w64[0], dirs, out=e64)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        E64, W64 = e64[0].cpu().numpy(), w64[0].cpu().numpy()
        fp64 = {"solves_per_s": 1.0 / t64, "ms_per_solve": t64 * 1e3, "gmres_iterations": int(info64.iterations),
                "converged": bool(info64.converged), "m2l": "stored FP64 coupling matrices",
                "far_field_rel_err_mixed_vs_fp64": float(np.abs(e_mixed - E64).max() / np.abs(E64).max()),
                "current_rel_err_mixed_vs_fp64": float(np.linalg.norm(w_mixed - W64) / np.linalg.norm(W64)),
                "note": "far-field error = max over 64 directions and 3 components of |E_mixed - E_fp64|, "
                        "relative to max |E_fp64|; both solves to GMRES 1e-6"}
    pk = peaks()
    n_eval = s.nfar * (w["q"] + 1) ** 4
    # 4 complex MACs on the folded fields (32) + kernel generation counted as 16: distance 9,
    # phase 2, 1/r 1, rotation 4, with sqrt / rcp / sin / cos weighted 1 each
    flops_per_eval = 48.0
    m2l_ms = mv["m2l"]
    achieved = n_eval * flops_per_eval / (m2l_ms * 1e-3) / 1e12
    if pk_alu:
        fp32_peak = max(pk_alu["ffma_flops"], pk_alu["ffma2_flops"]) / 1e12
        peak_note = ("FP32: measured on this GPU (microbench/peaks.cu), max of scalar FFMA "
                     f"{pk_alu['ffma_flops'] / 1e12:.1f} and packed FFMA2 {pk_alu['ffma2_flops'] / 1e12:.1f} TFLOP/s")
    else:
        fp32_peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        peak_note = f"FP32 derived (152 SMs x 128 lanes x 2 flop x max clock), not measured: {pk_err}"
    roof = {"kernel": "k_m2l_f32w", "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": None, "peak_note": peak_note,
            "work": f"{n_eval:.3e} kernel entries x {flops_per_eval:.0f} flop per matvec", "m2l_ms": m2l_ms}
    if pk_alu:
        # time each pipe needs for the entries at its measured rate (per entry: 8 packed FMAs on
        # the FMA pipe and 3 MUFU operations in the direct-phase form)
        mufu_rate = min(pk_alu["rsqrt_per_s"], pk_alu["sin_per_s"], pk_alu["cos_per_s"])
        roof["pipe_bound_ms"] = {"fma_32flop_per_entry": n_eval * 32 / pk_alu["ffma2_flops"] * 1e3,
                                 "mufu_3_per_entry": n_eval * 3 / mufu_rate * 1e3}
    # near-field apply timed alone (efie_near_apply, CUDA events on the library's stream) and, for
    # reference, inside the product where it shares the GPU with the far-field chain
    xs_t = torch.from_numpy(rng.standard_normal(s.nsup) + 1j * rng.standard_normal(s.nsup)).cuda()
    ys_t = torch.empty_like(xs_t)
    nt = []
    for i in range(13):
        s.near_apply(xs_t, out=ys_t)
        if i >= 3:
            nt.append(s.last_timings()["near"])
    near_alone = statistics.median(nt)
    near_bytes = s.nnear * s.nb * s.nb * (8 if prec else 16) + s.nsup * (8 + 16 + 16 if prec else 32)
    near_roof = {"kernel": "k_near_apply_w" if prec else "k_near_apply", "bound": "hbm",
                 "achieved": near_bytes / (near_alone * 1e-3) / 1e9, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                 "near_ms": near_alone, "near_ms_in_product": mv["near"], "bytes": near_bytes,
                 "work": "blocks (8 B per entry in FP32) + x* read (FP64) and converted (FP32 write + read) + y* write",
                 "peak_note": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
    near_roof["frac"] = near_roof["achieved"] / near_roof["peak"]
    st_ = {k: statistics.median([x_[k] for x_ in setups]) for k in setups[0]}
    # k_near_quad: per quadrature point and block entry, the integrand of eq. Vkh is a real
    # combination of two products (geometry term and div-div term: 2 FMA) scaled by the complex
    # kernel value (2 FMA): 8 FP64 flop per entry and point
    quad_flop = st_["near_quad_points"] * s.nb * s.nb * 8.0
    roof_setup = {"kernel": "k_near_quad", "bound": "alu (FP64)", "unit": "TFLOP/s",
                  "achieved": quad_flop / (st_["near_quad_ms"] * 1e-3) / 1e12, "near_quad_ms": st_["near_quad_ms"],
                  "setup_ms": st_["setup_ms"], "work": f"{st_['near_quad_points']:.3e} quadrature points x "
                                                        f"{s.nb}^2 entries x 8 flop",
                  "pairs_integrated": int(st_["near_quad_pairs"]),
                  "separated_pairs_ms": st_.get("near_sep_ms"), "separated_pairs": int(st_.get("near_sep_pairs", 0)),
                  "note": "touching pairs (Sauter-Schwab); the separated near pairs run in a second kernel "
                          "(element tables), timed separately"}
    if pk_alu:
        roof_setup["peak"] = pk_alu["dfma_flops"] / 1e12
        roof_setup["frac"] = roof_setup["achieved"] / roof_setup["peak"]
        roof_setup["peak_note"] = "FP64 DFMA measured on this GPU (microbench/peaks.cu)"

    # end to end through the C ABI with host buffers (copies inside the timed region)
    deg, ncp, knots, cp, wgt = flatten(geo)
    h2d = sum(a.nbytes for a in (deg, ncp, knots, cp, wgt, d_inc, p_inc, dirs))
    d2h = N * 16 + 64 * 3 * 16
    s_e2e = Solver(None, stream=stream.cuda_stream, precision=prec, **kw)
    e2e_ms = []
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s_e2e.set_geometry(geo)
        s_e2e.setup()
        wh, _, _ = s_e2e.solve_plane_waves(d_inc, p_inc)
        s_e2e.far_field(wh[0], dirs)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
    s.close()
    s64.close()
    s_e2e.close()

    variant = pairs = None
    if not args.no_variant:
        variant = variant_leg(args, stream, geo, kw, prec, d_inc, p_inc, dirs, e_mixed)
        pairs = m2l_pairs_leg(stream, geo, kw, prec, mv["m2l"])
    extra = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extra["multi"] = multi_leg(args, steps=args.multi_steps, pk_alu=pk_alu)
        extra["tesla_settings"] = tesla_leg(args)
        extra["serving"] = serving_leg(args)
        if not args.no_batch:
            # the first 16 of the 256 seeded solves (the whole mix: --workload batch)
            extra["batch"] = batch_leg(args, n=args.batch_n or 16)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, det = oracle_sample(its=int(np.median(its)))
        cpu = {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": det["sample"]}
        cpu.update({k: det[k] for k in det if k not in ("sample",)})
        try:
            cpu["timed_solve_small"] = oracle_timed_small_solve()
        except Exception as e:  # noqa: BLE001
            cpu["timed_solve_small"] = f"failed: {e}"

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-m2l/f64" if prec else "f64", "data": "synthetic",
            "config": dict(WORKLOAD, precision=args.precision, parallelism="replicas" if world > 1 else "single"),
            "gmres_iterations": int(np.median(its)), "converged": all(conv),
            "setup_ms": st_["setup_ms"],
            "matvec_per_s": 1000.0 / mv["total"], "matvec_ms_phases": mv,
            "matvec_ms_p10_p50_p90": [float(np.percentile([p["total"] for p in ph], q)) for q in (10, 50, 90)],
            "matvec_count": len(ph),
            "matvec_per_s_fp64": 1000.0 / mv64["total"], "matvec_ms_phases_fp64": mv64,
            "matvec_rel_err_vs_fp64": err_vs_fp64,
            "fp64_solve": fp64,
            "variant_dense_leaf": variant,
            "variant_m2l_unordered_pairs": pairs,
            "roofline": roof, "roofline_near": near_roof, "roofline_setup": roof_setup,
            "peaks_measured": pk_alu, "peaks_hbm_bf16": {k: pk.get(k) for k in ("hbm_gbs", "bf16_tflops",
                                                                               "bf16_tflops_sustained")},
            "cpu_baseline": cpu,
            "e2e": {"value": 1000.0 / statistics.median(e2e_ms), "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "steps": len(e2e_ms), "ms_min": min(e2e_ms),
                    "ms_median": statistics.median(e2e_ms), "ms_max": max(e2e_ms)},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def variant_leg(args, stream, geo, kw, prec, d_inc, p_inc, dirs, e_ref):
    """The leaf-level variant of the block tree (admissible pairs of two elements integrated as
    element blocks instead of compressed; option leaf_dense, a departure from the paper's FMM)
    on the same workload and form: solves/s over whole steps (setup, solve, far field), product
    phases, and the far-field difference from the paper's FMM solution."""
    import torch
    from paper_1807_03097_gb300 import Solver

    s = Solver(geo, stream=stream.cuda_stream, precision=prec, leaf_dense=1, **kw)
    N = s.ndof
    wdev = torch.zeros((1, N), dtype=torch.complex128, device="cuda")
    edev = torch.zeros((1, 64, 3), dtype=torch.complex128, device="cuda")
    for _ in range(2):
        s.setup()
        s.solve_plane_waves(d_inc, p_inc, out=wdev)
        s.far_field(wdev[0], dirs, out=edev)
    steps = 3
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = []
    for _ in range(steps):
        s.setup()
        _, info, _ = s.solve_plane_waves(d_inc, p_inc, out=wdev)
        s.far_field(wdev[0], dirs, out=edev)
        its.append(info.iterations)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    st = s.setup_timings()
    x = torch.from_numpy(np.random.default_rng(0).standard_normal(N) + 0j).cuda()
    y = torch.empty_like(x)
    ph = []
    for i in range(13):
        s.matvec(x, out=y)
        if i >= 3:
            ph.append(s.last_timings())
    mv = {k: statistics.median([p[k] for p in ph]) for k in ph[0]}
    e = edev[0].cpu().numpy()
    out = {"solves_per_s": 1000.0 / ms, "ms_per_step": ms, "gmres_iterations": int(np.median(its)),
           "setup_ms": st["setup_ms"], "separated_pairs": int(st["near_sep_pairs"]),
           "separated_pairs_ms": st["near_sep_ms"], "far_pairs": int(s.nfar), "near_pairs": int(s.nnear),
           "matvec_per_s": 1000.0 / mv["total"], "matvec_ms_phases": mv,
           "far_field_rel_diff_vs_fmm": float(np.abs(e - e_ref).max() / np.abs(e_ref).max()),
           "note": "timed on the host clock around synchronous calls, 3 steps after 2 warm-up steps"}
    s.close()
    return out


def m2l_pairs_leg(stream, geo, kw, prec, m2l_ms_ordered):
    """The M2L over unordered admissible pairs (option m2l_pairs: each coupling tile evaluated
    once and applied in both directions) on the same workload: product phases and the M2L
    time against the default form's."""
    import torch
    from paper_1807_03097_gb300 import Solver

    s = Solver(geo, stream=stream.cuda_stream, precision=prec, m2l_pairs=1, **kw)
    N = s.ndof
    x = torch.from_numpy(np.random.default_rng(0).standard_normal(N) + 0j).cuda()
    y = torch.empty_like(x)
    ph = []
    for i in range(13):
        s.matvec(x, out=y)
        if i >= 3:
            ph.append(s.last_timings())
    mv = {k: statistics.median([p[k] for p in ph]) for k in ph[0]}
    s.close()
    return {"matvec_per_s": 1000.0 / mv["total"], "matvec_ms_phases": mv, "m2l_ms_ordered_pairs": m2l_ms_ordered,
            "note": "M2L phase = pair kernel + per-cluster sum of the transposed contributions"}


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


def multi_leg(args, steps=None, pk_alu=None):
    """One step = one matrix-vector product of all 64 right-hand sides (a batched GMRES
    iteration's product); value = right-hand-side products per second.  Returns the line."""
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
    steps = steps or args.steps
    for _ in range(max(3, min(args.warmup, steps))):
        s.matvec(x, out=y)
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    l0 = s.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ph = []
    for _ in range(steps):
        s.matvec(x, out=y)
        ph.append(s.last_timings())
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = s.launch_count() - l0
    ms = ev0.elapsed_time(ev1) / steps
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
    if pk_alu and pk_alu.get("tcgen05_tf32_flops", 0) > 0:
        # the primary peak: tcgen05 TF32 as measured on this GPU (microbench/peaks.cu); the
        # BF16-derived figure stays beside it
        tf = pk_alu["tcgen05_tf32_flops"] / 1e12
        roof["peak_derived_bf16x1.1/2.25"] = tf32_peak
        roof["frac_of_derived_peak"] = roof["frac"]
        roof["peak"] = tf
        roof["frac"] = useful / m2l_s / 1e12 / tf
        roof["peak_note"] = "tcgen05.mma kind::tf32 (M128 N256) measured on this GPU (microbench/peaks.cu)"
        roof["executed_frac"] = executed / m2l_s / 1e12 / tf
    # end to end with host buffers
    yh = np.empty_like(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(max(1, args.e2e_steps)):
        s.matvec(b, out=yh)
    e2e_ms = (time.perf_counter() - t0) * 1000.0 / max(1, args.e2e_steps)
    line = {"metric": "FMM-EFIE matvec/s (right-hand-side products per second, 64 right-hand sides per "
                      "batched product), mixed precision",
            "value": R * 1000.0 / ms, "unit": "matvec/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "tf32x3-m2l/f32/f64", "data": "synthetic", "config": MULTI, "ndof": int(N),
            "far_pairs": int(s.nfar), "near_pairs": int(s.nnear), "setup_s": setup_s,
            "matvec_ms_phases": mv, "single_rhs_matvec_ms": single_ms,
            "tensor_vs_single_rhs_rel_diff": diffs, "rel_err_vs_fp64": fp64, "roofline": roof, "cpu_baseline": None,
            "cpu_baseline_note": "the FP64 oracle is timed on the default workload only",
            "e2e": {"value": R * 1000.0 / e2e_ms, "unit": "matvec/s", "h2d_bytes_per_step": int(b.nbytes),
                    "d2h_bytes_per_step": int(yh.nbytes)},
            "gpu_launches": int(launches), "clocks": clocks}
    s.close()
    return line


def run_multi(args):
    pk_alu, _ = measured_peaks()
    print(json.dumps(multi_leg(args, pk_alu=pk_alu)))
    return 0


# ---------------------------------------------------------------------------- Tesla settings
TESLA = {
    "workload": "multicell232_nurbs_p4_n2_kappa4_q14_eta0.1",
    "geometry": "synthetic surface of revolution of 9 bulges (232 rational biquadratic patches; stand-in for "
                "the paper's multi-cell cavities, whose geometry is not available)",
    "p": 4, "elements_per_patch": "2x2", "level_m": 1, "kappa": 4.0, "q": 14, "eta": 0.1, "gmres_tol": 1e-6,
    "incident": "dir +z, pol x", "precision": "mixed",
}


def tesla_leg(args):
    """The paper's Tesla settings (p = 4, eta = 0.1, q = 14) on the 232-patch stand-in: setup,
    matvec/s of the mixed and FP64 forms, their difference, and one mixed solve."""
    import torch
    from paper_1807_03097_gb300 import Solver

    w = TESLA
    geo = G.multicell()
    stream = torch.cuda.current_stream()
    kw = dict(p=w["p"], level_m=w["level_m"], kappa=w["kappa"], q=w["q"], eta=w["eta"], gmres_tol=w["gmres_tol"],
              gmres_maxit=1000)
    t0 = time.perf_counter()
    s = Solver(geo, stream=stream.cuda_stream, precision=1, **kw)
    setup_s = time.perf_counter() - t0
    N = s.ndof
    x = torch.from_numpy(np.random.default_rng(0).standard_normal(N) + 1j * np.random.default_rng(1).standard_normal(N)).cuda()
    y = torch.empty_like(x)
    ph = []
    for i in range(8):
        s.matvec(x, out=y)
        if i >= 3:
            ph.append(s.last_timings())
    mv = {k: statistics.median([p_[k] for p_ in ph]) for k in ph[0]}
    y32 = y.clone()
    s64 = Solver(geo, stream=stream.cuda_stream, precision=0, **kw)
    y64 = torch.empty_like(x)
    ph64 = []
    for i in range(3):
        s64.matvec(x, out=y64)
        ph64.append(s64.last_timings())
    mv64 = {k: statistics.median([p_[k] for p_ in ph64]) for k in ph64[0]}
    err = float(torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64))
    s64.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, info, st = s.solve_plane_waves(np.array([[0, 0, 1.0]]), np.array([[1.0, 0, 0]]))
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    out = {"config": TESLA, "ndof": int(N), "far_pairs": int(s.nfar), "near_pairs": int(s.nnear),
           "setup_s": setup_s, "matvec_per_s": 1000.0 / mv["total"], "matvec_ms_phases": mv,
           "matvec_per_s_fp64": 1000.0 / mv64["total"], "matvec_rel_err_vs_fp64": err,
           "solve_s": solve_s, "gmres_iterations": int(info.iterations), "converged": bool(info.converged),
           "relative_residual": float(info.residual), "status": int(st),
           "note": "unpreconditioned GMRES at p = 4 converges slowly (the paper's Tab. 2: up to ~8000 iterations); "
                   "the solve is capped at 1000 iterations and its residual reported"}
    s.close()
    return out


def run_tesla(args):
    print(json.dumps(tesla_leg(args)))
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
    "m2l": "autotuned per problem at setup (ordered vs unordered-pair kernel, m2l_pairs=2)",
    "execution": "256 contexts set up on 16 host threads (efie_setup_many), then one lockstep group solve "
                 "(efie_group_solve): per GMRES step one CUDA-graph launch holding every unfinished "
                 "problem's product chain as a branch and the Arnoldi/Givens kernels of all systems",
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


def batch_leg(args, n=None):
    """The 256-solve mix as one lockstep group; host clock around synchronous calls, from the
    geometry upload to the solutions in host memory."""
    import torch
    from paper_1807_03097_gb300 import Solver
    from paper_1807_03097_gb300.efie import Group, setup_many

    torch.cuda.set_device(0)
    reqs = batch_requests(n or BATCH["solves"], BATCH["seed"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solvers = []
    for r in reqs:
        sv = Solver(None, m2l_pairs=2, **r["opt"])
        sv.set_geometry(r["geo"])
        solvers.append(sv)
    setup_many(solvers, nthreads=16)
    t1 = time.perf_counter()
    bs = [sv.rhs(r["dirs"], r["pols"])[0] for sv, r in zip(solvers, reqs)]
    g = Group(solvers)
    t2 = time.perf_counter()
    xs, its, res, conv, st = g.solve(bs)
    t3 = time.perf_counter()
    stats = g.stats()
    tune = [sv.setup_timings() for sv in solvers]
    launches_setup = sum(sv.launch_count() for sv in solvers)
    g.close()
    for sv in solvers:
        sv.close()
    total = t3 - t0
    kept = [int(t["m2l_kept"]) for t in tune]
    return {"metric": "batch of independent solves: solves/s (mixed precision, GMRES 1e-5)",
            "sample": f"the first {len(reqs)} of the {BATCH['solves']} seeded solves of the mix",
            "value": len(reqs) / total, "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "solves": len(reqs), "converged": int(conv.sum()), "total_s": total, "setup_s": t1 - t0,
            "rhs_and_group_s": t2 - t1, "group_solve_s": t3 - t2,
            "steps": int(stats["steps"]), "ms_per_step": (t3 - t2) * 1e3 / max(stats["steps"], 1),
            "product_graph_captures": int(stats["graph_captures"]),
            "product_graph_kernels_first": int(stats["product_graph_kernels"]),
            "kernels_in_solve": int(stats["kernels"]), "kernels_setup_and_warmup": int(launches_setup),
            "graph_device_ms": {"pre": stats.get("pre_ms"), "products": stats.get("products_ms"),
                                "post_gmres": stats.get("post_ms")},
            "gmres_iterations_median": int(np.median(its)), "gmres_iterations_max": int(its.max()),
            "residual_max": float(res.max()),
            "m2l_autotune": {"unordered_pairs_kept": int(sum(kept)), "ordered_kept": int(len(kept) - sum(kept))},
            "total_dofs": int(sum(sv_n for sv_n in (x.shape[-1] for x in xs))), "data": "synthetic",
            "config": BATCH}


def run_batch(args):
    clk = ClockSampler(0)
    clk.start()
    line = batch_leg(args, n=args.batch_n)
    line["clocks"] = clk.stop()
    print(json.dumps(line))
    return 0


def serving_leg(args):
    """The serving stream: Poisson arrivals through the serving loop; returns the line."""
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
            "dofs": [int(x[0].ndof) for x in res], "data": "synthetic", "config": SERVING,
            "footprint_over_device_peak_min": float(min(x[0].footprint_bytes / max(x[0].device_peak_bytes, 1)
                                                        for x in res)),
            "footprint_over_device_peak": [round(x[0].footprint_bytes / max(x[0].device_peak_bytes, 1), 3)
                                           for x in res],
            "trace": [{"arrival_s": round(r["t"], 4), "ndof": int(x[0].ndof), "directions": len(r["dirs"]),
                       "p": r["opt"]["p"], "kappa": round(r["opt"]["kappa"], 3), "status": int(x[0].status),
                       "iterations": int(x[0].iterations), "queue_ms": round(x[0].queue_ms, 1),
                       "latency_ms": round(x[0].latency_ms, 1)} for r, x in zip(reqs, res)]}
    return line


def run_serving(args):
    print(json.dumps(serving_leg(args)))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--maxit", type=int, default=MAXIT)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the 64-right-hand-side torus and serving legs")
    ap.add_argument("--no-fp64-solve", action="store_true", help="skip the plain FP64 solve of the workload")
    ap.add_argument("--no-variant", action="store_true", help="skip the leaf-level block-tree variant")
    ap.add_argument("--multi-steps", type=int, default=3, help="timed batched products of the torus leg")
    ap.add_argument("--ref-iterations", type=int, default=WORKLOAD_ITERATIONS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-steps", action="store_true", help="time the steps only (for launch-list profiling)")
    ap.add_argument("--workload", default="solve", choices=["solve", "serving", "multi", "batch", "tesla"])
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-solve group leg of the default run")
    ap.add_argument("--batch-n", type=int, default=None, help="solves of the batch leg (default 256)")
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
    if args.workload == "tesla":
        return run_tesla(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
