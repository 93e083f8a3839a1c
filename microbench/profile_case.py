"""Run a few matrix-vector products of one configurable case (for profiling a kernel on a
case smaller than the benchmark's).  Example:
    python microbench/profile_case.py --p 2 --m 4 --kappa 10 --q 8 --precision mixed --matvecs 3
--nrhs R > 1 applies each product to R random right-hand sides at once (batched product);
--near-only applies the near-field blocks alone (efie_near_apply) instead of the product.
"""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--geometry", default="sphere", choices=["sphere", "torus", "cube"])
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--m", type=int, default=4)
    ap.add_argument("--kappa", type=float, default=10.0)
    ap.add_argument("--q", type=int, default=8)
    ap.add_argument("--eta", type=float, default=1.6)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--matvecs", type=int, default=3)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--m2l-batch", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--near-only", action="store_true", help="near-field product alone (one superspace vector)")
    ap.add_argument("--m2l-pairs", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--lib", default=None, help="path of another build of libefie.so")
    a = ap.parse_args()
    from paper_1807_03097_gb300 import Solver, efie

    if a.lib:
        efie.load(a.lib)
    from workloads import geometry as G

    geo = {"sphere": G.sphere, "torus": G.torus, "cube": G.cube}[a.geometry]()
    import time

    t0 = time.perf_counter()
    s = Solver(geo, p=a.p, level_m=a.m, kappa=a.kappa, q=a.q, eta=a.eta, precision=1 if a.precision == "mixed" else 0,
               m2l_batch=a.m2l_batch, m2l_pairs=a.m2l_pairs)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    s.setup()
    t_setup2 = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    n = s.nsup if a.near_only else s.ndof
    shape = (a.nrhs, n) if a.nrhs > 1 else (n,)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for _ in range(a.matvecs):
        y = s.near_apply(x) if a.near_only else s.matvec(x)
    t = s.last_timings()
    print(f"nrhs {a.nrhs} ndof {s.ndof} far {s.nfar} near {s.nnear} setup s {t_setup:.3f} (again {t_setup2:.3f}) matvec ms "
          + " ".join(f"{k}={v:.3f}" for k, v in t.items()))
    s.close()


if __name__ == "__main__":
    main()
