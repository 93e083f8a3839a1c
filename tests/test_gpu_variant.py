"""Leaf-level variant of the block tree (option leaf_dense): admissible pairs of two elements are
integrated as element blocks (tensor Gauss, quad_regular points) instead of being compressed.
The library's variant against the oracle's variant: block lists identical, near-field blocks and
FP64 products within 1e-11, mixed products within 1e-5; the variant on the sphere at m = 1
(every admissible pair a pair of leaves) against the dense Galerkin product."""
import numpy as np
import pytest

import oracle as O
from workloads import geometry as G

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32 = 1e-5

CASES = {
    "sphere_p2_m2_q5": (G.sphere, 2, 2, 3.0, 5, 1.6),
    "torus_p1_m2_q4": (G.torus, 1, 2, 2.0, 4, 1.6),
    "sphere_p1_m1_q4": (G.sphere, 1, 1, 2.0, 4, 1.6),
}


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name", list(CASES))
def test_leaf_dense_variant_vs_oracle(name):
    from paper_1807_03097_gb300 import Solver

    mk, p, m, k, q, eta = CASES[name]
    geo = mk()
    s = Solver(geo, p=p, level_m=m, kappa=k, q=q, eta=eta, leaf_dense=1)
    s32 = Solver(geo, p=p, level_m=m, kappa=k, q=q, eta=eta, leaf_dense=1, precision=1)
    r = O.Problem(geo, p=p, m=m, kappa=k, q=q, eta=eta, leaf_dense=True)
    far, near = s.blocks()
    assert sorted(map(tuple, far)) == sorted(map(tuple, r.far_pairs()))
    assert sorted(map(tuple, near)) == sorted(map(tuple, r.near_pairs()))
    idx = {tuple(x_): i for i, x_ in enumerate(r.near_pairs())}
    perm = [idx[tuple(x_)] for x_ in near]
    assert relmax(s.near_blocks(), r.near_blocks()[perm]) < TOL64
    rng = np.random.default_rng(80)
    x = rng.standard_normal(s.ndof) + 1j * rng.standard_normal(s.ndof)
    yr = r.fmm_matvec(x)[0]
    assert relmax(s.matvec(x), yr) < TOL64
    assert np.linalg.norm(s32.matvec(x) - yr) / np.linalg.norm(yr) < TOL32
    if name == "sphere_p1_m1_q4":
        assert len(far) == 0
        yd = r.dense_matvec(x)[0]
        assert relmax(s.matvec(x), yd) < TOL64
    s.close()
    s32.close()


@pytest.mark.parametrize("name", ["sphere_p2_m2_q5", "torus_p1_m2_q4"])
def test_unordered_pair_m2l_vs_oracle(name):
    """Option m2l_pairs = 1: each admissible pair's coupling tile evaluated once and applied in
    both directions (K_st = K_ts^T); the mixed product against the oracle (1e-5) and against the
    default form, including the full-size sphere workload's sampled rows."""
    from paper_1807_03097_gb300 import Solver

    mk, p, m, k, q, eta = CASES[name]
    geo = mk()
    s = Solver(geo, p=p, level_m=m, kappa=k, q=q, eta=eta, precision=1, m2l_pairs=1)
    s0 = Solver(geo, p=p, level_m=m, kappa=k, q=q, eta=eta, precision=1)
    r = O.Problem(geo, p=p, m=m, kappa=k, q=q, eta=eta)
    rng = np.random.default_rng(81)
    x = rng.standard_normal(s.ndof) + 1j * rng.standard_normal(s.ndof)
    yr = r.fmm_matvec(x)[0]
    y = s.matvec(x)
    assert np.linalg.norm(y - yr) / np.linalg.norm(yr) < TOL32
    assert np.linalg.norm(y - s0.matvec(x)) / np.linalg.norm(yr) < TOL32
    s.close()
    s0.close()


def test_unordered_pair_m2l_full_size_rows():
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    kw = dict(p=2, level_m=5, kappa=10.0, q=8, eta=1.6)
    s = Solver(geo, precision=1, m2l_pairs=1, **kw)
    r = O.Problem(geo, p=2, m=5, kappa=10.0, q=8, eta=1.6)
    rng = np.random.default_rng(82)
    xs = rng.standard_normal(s.nsup) + 1j * rng.standard_normal(s.nsup)
    y = s.matvec_superspace(xs).reshape(-1, 18)
    elems = np.array([0, 777, 3 * 1024 + 517, 6143])
    rows = r.fmm_rows(xs, elems)
    assert np.abs(y[elems] - rows).max() / np.abs(rows).max() < TOL32
    s.close()


def test_m2l_autotune_keeps_a_timed_kernel_and_matches_oracle():
    """Option m2l_pairs = 2: setup times the ordered and the unordered-pair M2L on the problem's
    own blocks and keeps the faster; the product is then bitwise the product of the kernel kept
    (the same solver built with m2l_pairs 0 or 1), and within 1e-5 of the oracle."""
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    kw = dict(p=1, level_m=3, kappa=3.0, q=5, eta=1.6, precision=1)
    s = Solver(geo, m2l_pairs=2, **kw)
    t = s.setup_timings()
    assert t["m2l_ordered_ms"] > 0 and t["m2l_pairs_ms"] > 0
    kept = int(t["m2l_kept"])
    assert kept == (0 if t["m2l_ordered_ms"] <= t["m2l_pairs_ms"] else 1)
    ref = Solver(geo, m2l_pairs=kept, **kw)
    r = O.Problem(geo, p=1, m=3, kappa=3.0, q=5, eta=1.6)
    rng = np.random.default_rng(83)
    x = rng.standard_normal(s.ndof) + 1j * rng.standard_normal(s.ndof)
    y = s.matvec(x)
    assert np.array_equal(y, ref.matvec(x))
    yr = r.fmm_matvec(x)[0]
    assert np.linalg.norm(y - yr) / np.linalg.norm(yr) < TOL32
    s.close()
    ref.close()
