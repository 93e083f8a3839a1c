"""Lockstep group of independent problems (efie_group_*): problems of different geometry,
degree, refinement, wavenumber and precision solved together, one CUDA-graph launch of all
products per GMRES step.

A system solved in the group takes the same arithmetic in the same order as efie_solve alone
(the product chain of its context, and the Arnoldi/Givens steps of the single-system solver), so
its iterates, iteration count and solution are compared bit for bit with the solve alone; one
problem of each precision is also checked against the FP64 oracle (true residual of the
returned current with the oracle's operator, eq. linsys)."""
import numpy as np
import pytest

import oracle as O
from workloads import geometry as G

pytestmark = pytest.mark.gpu

PROBLEMS = [
    # geometry, p, m, kappa, precision
    (lambda: G.sphere(radius=0.8), 1, 2, 2.0, 1),
    (G.cube, 2, 1, 1.5, 0),
    (G.torus, 1, 2, 3.0, 1),
    (lambda: G.sphere(radius=1.3), 2, 2, 4.0, 0),
]


def make(i, tol=None, maxit=400, restart=1500):
    """FP64 problems solve to 1e-8; mixed ones to 1e-6 (their operator carries FP32 rounding)."""
    from paper_1807_03097_gb300 import Solver

    mk, p, m, k, prec = PROBLEMS[i]
    tol = tol if tol is not None else (1e-6 if prec else 1e-8)
    return Solver(mk(), p=p, level_m=m, kappa=k, q=4, eta=1.6, precision=prec, gmres_tol=tol, gmres_maxit=maxit,
                  gmres_restart=restart)


def rhs(s, i):
    rng = np.random.default_rng(50 + i)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    pol = np.cross(d, [0.2, 0.7, 0.1])
    pol /= np.linalg.norm(pol)
    return s.rhs(d, pol)[0], d, pol


def test_group_equals_each_solve_alone_bitwise():
    from paper_1807_03097_gb300.efie import Group

    solvers = [make(i) for i in range(len(PROBLEMS))]
    bs = [rhs(s, i)[0] for i, s in enumerate(solvers)]
    g = Group(solvers)
    xs, its, res, conv, st = g.solve(bs)
    assert st == 0 and conv.all()
    stats = g.stats()
    assert stats["steps"] >= its.max() and stats["products_ms"] > 0 and stats["post_ms"] > 0
    g.close()
    for i, s in enumerate(solvers):
        x1, info, _ = s.solve(bs[i])
        assert info.converged and info.iterations == its[i], (i, info.iterations, its[i])
        assert np.array_equal(x1, xs[i]), (i, np.abs(x1 - xs[i]).max())
        assert abs(info.residual - res[i]) <= 1e-15 * max(1.0, abs(info.residual))
    for s in solvers:
        s.close()


def test_group_solutions_solve_the_oracle_system():
    from paper_1807_03097_gb300.efie import Group

    idx = [0, 1]  # mixed sphere, FP64 cube
    solvers = [make(i) for i in idx]
    data = [rhs(s, i) for s, i in zip(solvers, idx)]
    g = Group(solvers)
    xs, its, res, conv, st = g.solve([d[0] for d in data])
    g.close()
    assert conv.all()
    for k, i in enumerate(idx):
        mk, p, m, kap, prec = PROBLEMS[i]
        ref = O.Problem(mk(), p=p, m=m, kappa=kap, q=4, eta=1.6)
        b = ref.rhs(data[k][1], data[k][2])
        assert np.abs(b - data[k][0]).max() < 1e-11 * np.abs(b).max()
        r = np.linalg.norm(b - ref.fmm_matvec(xs[k])[0]) / np.linalg.norm(b)
        # FP64: the GMRES tolerance; mixed: its tolerance plus the mixed operator's error (1e-5)
        assert r < (2e-8 if prec == 0 else 2e-5), (i, r)
    for s in solvers:
        s.close()


def test_group_device_pointers_zero_rhs_and_non_convergence():
    torch = pytest.importorskip("torch")
    from paper_1807_03097_gb300.efie import Group

    solvers = [make(0), make(1, maxit=7), make(2)]
    bs = [rhs(s, i)[0] for i, s in enumerate(solvers)]
    bs[2] = np.zeros_like(bs[2])
    g = Group(solvers)
    xh, its, res, conv, st = g.solve(bs)
    assert st == 1  # EFIE_NOT_CONVERGED: the capped system
    assert conv[0] == 1 and conv[1] == 0 and its[1] == 7 and conv[2] == 1 and its[2] == 0
    assert not np.any(xh[2])
    xd, its2, res2, conv2, st2 = g.solve([torch.from_numpy(b).cuda() for b in bs])
    torch.cuda.synchronize()
    for a, b in zip(xh, xd):
        assert np.array_equal(a, b.cpu().numpy())
    assert np.array_equal(its, its2) and np.array_equal(conv, conv2)
    # the capped system as a solve alone stops at the same iterate
    x1, info, _ = solvers[1].solve(bs[1])
    assert not info.converged and np.array_equal(x1, xh[1])
    g.close()
    for s in solvers:
        s.close()


def test_group_recaptures_products_as_systems_finish_and_setup_many():
    from paper_1807_03097_gb300 import Solver
    from paper_1807_03097_gb300.efie import Group, setup_many

    # ten problems, from easy (small kappa, few elements) to harder: they finish at different
    # steps, so the product graph is captured again without the finished ones
    solvers = []
    for i in range(10):
        s = Solver(None, p=1, level_m=1 + (i % 3), kappa=1.0 + 0.8 * i, q=4, eta=1.6, precision=1, gmres_tol=1e-6,
                   gmres_maxit=500)
        s.set_geometry(G.sphere(radius=0.5 + 0.1 * i) if i % 2 else G.cube(side=1.0 + 0.1 * i))
        solvers.append(s)
    setup_many(solvers, nthreads=4)
    bs = [rhs(s, i)[0] for i, s in enumerate(solvers)]
    g = Group(solvers)
    xs, its, res, conv, st = g.solve(bs)
    stats = g.stats()
    g.close()
    assert conv.all() and len(set(its.tolist())) > 3
    assert stats["graph_captures"] >= 2
    for i in (0, 9):
        x1, info, _ = solvers[i].solve(bs[i])
        assert info.iterations == its[i] and np.array_equal(x1, xs[i])
    for s in solvers:
        s.close()


def test_group_refuses_a_problem_set_up_again_with_other_sizes():
    """A context set up again with another geometry (another number of DOFs) after the group was
    made is refused at solve time (EFIE_ESTATE) instead of being solved with stale tables."""
    from paper_1807_03097_gb300.efie import Group

    s = make(0)
    g = Group([s])
    b0 = rhs(s, 0)[0]
    xs, its, res, conv, st = g.solve([b0])
    assert conv.all()
    s.set_geometry(G.torus())  # 16 patches: 512 DOFs instead of the sphere's 192
    s.setup()
    with pytest.raises(RuntimeError, match="set up again"):
        g.solve([rhs(s, 0)[0]])
    g.close()
    s.close()
