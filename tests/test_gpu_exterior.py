"""Electric field off the surface (eq. ESLP) and the manufactured solution of Sec. 5.2 on the
GPU, through the C ABI, against the FP64 oracle (1e-11, same quadrature rules) and against
the Hertz dipole itself."""
import numpy as np
import pytest

import oracle as O
from workloads import geometry as G

pytestmark = pytest.mark.gpu

X0 = np.array([0.0, 0.1, 0.1])
P0 = np.array([0.0, 0.1, 0.1])


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def sphere_points(n, radius):
    k = np.arange(n) + 0.5
    z = 1 - 2 * k / n
    ph = np.pi * (1 + 5 ** 0.5) * k
    r = np.sqrt(1 - z * z)
    return radius * np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)


@pytest.mark.parametrize("case", [(G.sphere, 2, 1, 3.0), (G.torus, 1, 1, 1.5)], ids=["sphere_p2", "torus_p1"])
def test_exterior_field_and_dipole_rhs_match_oracle(case):
    from paper_1807_03097_gb300 import Solver

    mk, p, m, k = case
    geo = mk()
    s = Solver(geo, p=p, level_m=m, kappa=k, q=4, eta=1.6)
    r = O.Problem(geo, p=p, m=m, kappa=k, q=4, eta=1.6)
    rng = np.random.default_rng(50)
    w = rng.standard_normal((2, s.ndof)) + 1j * rng.standard_normal((2, s.ndof))
    pts = np.concatenate([sphere_points(7, 4.0), sphere_points(5, 6.5)])
    e = s.exterior_field(w, pts)
    for i in range(2):
        assert relmax(e[i], r.exterior_field(w[i], pts)) < 1e-11
    g = s.rhs_dipole([X0, -X0], [P0, P0])
    assert relmax(g[0], r.rhs_dipole(X0, P0)) < 1e-11
    assert relmax(g[1], r.rhs_dipole(-X0, P0)) < 1e-11
    s.close()


def test_manufactured_dipole_solution_on_the_sphere():
    """Sec. 5.2: solve with the dipole's trace, evaluate the field at 100 points on |x| = 3;
    p = 1 with 4x4 elements per patch, kappa = 1: the error is the oracle's dense-solve value
    (1.46e-4) up to the FMM and GMRES tolerances."""
    from paper_1807_03097_gb300 import Solver

    s = Solver(G.sphere(), p=1, level_m=2, kappa=1.0, q=8, eta=1.6, gmres_tol=1e-10)
    b = s.rhs_dipole(X0, P0)[0]
    x, info, st = s.solve(b)
    assert st == 0 and info.converged
    pts = sphere_points(100, 3.0)
    err = np.linalg.norm(s.exterior_field(x, pts)[0] - O.dipole_field(1.0, X0, P0, pts), axis=1).max()
    assert 1.2e-4 < err < 1.8e-4, err
    s.close()
