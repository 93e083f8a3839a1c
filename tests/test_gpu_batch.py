"""Several right-hand sides at once (mixed form): batched matvec and lockstep GMRES.

The batched M2L evaluates each coupling tile once per admissible block and applies it to the
fields of up to 8 right-hand sides; every result is checked against the FP64 oracle at the
mixed-precision tolerance (1e-5 relative, 2-norm per right-hand side) and against the
single-right-hand-side mixed product.  Lockstep solves are checked through the oracle's own
FP64 operator: each returned iterate must have a true relative residual within the GMRES
tolerance plus the mixed operator's error.
"""
import numpy as np
import pytest

import oracle as O
from workloads import geometry as G

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def rel2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def random_block(n, ndof, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, ndof)) + 1j * rng.standard_normal((n, ndof))


MATVEC_CASES = {
    # (geometry, p, m, kappa, q, nrhs): ragged field groups (11 -> 44 fields), a torus, 20
    # right-hand sides (80 fields: a full and a ragged tensor-core group), the largest
    # tensor-core tile (q = 10, 121 nodes), the largest CUDA-core tile (q = 11, 144 nodes),
    # and q = 12, where every right-hand side takes the single-field kernel
    "sphere_p2_m2_q6_r11": (G.sphere, 2, 2, 3.0, 6, 11),
    "torus_p2_m1_q5_r3": (G.torus, 2, 1, 2.0, 5, 3),
    "sphere_p1_m2_q8_r20": (G.sphere, 1, 2, 4.0, 8, 20),
    "sphere_p1_m1_q10_r17": (G.sphere, 1, 1, 2.0, 10, 17),
    "sphere_p1_m1_q11_r9": (G.sphere, 1, 1, 2.0, 11, 9),
    "sphere_p1_m1_q12_r2": (G.sphere, 1, 1, 2.0, 12, 2),
    # p = 3 and p = 4: near-field blocks of 32 x 32 and 50 x 50 in the batched near field
    "cube_p3_m1_q5_r9": (G.cube, 3, 1, 1.5, 5, 9),
    "sphere_p4_m1_q4_r5": (G.sphere, 4, 1, 1.0, 4, 5),
}
# m2l_batch: 1 CUDA cores, 2 tensor cores (q <= 10)
MATVEC_PARAMS = [(c, b) for c in MATVEC_CASES for b in (1, 2) if b == 1 or MATVEC_CASES[c][4] <= 10]


@pytest.mark.parametrize("name,batch", MATVEC_PARAMS,
                         ids=[f"{c}-{'cuda' if b == 1 else 'tensor'}" for c, b in MATVEC_PARAMS])
def test_batched_matvec_vs_oracle(name, batch):
    from paper_1807_03097_gb300 import Solver

    mk, p, m, k, q, nrhs = MATVEC_CASES[name]
    geo = mk()
    s = Solver(geo, p=p, level_m=m, kappa=k, q=q, eta=1.6, precision=1, m2l_batch=batch)
    r = O.Problem(geo, p=p, m=m, kappa=k, q=q, eta=1.6)
    x = random_block(nrhs, s.ndof, 21)
    y = s.matvec(x)
    yr = r.fmm_matvec(x)
    for i in range(nrhs):
        assert rel2(y[i], yr[i]) < TOL32, (i, rel2(y[i], yr[i]))
        assert rel2(y[i], s.matvec(x[i])) < TOL32
    s.close()


def test_tensor_core_m2l_rejects_large_q():
    from paper_1807_03097_gb300 import Solver
    from paper_1807_03097_gb300.efie import EfieError

    with pytest.raises(EfieError):
        Solver(G.sphere(), p=1, level_m=1, kappa=1.0, q=11, eta=1.6, precision=1, m2l_batch=2)


def test_batched_matvec_more_than_one_chunk():
    """70 right-hand sides: two passes (64 + 6)."""
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    s = Solver(geo, p=1, level_m=2, kappa=1.0, q=4, eta=1.6, precision=1)
    r = O.Problem(geo, p=1, m=2, kappa=1.0, q=4, eta=1.6)
    x = random_block(70, s.ndof, 22)
    y = s.matvec(x)
    for i in (0, 31, 32, 63, 64, 69):
        assert rel2(y[i], r.fmm_matvec(x[i])[0]) < TOL32, i
    s.close()


def test_batched_matvec_varying_count():
    """Products with 11, 2, then 7 right-hand sides on one context (as in a lockstep solve
    whose systems finish at different steps): each must match the oracle."""
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    s = Solver(geo, p=2, level_m=2, kappa=3.0, q=4, eta=1.6, precision=1)
    r = O.Problem(geo, p=2, m=2, kappa=3.0, q=4, eta=1.6)
    for n, seed in ((11, 31), (2, 32), (7, 33)):
        x = random_block(n, s.ndof, seed)
        y = s.matvec(x)
        yr = r.fmm_matvec(x)
        for i in range(n):
            assert rel2(y[i], yr[i]) < TOL32, (n, i, rel2(y[i], yr[i]))
    s.close()


def test_batched_matvec_device_pointers_match_host():
    torch = pytest.importorskip("torch")
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    s = Solver(geo, p=2, level_m=1, kappa=2.0, q=5, eta=1.6, precision=1)
    x = random_block(5, s.ndof, 23)
    yh = s.matvec(x)
    yd = s.matvec(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), yh)
    s.close()


@pytest.mark.parametrize("restart", [1500, 9], ids=["no_restart", "restart9"])
def test_lockstep_solve_residuals(restart):
    """Five plane waves and a zero right-hand side solved together; systems finish at
    different steps (and, with restart 9, restart at different steps)."""
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    tol = 1e-5
    s = Solver(geo, p=1, level_m=2, kappa=1.0, q=4, eta=1.6, precision=1, gmres_tol=tol, gmres_restart=restart)
    r = O.Problem(geo, p=1, m=2, kappa=1.0, q=4, eta=1.6)
    rng = np.random.default_rng(24)
    d = rng.standard_normal((5, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pol = np.cross(d, rng.standard_normal((5, 3)))
    pol /= np.linalg.norm(pol, axis=1, keepdims=True)
    B = np.stack([r.rhs(d[i], pol[i]) for i in range(5)] + [np.zeros(s.ndof, complex)])
    X, info, st = s.solve(B)
    assert st == 0 and info.converged
    assert np.all(X[5] == 0)
    for i in range(5):
        res = np.linalg.norm(B[i] - r.fmm_matvec(X[i])[0]) / np.linalg.norm(B[i])
        assert res < 2 * tol, (i, res)
        # the same system solved alone
        xi, inf1, st1 = s.solve(B[i])
        assert st1 == 0 and inf1.converged
        assert rel2(X[i], xi) < 1e-3
    # plane-wave entry point: the same as solving the assembled right-hand sides
    W, info2, st2 = s.solve_plane_waves(d, pol)
    assert st2 == 0 and info2.converged
    for i in range(5):
        assert rel2(W[i], X[i]) < 1e-4
    s.close()


def test_lockstep_not_converged():
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    s = Solver(geo, p=1, level_m=1, kappa=1.0, q=4, eta=1.6, precision=1, gmres_maxit=3, gmres_tol=1e-12)
    w, info, st = s.solve_plane_waves([[0, 0, 1.0], [1.0, 0, 0]], [[1.0, 0, 0], [0, 1.0, 0]])
    assert st == 1 and not info.converged and info.iterations == 3
    assert np.all(np.isfinite(w)) and np.abs(w).max() > 0
    s.close()
