"""Settings of the paper's Tesla-cavity runs (Sec. 5.3: p = 4, eta = 0.1, q = 14) on the synthetic
232-patch surface of revolution (the cavity geometries are not available): block lists, sampled
superspace rows of the FP64 and mixed products against the oracle (1e-11, 1e-5), the batched
product of several right-hand sides (its M2L tile is beyond the shared-memory kernels, so each
right-hand side takes the single-field kernel) against the single products, and a capped solve
whose reported residual is checked with the oracle's operator."""
import numpy as np
import pytest

import oracle as O
from workloads import geometry as G

pytestmark = pytest.mark.gpu

KW = dict(p=4, level_m=0, kappa=4.0, q=14, eta=0.1)


@pytest.fixture(scope="module")
def cavity():
    from paper_1807_03097_gb300 import Solver

    geo = G.multicell()
    s64 = Solver(geo, **KW)
    s32 = Solver(geo, precision=1, **KW)
    r = O.Problem(geo, p=KW["p"], m=KW["level_m"], kappa=KW["kappa"], q=KW["q"], eta=KW["eta"])
    yield s64, s32, r
    s64.close()
    s32.close()


def test_f2_block_lists(cavity):
    s64, s32, r = cavity
    far, near = s64.blocks()
    assert len(far) > 0
    assert sorted(map(tuple, far)) == sorted(map(tuple, r.far_pairs()))
    assert sorted(map(tuple, near)) == sorted(map(tuple, r.near_pairs()))


def test_f2_sampled_rows_vs_oracle(cavity):
    s64, s32, r = cavity
    rng = np.random.default_rng(90)
    xs = rng.standard_normal(r.nsup) + 1j * rng.standard_normal(r.nsup)
    y64 = s64.matvec_superspace(xs).reshape(r.nE, r.nb)
    y32 = s32.matvec_superspace(xs).reshape(r.nE, r.nb)
    elems = np.array([3, 150])
    rows = r.fmm_rows(xs, elems)
    scale = np.abs(rows).max()
    assert np.abs(y64[elems] - rows).max() / scale < 1e-11
    assert np.abs(y32[elems] - rows).max() / scale < 1e-5


def test_f2_batched_product_and_solve(cavity):
    s64, s32, r = cavity
    rng = np.random.default_rng(91)
    x = rng.standard_normal((3, s32.ndof)) + 1j * rng.standard_normal((3, s32.ndof))
    y = s32.matvec(x)
    for i in range(3):
        yi = s32.matvec(x[i])
        assert np.linalg.norm(y[i] - yi) / np.linalg.norm(yi) < 1e-6
    # unpreconditioned GMRES converges slowly at p = 4 (the paper's Tab. 2 needs up to ~8000
    # iterations): a capped solve must return its last iterate, whose true residual with the
    # oracle's operator is the residual the library reports (up to the mixed operator's error)
    from paper_1807_03097_gb300 import Solver

    s = Solver(G.multicell(), precision=1, gmres_maxit=150, gmres_tol=1e-8, **KW)
    d, pol = G.plane_waves(1, seed=93)
    w, info, st = s.solve_plane_waves(d, pol)
    s.close()
    assert st == 1 and not info.converged and info.iterations == 150
    b = r.rhs(d[0], pol[0])
    res = np.linalg.norm(b - r.fmm_matvec(w[0])[0]) / np.linalg.norm(b)
    assert res < 1.0 and abs(res - info.residual) < 1e-5 + 1e-3 * res, (res, info.residual)
