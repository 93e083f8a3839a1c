"""Device GMRES and the scattering solve against the oracle and the paper (Tab. 1)."""
import numpy as np
import pytest

import oracle as O
from conftest import golden
from workloads import geometry as G

pytestmark = pytest.mark.gpu


def test_solve_sphere_p1_matches_oracle_and_paper():
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    s = Solver(geo, p=1, level_m=2, kappa=1.0, q=4, eta=1.6, gmres_tol=1e-8)
    r = O.Problem(geo, p=1, m=2, kappa=1.0, q=4, eta=1.6)
    w, info, st = s.solve_plane_waves([[0, 0, 1.0]], [[1.0, 0, 0]])
    assert st == 0 and info.converged and info.iterations > 10
    b = r.rhs(np.array([0, 0, 1.0]), np.array([1.0, 0, 0]))
    res = np.linalg.norm(b - r.fmm_matvec(w[0])[0]) / np.linalg.norm(b)
    assert res <= 1.1e-8, res
    xo, its, rres, rc = r.gmres(b, use_fmm=True, tol=1e-8)
    assert np.linalg.norm(w[0] - xo) / np.linalg.norm(xo) < 1e-8 * 10 * its
    err, nrm = r.mie_l2(w[0])
    paper = golden("table1_sphere.txt")
    ref = paper[(paper[:, 0] == 1) & (paper[:, 1] == 4)][0, 5]
    assert abs(err - ref) / ref < 0.1
    s.close()


def test_solve_mixed_precision_and_restart():
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    r = O.Problem(geo, p=1, m=2, kappa=1.0, q=4, eta=1.6)
    b = r.rhs(np.array([0, 0, 1.0]), np.array([1.0, 0, 0]))
    # short restart exercises the restart path; mixed precision at a 1e-5 tolerance
    s = Solver(geo, p=1, level_m=2, kappa=1.0, q=4, eta=1.6, precision=1, gmres_restart=20, gmres_tol=1e-5)
    x, info, st = s.solve(b)
    assert st == 0 and info.converged
    res = np.linalg.norm(b - r.fmm_matvec(x)[0]) / np.linalg.norm(b)
    assert res < 2e-5, res
    s.close()


def test_not_converged_reports_last_iterate():
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    s = Solver(geo, p=1, level_m=1, kappa=1.0, q=4, eta=1.6, gmres_maxit=3, gmres_tol=1e-12)
    w, info, st = s.solve_plane_waves([[0, 0, 1.0]], [[1.0, 0, 0]])
    assert st == 1 and not info.converged and info.iterations == 3
    assert np.all(np.isfinite(w)) and np.abs(w).max() > 0
    s.close()


def test_device_wait_timeout_is_reported_and_context_stays_usable():
    """Failure detection of the device-side waits: a bounded wait on a barrier that nothing
    completes reports EFIE_ETIMEOUT through the same flag as the tensor-core M2L, and the
    context keeps working (single and batched tensor-core products afterwards)."""
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    s = Solver(geo, p=1, level_m=2, kappa=1.0, q=4, eta=1.6, precision=1)
    rng = np.random.default_rng(40)
    x = rng.standard_normal((17, s.ndof)) + 1j * rng.standard_normal((17, s.ndof))
    y0 = s.matvec(x[0])
    yb0 = s.matvec(x)
    st, msg = s.check_device_waits(1 << 20)
    assert st == -6 and "ran out" in msg
    assert np.array_equal(s.matvec(x[0]), y0)
    assert np.array_equal(s.matvec(x), yb0)
    s.close()


def test_geometry_errors():
    from paper_1807_03097_gb300 import Solver
    from paper_1807_03097_gb300.efie import EfieError

    with pytest.raises(EfieError, match="-3"):
        Solver(G.cube()[:5], p=1, level_m=1, kappa=1.0, q=2, eta=1.6)     # open surface
    flipped = []
    for pt in G.sphere():
        q = dict(pt)
        q["cp"] = pt["cp"][::-1].copy()
        q["w"] = pt["w"][::-1].copy()
        flipped.append(q)
    with pytest.raises(EfieError, match="-3"):
        Solver(flipped, p=1, level_m=1, kappa=1.0, q=2, eta=1.6)          # inward normals
    s = Solver(None, p=1, level_m=1)
    with pytest.raises(EfieError, match="-5"):
        s.setup()                                                        # no geometry yet
    s.close()


def test_zero_right_hand_sides_and_zero_vector():
    from paper_1807_03097_gb300 import Solver

    s = Solver(G.sphere(), p=1, level_m=1, kappa=1.0, q=3, eta=1.6)
    y = s.matvec(np.zeros((0, s.ndof), np.complex128))
    assert y.shape == (0, s.ndof)
    x, info, st = s.solve(np.zeros(s.ndof, np.complex128))
    assert st == 0 and np.all(x == 0)
    s.close()


def test_temporaries_are_returned_to_the_pool():
    """Every call's temporary device buffers are returned (stream-ordered) when it ends: after a
    first call of each kind (which may allocate the context's persistent work arrays), repeating
    it leaves the context's live device bytes unchanged, and destroying the context after a
    failed call is clean."""
    from paper_1807_03097_gb300 import Solver

    s = Solver(G.sphere(), p=2, level_m=2, kappa=3.0, q=5, eta=1.6, precision=1)
    rng = np.random.default_rng(90)
    x = rng.standard_normal((3, s.ndof)) + 1j * rng.standard_normal((3, s.ndof))
    xs = rng.standard_normal((3, s.nsup)) + 1j * rng.standard_normal((3, s.nsup))
    dirs = np.array([[0, 0, 1.0], [0, 1.0, 0]])
    pts = np.array([[3.0, 0, 0], [0, 0, -4.0]])
    calls = [
        lambda: s.matvec(x[0]),
        lambda: s.matvec(x),
        lambda: s.matvec_superspace(xs[0]),
        lambda: s.matvec_superspace(xs),
        lambda: s.far_field(x, dirs),
        lambda: s.exterior_field(x, pts),
        lambda: s.rhs(dirs, [[1.0, 0, 0], [1.0, 0, 0]]),
        lambda: s.solve_plane_waves(dirs, [[1.0, 0, 0], [1.0, 0, 0]]),
    ]
    for f in calls:
        f()
        live1, _ = s.device_bytes()
        f()
        live2, peak = s.device_bytes()
        assert live2 == live1 and peak >= live2 > 0
    # a call rejected after the context is set up leaves nothing behind
    live, _ = s.device_bytes()
    with pytest.raises(Exception):
        s.exterior_field(x[0], np.zeros((70000, 3)) + 5.0)
    assert s.device_bytes()[0] == live
    s.close()
