"""Serving loop (efie_server_*): continuous admission of scattering requests of different
geometries, sizes and wavenumbers; each result must be the same whether the request runs
alone or among others (every reduction has a fixed order, so the results are bitwise equal)."""
import numpy as np
import pytest

from workloads import geometry as G

pytestmark = pytest.mark.gpu

REQUESTS = [
    (G.sphere, dict(p=1, level_m=2, kappa=1.0, q=4, eta=1.6)),
    (G.torus, dict(p=2, level_m=1, kappa=2.0, q=5, eta=1.6, precision=1)),
    (G.cube, dict(p=1, level_m=2, kappa=1.5, q=4, eta=1.6)),
    (G.sphere, dict(p=2, level_m=2, kappa=3.0, q=5, eta=1.6, precision=1)),
    (G.sphere, dict(p=1, level_m=3, kappa=2.0, q=4, eta=1.6, precision=1)),
    (G.torus, dict(p=1, level_m=2, kappa=1.0, q=4, eta=1.6)),
    # tori at p = 3 have the most near-field blocks per element of the serving mix (the
    # admission estimate must still bound their device peak)
    (G.torus, dict(p=3, level_m=2, kappa=11.7, q=6, eta=1.6, precision=1)),
    (G.torus, dict(p=3, level_m=3, kappa=8.0, q=6, eta=1.6, precision=1)),
]


def run_requests(srv, reqs, first=0):
    """Submit all requests at once (request k uses seed k for its plane waves) and wait."""
    tickets = []
    for k, (mk, opt) in enumerate(reqs):
        rng = np.random.default_rng(first + k)
        d = rng.standard_normal((2, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pol = np.cross(d, [0.3, 0.5, 0.8])
        pol /= np.linalg.norm(pol, axis=1, keepdims=True)
        ff = np.array([[0, 0, 1.0], [1.0, 0, 0]])
        tol = 1e-5 if opt.get("precision", 0) == 1 else 1e-8   # mixed form served at 1e-5
        tickets.append(srv.submit(mk(), d, pol, ff, gmres_tol=tol, gmres_maxit=3000, **opt))
    return [srv.wait(t) for t in tickets]


def test_alone_and_in_the_mix_are_identical():
    from paper_1807_03097_gb300.efie import Server

    mixed = Server(hbm_budget_bytes=40 << 30, max_slots=4)
    res_mix = run_requests(mixed, REQUESTS)
    mixed.close()
    # every request alone in a single-slot server, with the same seeded plane waves
    for k in range(len(REQUESTS)):
        srv = Server(hbm_budget_bytes=40 << 30, max_slots=1)
        out = run_requests(srv, [REQUESTS[k]], first=k)[0]
        srv.close()
        r, w, e = out
        rm, wm, em = res_mix[k]
        assert r.status == 0 and rm.status == 0
        assert r.iterations == rm.iterations
        assert np.array_equal(w, wm), k
        assert np.array_equal(e, em), k
        tol = 1e-5 if REQUESTS[k][1].get("precision", 0) == 1 else 1e-8
        assert rm.residual <= tol * 1.05
        assert rm.latency_ms >= rm.queue_ms >= 0.0
        # the admission's estimate covers what the request's context really held
        assert 0 < rm.device_peak_bytes <= rm.footprint_bytes, (k, rm.device_peak_bytes, rm.footprint_bytes)


def test_served_results_solve_the_oracle_system():
    """One served request per geometry, checked against the FP64 oracle (Sec. 4.2 operator,
    eq. linsys right-hand side): the true relative residual of each returned current, with the
    oracle's operator, is within the served tolerance plus the mixed form's operator error; the
    served far field equals the oracle's far field of the returned current."""
    import oracle as O
    from paper_1807_03097_gb300.efie import Server

    cases = [REQUESTS[0], REQUESTS[1], REQUESTS[2]]  # sphere (FP64), torus (mixed), cube (FP64)
    srv = Server(hbm_budget_bytes=40 << 30, max_slots=3)
    out = run_requests(srv, cases, first=100)
    srv.close()
    for k, (mk, opt) in enumerate(cases):
        r, w, e = out[k]
        assert r.status == 0
        rng = np.random.default_rng(100 + k)
        d = rng.standard_normal((2, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pol = np.cross(d, [0.3, 0.5, 0.8])
        pol /= np.linalg.norm(pol, axis=1, keepdims=True)
        ref = O.Problem(mk(), p=opt["p"], m=opt["level_m"], kappa=opt["kappa"], q=opt["q"], eta=opt["eta"])
        tol = 1e-5 if opt.get("precision", 0) == 1 else 1e-8
        ff = np.array([[0, 0, 1.0], [1.0, 0, 0]])
        for i in range(2):
            b = ref.rhs(d[i], pol[i])
            res = np.linalg.norm(b - ref.fmm_matvec(w[i])[0]) / np.linalg.norm(b)
            assert res < 2 * tol, (k, i, res)
            e_ref = ref.far_field(w[i], ff)
            assert np.abs(e[i] - e_ref).max() < 1e-11 * np.abs(e_ref).max(), (k, i)


def test_tight_budget_serialises_and_errors_are_reported():
    from paper_1807_03097_gb300.efie import Server

    srv = Server(hbm_budget_bytes=1, max_slots=3)   # every request exceeds the budget: one at a time
    t_ok = srv.submit(G.sphere(), [[0, 0, 1.0]], [[1.0, 0, 0]], None, p=1, level_m=1, kappa=1.0, q=3, eta=1.6)
    t_bad = srv.submit(G.cube()[:5], [[0, 0, 1.0]], [[1.0, 0, 0]], None, p=1, level_m=1, kappa=1.0, q=3, eta=1.6)
    r_ok, w, _ = srv.wait(t_ok)
    r_bad, _, _ = srv.wait(t_bad)
    assert r_ok.status == 0 and np.abs(w).max() > 0
    assert r_bad.status == -3          # open surface
    with pytest.raises(Exception, match="-1"):
        srv.poll(t_ok + 1000)            # unknown ticket
    srv.close()
