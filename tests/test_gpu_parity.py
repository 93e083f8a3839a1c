"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: FP64 path 1e-11 relative (max-norm over the vector) for the matrix-vector
product, the near-field blocks, the right-hand side and the far field; the two codes share
the quadrature rules and differ only in the order of rounding.  Mixed precision: 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from workloads import geometry as G

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32 = 1e-5

CASES = {
    # name: (patches, p, m, kappa, q, eta)
    "sphere_p1_m2_q4": (G.sphere, 1, 2, 1.0, 4, 1.6),     # the small sphere workload, full size
    "sphere_p2_m1_q6": (G.sphere, 2, 1, 3.0, 6, 1.6),
    "torus_p2_m1_q5": (G.torus, 2, 1, 2.0, 5, 1.6),
    "cube_p3_m1_q3": (G.cube, 3, 1, 1.5, 3, 1.2),
    "sphere_p1_m0_q2": (G.sphere, 1, 0, 1.0, 2, 1.6),     # degenerate: one element per patch, no far field
}


def relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module", params=[(c, st) for c in CASES for st in (1, 2)],
                ids=[f"{c}-{'evaluated' if st == 1 else 'stored'}" for c in CASES for st in (1, 2)])
def pair(request):
    """The FP64 library with M2L coupling matrices evaluated in every product (m2l_store=1)
    or kept in device memory (m2l_store=2), and the oracle."""
    from paper_1807_03097_gb300 import Solver

    name, store = request.param
    mk, p, m, k, q, eta = CASES[name]
    geo = mk()
    s = Solver(geo, p=p, level_m=m, kappa=k, q=q, eta=eta, m2l_store=store)
    r = O.Problem(geo, p=p, m=m, kappa=k, q=q, eta=eta)
    yield name, s, r
    s.close()


def test_dofs_and_block_lists_identical(pair):
    name, s, r = pair
    assert s.ndof == r.ndof
    far, near = s.blocks()
    assert sorted(map(tuple, far)) == sorted(map(tuple, r.far_pairs()))
    assert sorted(map(tuple, near)) == sorted(map(tuple, r.near_pairs()))


def test_near_field_blocks(pair):
    name, s, r = pair
    far, near = s.blocks()
    bs = s.near_blocks()
    br = r.near_blocks()
    idx = {tuple(x): i for i, x in enumerate(r.near_pairs())}
    perm = [idx[tuple(x)] for x in near]
    assert relmax(bs, br[perm]) < TOL64


def test_matvec_fp64(pair):
    name, s, r = pair
    rng = np.random.default_rng(7)
    x = rng.standard_normal((2, s.ndof)) + 1j * rng.standard_normal((2, s.ndof))
    y = s.matvec(x)
    yr = r.fmm_matvec(x)
    for k in range(2):
        assert relmax(y[k], yr[k]) < TOL64, (name, relmax(y[k], yr[k]))


def test_matvec_superspace_fp64(pair):
    name, s, r = pair
    rng = np.random.default_rng(8)
    xs = rng.standard_normal(s.nsup) + 1j * rng.standard_normal(s.nsup)
    assert relmax(s.matvec_superspace(xs), r.fmm_matvec_superspace(xs)) < TOL64


def test_rhs_and_far_field(pair):
    name, s, r = pair
    d = np.array([0.0, 0.6, 0.8])
    pol = np.array([1.0, 0.0, 0.0])
    g = s.rhs(d, pol)[0]
    assert relmax(g, r.rhs(d, pol)) < TOL64
    rng = np.random.default_rng(9)
    w = rng.standard_normal(s.ndof) + 1j * rng.standard_normal(s.ndof)
    dirs = rng.standard_normal((5, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    assert relmax(s.far_field(w, dirs)[0], r.far_field(w, dirs)) < TOL64


def test_device_pointers_match_host_pointers(pair):
    torch = pytest.importorskip("torch")
    name, s, r = pair
    rng = np.random.default_rng(10)
    x = rng.standard_normal(s.ndof) + 1j * rng.standard_normal(s.ndof)
    yh = s.matvec(x)
    xd = torch.from_numpy(x).cuda()
    yd = s.matvec(xd)
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), yh)


@pytest.mark.parametrize("store", [1, 2], ids=["evaluated", "stored"])
def test_mixed_precision_matvec(store):
    from paper_1807_03097_gb300 import Solver

    for mk, p, m, k, q in [(G.sphere, 1, 2, 1.0, 4), (G.torus, 2, 1, 2.0, 5)]:
        geo = mk()
        s = Solver(geo, p=p, level_m=m, kappa=k, q=q, eta=1.6, precision=1, m2l_store=store)
        r = O.Problem(geo, p=p, m=m, kappa=k, q=q, eta=1.6)
        rng = np.random.default_rng(3)
        x = rng.standard_normal(s.ndof) + 1j * rng.standard_normal(s.ndof)
        e = np.linalg.norm(s.matvec(x) - r.fmm_matvec(x)[0]) / np.linalg.norm(r.fmm_matvec(x)[0])
        assert e < TOL32, e
        s.close()


def near_product_oracle(r, xs):
    """ys[a] = sum over the near pairs (a, b) of B_ab xs[b], from the oracle's element blocks."""
    X = xs.reshape(r.nE, r.nb)
    Y = np.zeros_like(X)
    for (a, b), B in zip(r.near_pairs(), r.near_blocks()):
        Y[a] += B @ X[b]
    return Y.reshape(-1)


def test_near_apply_fp64(pair):
    name, s, r = pair
    rng = np.random.default_rng(11)
    xs = rng.standard_normal(s.nsup) + 1j * rng.standard_normal(s.nsup)
    assert relmax(s.near_apply(xs), near_product_oracle(r, xs)) < TOL64


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_near_apply_mixed(p):
    """FP32 blocks (one kernel per block size 2(p+1)^2 = 8, 18, 32, 50), FP32 copy of x*,
    compensated FP32 sums; against the FP64 oracle blocks, and device pointers against host
    pointers bit for bit."""
    torch = pytest.importorskip("torch")
    from paper_1807_03097_gb300 import Solver

    geo = G.torus()
    kw = dict(p=p, m=2 if p < 4 else 1, kappa=2.0, q=4, eta=1.6)
    s = Solver(geo, p=p, level_m=kw["m"], kappa=2.0, q=4, eta=1.6, precision=1)
    r = O.Problem(geo, **kw)
    rng = np.random.default_rng(12 + p)
    xs = rng.standard_normal(s.nsup) + 1j * rng.standard_normal(s.nsup)
    yh = s.near_apply(xs)
    assert relmax(yh, near_product_oracle(r, xs)) < TOL32
    yd = s.near_apply(torch.from_numpy(xs).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), yh)
    assert s.last_timings()["near"] > 0
    s.close()
