"""Parity at the benchmark's full size (6-patch sphere, p = 2, 32 x 32 elements per patch,
kappa = 10, q = 8, eta = 1.6) on sampled outputs: the oracle computes single superspace rows
(near blocks integrated on demand, far field from direct moments)."""
import numpy as np
import pytest

import oracle as O
from workloads import geometry as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    from paper_1807_03097_gb300 import Solver

    geo = G.sphere()
    kw = dict(p=2, level_m=5, kappa=10.0, q=8, eta=1.6)
    s64 = Solver(geo, m2l_store=2, **kw)
    s32 = Solver(geo, precision=1, m2l_store=2, **kw)
    s32e = Solver(geo, precision=1, m2l_store=1, **kw)
    r = O.Problem(geo, p=2, m=5, kappa=10.0, q=8, eta=1.6)
    yield s64, s32, s32e, r
    s64.close()
    s32.close()
    s32e.close()


def test_fullsize_counts(big):
    s64, s32, s32e, r = big
    assert s64.ndof == r.ndof == 2 * 6 * (32 + 2 - 1) ** 2 == 13068
    far, near = s64.blocks()
    assert len(far) == len(r.far_pairs()) and len(near) == len(r.near_pairs())
    assert sorted(map(tuple, near)) == sorted(map(tuple, r.near_pairs()))


def test_fullsize_sampled_rows(big):
    s64, s32, s32e, r = big
    rng = np.random.default_rng(42)
    xs = rng.standard_normal(s64.nsup) + 1j * rng.standard_normal(s64.nsup)
    y64 = s64.matvec_superspace(xs).reshape(-1, s64.nb if hasattr(s64, "nb") else 18)
    y32 = s32.matvec_superspace(xs).reshape(y64.shape)
    y32e = s32e.matvec_superspace(xs).reshape(y64.shape)
    # corner elements of two patches, an edge element, interior elements
    n2 = 32 * 32
    elems = np.array([0, 5, n2 - 1, 3 * n2 + 517, 5 * n2 + 1000])
    rows = r.fmm_rows(xs, elems)
    scale = np.abs(rows).max()
    assert np.abs(y64[elems] - rows).max() / scale < 1e-11
    assert np.abs(y32[elems] - rows).max() / scale < 1e-5
    assert np.abs(y32e[elems] - rows).max() / scale < 1e-5
