"""The tensor-core M2L (split TF32, FP32 accumulation) at the far-list lengths of the 139k-DOF
torus workload: torus R = 2, r = 0.5 (16 patches), p = 3, 32 x 32 elements per patch, kappa =
20, q = 10 (121 interpolation nodes, the tile of that workload), eta = 1.6, 16 right-hand
sides in one batched product (and 40: three blocks of 64 fields, the last one ragged).  Sampled
superspace rows of every right-hand side are compared
with the FP64 oracle element by element (max-norm relative, 1e-5): the far part from
oracle.fmm_rows_far (direct moments, far field of the blocks whose target cluster contains the
element) and the near part from the oracle's element blocks, which are pinned to equal
oracle.fmm_rows in the CPU tests."""
import numpy as np
import pytest

import oracle as O
from workloads import geometry as G

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
KW = dict(p=3, level_m=5, kappa=20.0, q=10, eta=1.6)


@pytest.fixture(scope="module")
def torus():
    from paper_1807_03097_gb300 import Solver

    geo = G.torus(R=2.0, r=0.5)
    s = Solver(geo, precision=1, m2l_batch=2, **KW)
    r = O.Problem(geo, p=KW["p"], m=KW["level_m"], kappa=KW["kappa"], q=KW["q"], eta=KW["eta"])
    yield s, r
    s.close()


@pytest.mark.parametrize("R", [16, 40])
def test_tensor_core_batched_rows_vs_oracle(torus, R):
    """16 right-hand sides: one block of 64 fields per target cluster; 40: 160 fields, two full
    blocks and a ragged one of 32."""
    s, r = torus
    assert s.nfar == len(r.far_pairs()) and s.nsup == r.nsup
    # far lists as long as in the 139k-DOF workload: tens of admissible sources per cluster
    far = r.far_pairs()
    per_target = np.bincount(far[:, 1])
    assert per_target.max() >= 100
    rng = np.random.default_rng(77 + R)
    xs = rng.standard_normal((R, s.nsup)) + 1j * rng.standard_normal((R, s.nsup))
    ys = s.matvec_superspace(xs).reshape(R, r.nE, r.nb)
    n2 = 32 * 32
    elems = np.array([0, n2 - 1, 5 * n2 + 517, 11 * n2 + 31])
    near = r.near_pairs()
    blocks = {}
    for e in elems:
        for a, b in near:
            if a == e:
                blocks[(int(a), int(b))] = r.pair_block(int(a), int(b))
    for i in range(R):
        X = xs[i].reshape(r.nE, r.nb)
        rows = r.fmm_rows_far(xs[i], elems)
        for k, e in enumerate(elems):
            for (a, b), B in blocks.items():
                if a == e:
                    rows[k] += B @ X[b]
        scale = np.abs(rows).max()
        err = np.abs(ys[i][elems] - rows).max() / scale
        assert err < TOL32, (i, err)


@pytest.mark.parametrize("R", [5, 36])
def test_tensor_core_matches_cuda_core_batched_product(torus, R):
    """The same batched product with the M2L on the CUDA cores (FP32, compensated sums), on all
    rows: the two mixed forms agree within the mixed tolerance (5 right-hand sides: one ragged
    block of 20 fields; 36: two full blocks of 64 fields and a ragged one of 16)."""
    s, r = torus
    from paper_1807_03097_gb300 import Solver

    s1 = Solver(G.torus(R=2.0, r=0.5), precision=1, m2l_batch=1, **KW)
    rng = np.random.default_rng(78 + R)
    xs = rng.standard_normal((R, s.nsup)) + 1j * rng.standard_normal((R, s.nsup))
    y_tc = s.matvec_superspace(xs)
    y_cc = s1.matvec_superspace(xs)
    s1.close()
    for i in range(R):
        assert np.linalg.norm(y_tc[i] - y_cc[i]) / np.linalg.norm(y_cc[i]) < TOL32
