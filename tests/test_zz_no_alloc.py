"""efie_far_field_noalloc: the far field for callers that must not allocate device memory
during the call (fixed device-memory budget owned by another allocator, or no tolerance for
cudaMalloc / cudaFree synchronising the device).  Its result must match efie_far_field
within the FP64 tolerance of the other tests, on two calls in a row (the second call reuses
the shared scratch array that the first one left behind).  This file is collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


def test_far_field_noalloc_matches_far_field_twice():
    torch = pytest.importorskip("torch")
    from paper_1807_03097_gb300 import Solver
    from workloads import geometry as G

    s = Solver(G.sphere(), p=2, level_m=2, kappa=3.0, q=5, eta=1.6)
    rng = np.random.default_rng(17)
    for call in range(2):
        w = rng.standard_normal(s.ndof) + 1j * rng.standard_normal(s.ndof)
        ndir = 7 + 5 * call
        dirs = rng.standard_normal((ndir, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        ref = s.far_field(w, dirs)[0]
        wd = torch.from_numpy(w).cuda()
        dd = torch.from_numpy(dirs).cuda()
        out = torch.full((ndir, 3), complex("nan"), dtype=torch.complex128, device="cuda")
        s.far_field_noalloc(wd, dd, out)
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() / np.abs(ref).max() < TOL64, call
    # a request beyond the fixed scratch is rejected
    big = torch.zeros((200000, 3), dtype=torch.float64, device="cuda")
    big[:, 2] = 1.0
    res = torch.zeros((200000, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(Exception, match="-1"):
        s.far_field_noalloc(wd, big, res)
    s.close()
