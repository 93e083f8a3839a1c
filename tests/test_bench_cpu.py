"""Host logic of the benchmark: the seeded workload generators are deterministic and produce
the sizes and parameter ranges the configurations state."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def dofs(npatch, m, p):
    n = 1 << m
    return 2 * npatch * (n + p - 1) ** 2


def test_serving_requests_deterministic_and_in_range():
    a, b = bench.serving_requests(32), bench.serving_requests(32)
    assert len(a) == 32
    t = [r["t"] for r in a]
    assert all(t1 < t2 for t1, t2 in zip(t, t[1:]))
    for ra, rb in zip(a, b):
        assert ra["t"] == rb["t"] and ra["opt"] == rb["opt"] and np.array_equal(ra["dirs"], rb["dirs"])
        o = ra["opt"]
        assert 1 <= o["p"] <= 3 and 1.0 <= o["kappa"] <= 30.0 and o["q"] == 6 and o["precision"] == 1
        assert 1000 <= dofs(len(ra["geo"]), o["level_m"], o["p"]) <= 30000
        assert 1 <= len(ra["dirs"]) <= 16
        d = ra["dirs"]
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
        assert np.allclose(np.sum(d * ra["pols"], axis=1), 0.0, atol=1e-12)
    # mean arrival rate near 50 per second
    assert 0.3 < t[-1] < 1.5


def test_batch_requests_deterministic_and_in_range():
    a, b = bench.batch_requests(256), bench.batch_requests(256)
    assert len(a) == 256
    kinds = set()
    for ra, rb in zip(a, b):
        assert ra["opt"] == rb["opt"] and np.array_equal(ra["dirs"], rb["dirs"])
        o = ra["opt"]
        assert o["p"] in (1, 2) and 2 <= o["level_m"] <= 5 and 1.0 <= o["kappa"] <= 15.0 and o["q"] == 6
        kinds.add(len(ra["geo"]))
        assert len(ra["dirs"]) == 1
    assert kinds == {6, 16}


def test_multi_workload_size():
    w = bench.MULTI
    assert dofs(16, w["level_m"], w["p"]) == 139392
    assert w["rhs"] == 64 and (w["q"] + 1) ** 2 == 121


def test_far_directions_are_unit_vectors():
    d = bench.far_dirs(64)
    assert d.shape == (64, 3) and np.allclose(np.linalg.norm(d, axis=1), 1.0)
