"""Host-side checks of the C-ABI library (no GPU needed, no compute calls)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "efie.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1807_03097_gb300 import build, efie

    if not os.path.exists(efie.LIB_PATH):
        build.build()
    return efie.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(efie_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib):
    from paper_1807_03097_gb300 import efie

    names = declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(efie.ABI_SYMBOLS) == names


def test_default_options_and_status_strings(lib):
    from paper_1807_03097_gb300 import efie

    o = efie.options()
    assert (o.p, o.level_m, o.q, o.gmres_restart, o.tol_is_relative) == (1, 2, 4, 1500, 1)
    assert abs(o.eta - 1.6) < 1e-15 and abs(o.gmres_tol - 1e-8) < 1e-20
    for s in (0, 1, -1, -2, -3, -4, -5, -6):
        assert lib.efie_status_string(s)
    assert lib.efie_status_string(-99) == b"unknown status"


def test_invalid_arguments_rejected_before_any_device_work(lib):
    from paper_1807_03097_gb300 import efie

    assert lib.efie_create(None, None, None) == -1
    h = ctypes.c_void_p()
    for bad in (dict(p=0), dict(p=5), dict(q=0), dict(q=40), dict(kappa=0.0), dict(kappa=-1.0), dict(eta=0.0),
                dict(level_m=11), dict(precision=7), dict(gmres_restart=0), dict(gmres_tol=0.0)):
        o = efie.options(**bad)
        assert lib.efie_create(ctypes.byref(h), ctypes.byref(o), None) == -1, bad
    assert lib.efie_default_options(None) == -1
    assert lib.efie_destroy(None) == 0
    assert lib.efie_setup(None) == -1
    assert lib.efie_matvec(None, 1, None, None, 0) == -1
    assert lib.efie_check_device_waits(None, 1000) == -1
    assert lib.efie_exterior_field(None, 1, None, 1, None, None, 0) == -1
    assert lib.efie_rhs_dipole(None, 1, None, None, None, 0) == -1
    assert lib.efie_far_field_noalloc(None, None, 1, None, None) == -1
    assert lib.efie_solve(None, 1, None, None, 0, None) == -1
    assert lib.efie_solve_plane_waves(None, 1, None, None, None, 0, None) == -1
    assert lib.efie_rhs_plane_waves(None, 1, None, None, None, 0) == -1
    assert lib.efie_far_field(None, 1, None, 1, None, None, 0) == -1
    assert lib.efie_server_submit(None, None, None) == -1
    assert lib.efie_server_poll(None, 0, None) == -1
    assert lib.efie_server_destroy(None) == 0
    assert lib.efie_launch_count(None) == -1
    assert lib.efie_last_error(None) == b""
    # near-field product alone, batched superspace product, setup timings, device bytes
    assert lib.efie_near_apply(None, None, None, 0) == -1
    assert lib.efie_matvec_superspace_batch(None, 1, None, None, 0) == -1
    assert lib.efie_setup_timings(None, None, 0) == 0
    assert lib.efie_device_bytes(None, None, None) == -1
    # groups of problems
    g = ctypes.c_void_p()
    assert lib.efie_group_create(None, None, 1) == -1
    assert lib.efie_group_create(ctypes.byref(g), None, 1) == -1
    arr = (ctypes.c_void_p * 1)(None)
    assert lib.efie_group_create(ctypes.byref(g), arr, 0) == -1
    assert lib.efie_group_create(ctypes.byref(g), arr, 1) == -1   # a null context
    assert lib.efie_group_solve(None, None, None, 0, None, None, None) == -1
    assert lib.efie_group_stats(None, None, 0) == 0
    assert lib.efie_group_destroy(None) == 0
    assert lib.efie_group_last_error(None) == b"null group"
    assert lib.efie_setup_many(None, 1, 1, None) == -1
    assert lib.efie_setup_many(arr, 1, 0, None) == -1
    for bad in (dict(m2l_store=3), dict(m2l_batch=3), dict(m2l_batch=2, q=11), dict(m2l_pairs=3), dict(leaf_dense=2)):
        o = efie.options(**bad)
        assert lib.efie_create(ctypes.byref(h), ctypes.byref(o), None) == -1, bad


def test_package_fails_loudly_without_library(tmp_path):
    from paper_1807_03097_gb300 import efie

    saved = efie._lib
    try:
        efie._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            efie.load(str(tmp_path / "missing.so"))
    finally:
        efie._lib = saved
