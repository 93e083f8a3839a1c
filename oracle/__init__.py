"""Python access to the FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It builds ``efie_oracle.c`` with gcc and calls it through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "efie_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
_lib = None


def build(openmp: bool = True) -> str:
    """Compile the oracle into oracle/_build/liborc.so (plain C, any architecture)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-o", _LIB, _SRC, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        build()
    L = ctypes.CDLL(_LIB)
    P, D, I = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    c_int, c_double = ctypes.c_int, ctypes.c_double
    sig = {
        "orc_create": (P, [c_int, I, I, D, D, D, c_int, c_int, c_double, c_int, c_double, c_int, c_int]),
        "orc_create_variant": (P, [c_int, I, I, D, D, D, c_int, c_int, c_double, c_int, c_double, c_int, c_int,
                                   c_int]),
        "orc_destroy": (None, [P]),
        "orc_status": (c_int, [P, ctypes.c_char_p, c_int]),
        "orc_num_dofs": (c_int, [P]),
        "orc_num_elements": (c_int, [P]),
        "orc_superspace_size": (c_int, [P]),
        "orc_num_clusters": (c_int, [P]),
        "orc_eval_patch": (None, [P, c_int, c_int, D, D, D, D]),
        "orc_T_coo": (c_int, [P, c_int, I, I, D]),
        "orc_cluster_balls": (None, [P, D]),
        "orc_num_far": (c_int, [P]),
        "orc_num_near": (c_int, [P]),
        "orc_far_pairs": (None, [P, I]),
        "orc_near_pairs": (None, [P, I]),
        "orc_near_blocks": (None, [P, D]),
        "orc_pair_block": (None, [P, c_int, c_int, c_int, c_int, D]),
        "orc_pair_scalar": (None, [P, c_int, c_int, c_int, c_int, c_double, D]),
        "orc_pair_kind": (c_int, [P, c_int, c_int]),
        "orc_dense_superspace": (None, [P, D]),
        "orc_dense_matvec": (None, [P, c_int, D, D]),
        "orc_fmm_matvec": (None, [P, c_int, D, D]),
        "orc_fmm_matvec_superspace": (None, [P, D, D]),
        "orc_fmm_rows": (None, [P, D, c_int, I, D]),
        "orc_fmm_rows_far": (None, [P, D, c_int, I, D]),
        "orc_rhs": (None, [P, D, D, D]),
        "orc_gmres": (c_int, [P, c_int, D, D, c_int, c_double, c_int, I, D]),
        "orc_far_field": (None, [P, D, c_int, D, D]),
        "orc_div_integral": (None, [P, D, D]),
        "orc_area": (c_double, [P]),
        "orc_mie_l2": (None, [P, D, c_double, D]),
        "orc_mie_field": (None, [c_double, c_double, c_int, c_int, D, D]),
        "orc_dipole_field": (None, [c_double, D, D, c_int, D, D]),
        "orc_rhs_dipole": (None, [P, D, D, D]),
        "orc_exterior_field": (None, [P, D, c_int, D, D]),
        "orc_gauss01": (None, [c_int, D, D]),
        "orc_cheb01": (None, [c_int, D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _cz(a):
    """complex128 array -> contiguous complex128 (interleaved doubles)"""
    return np.ascontiguousarray(a, dtype=np.complex128)


def gauss01(g):
    L = _load()
    x, w = np.zeros(g), np.zeros(g)
    L.orc_gauss01(g, _d(x), _d(w))
    return x, w


def cheb01(q):
    L = _load()
    x = np.zeros(q + 1)
    L.orc_cheb01(q, _d(x))
    return x


def mie_field(kappa, radius, which, pts):
    """which: 0 incident E, 1 scattered E, 2 curl E_total, 3 surface current n x curl E_tot."""
    L = _load()
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((pts.shape[0], 3), dtype=np.complex128)
    L.orc_mie_field(kappa, radius, which, pts.shape[0], _d(pts), _d(out.view(np.float64)))
    return out


def dipole_field(kappa, x0, p0, pts):
    """Hertz dipole DP_{x0,p0} (Sec. 5.2) at points [n][3] -> [n][3] complex."""
    L = _load()
    x0 = np.ascontiguousarray(x0, float)
    p0 = np.ascontiguousarray(p0, float)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((pts.shape[0], 3), dtype=np.complex128)
    L.orc_dipole_field(kappa, _d(x0), _d(p0), pts.shape[0], _d(pts), _d(out.view(np.float64)))
    return out


class Problem:
    """One discretised EFIE problem in the oracle."""

    def __init__(self, patches, p, m, kappa, q, eta, g_reg=None, g_sing=None, leaf_dense=False):
        from workloads.geometry import flatten

        L = _load()
        self._L = L
        deg, ncp, knots, cp, w = flatten(patches)
        self._keep = (deg, ncp, knots, cp, w)
        self.p, self.m, self.kappa, self.q, self.eta = p, m, kappa, q, eta
        self.g_reg = g_reg if g_reg is not None else p + 4
        self.g_sing = g_sing if g_sing is not None else p + 4
        self.h = L.orc_create_variant(len(patches), _i(deg), _i(ncp), _d(knots), _d(cp), _d(w), p, m, kappa, q,
                                      eta, self.g_reg, self.g_sing, int(bool(leaf_dense)))
        if not self.h:
            raise MemoryError("oracle allocation failed")
        buf = ctypes.create_string_buffer(256)
        st = L.orc_status(self.h, buf, 256)
        if st != 0:
            msg = buf.value.decode()
            L.orc_destroy(self.h)
            self.h = None
            raise ValueError(f"oracle geometry error {st}: {msg}")
        self.ndof = L.orc_num_dofs(self.h)
        self.nE = L.orc_num_elements(self.h)
        self.nsup = L.orc_superspace_size(self.h)
        self.ncl = L.orc_num_clusters(self.h)
        self.nb = 2 * (p + 1) ** 2

    def __del__(self):
        if getattr(self, "h", None):
            self._L.orc_destroy(self.h)
            self.h = None

    # ---- geometry / space ----
    def eval_patch(self, patch, s):
        s = np.ascontiguousarray(s, dtype=np.float64).reshape(-1, 2)
        x, d1, d2 = (np.zeros((s.shape[0], 3)) for _ in range(3))
        self._L.orc_eval_patch(self.h, patch, s.shape[0], _d(s), _d(x), _d(d1), _d(d2))
        return x, d1, d2

    def T(self):
        n = self._L.orc_T_coo(self.h, 0, None, None, None)
        r, c, v = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n)
        self._L.orc_T_coo(self.h, n, _i(r), _i(c), _d(v))
        return r, c, v

    def balls(self):
        out = np.zeros((self.ncl, 4))
        self._L.orc_cluster_balls(self.h, _d(out))
        return out

    def far_pairs(self):
        n = self._L.orc_num_far(self.h)
        out = np.zeros((n, 3), np.int32)
        if n:
            self._L.orc_far_pairs(self.h, _i(out))
        return out

    def near_pairs(self):
        n = self._L.orc_num_near(self.h)
        out = np.zeros((n, 2), np.int32)
        if n:
            self._L.orc_near_pairs(self.h, _i(out))
        return out

    def near_blocks(self):
        n = self._L.orc_num_near(self.h)
        out = np.zeros((n, self.nb, self.nb), np.complex128)
        self._L.orc_near_blocks(self.h, _d(out.view(np.float64)))
        return out

    def pair_block(self, e, e2, g_reg=None, g_sing=None):
        out = np.zeros((self.nb, self.nb), np.complex128)
        self._L.orc_pair_block(self.h, e, e2, g_reg or self.g_reg, g_sing or self.g_sing, _d(out.view(np.float64)))
        return out

    def pair_scalar(self, e, e2, g_reg, g_sing, kappa):
        out = np.zeros(2)
        self._L.orc_pair_scalar(self.h, e, e2, g_reg, g_sing, kappa, _d(out))
        return complex(out[0], out[1])

    def pair_kind(self, e, e2):
        return self._L.orc_pair_kind(self.h, e, e2)

    # ---- operators ----
    def dense_superspace(self):
        out = np.zeros((self.nsup, self.nsup), np.complex128)
        self._L.orc_dense_superspace(self.h, _d(out.view(np.float64)))
        return out

    def dense_matvec(self, x):
        x = _cz(x).reshape(-1, self.ndof)
        y = np.zeros_like(x)
        self._L.orc_dense_matvec(self.h, x.shape[0], _d(x.view(np.float64)), _d(y.view(np.float64)))
        return y

    def fmm_matvec(self, x):
        x = _cz(x).reshape(-1, self.ndof)
        y = np.zeros_like(x)
        self._L.orc_fmm_matvec(self.h, x.shape[0], _d(x.view(np.float64)), _d(y.view(np.float64)))
        return y

    def fmm_matvec_superspace(self, xs):
        xs = _cz(xs).reshape(self.nsup)
        ys = np.zeros_like(xs)
        self._L.orc_fmm_matvec_superspace(self.h, _d(xs.view(np.float64)), _d(ys.view(np.float64)))
        return ys

    def fmm_rows(self, xs, elems):
        xs = _cz(xs).reshape(self.nsup)
        elems = np.ascontiguousarray(elems, np.int32)
        out = np.zeros((len(elems), self.nb), np.complex128)
        self._L.orc_fmm_rows(self.h, _d(xs.view(np.float64)), len(elems), _i(elems), _d(out.view(np.float64)))
        return out

    def fmm_rows_far(self, xs, elems):
        """Far-field part of fmm_rows (no near blocks)."""
        xs = _cz(xs).reshape(self.nsup)
        elems = np.ascontiguousarray(elems, np.int32)
        out = np.zeros((len(elems), self.nb), np.complex128)
        self._L.orc_fmm_rows_far(self.h, _d(xs.view(np.float64)), len(elems), _i(elems), _d(out.view(np.float64)))
        return out

    def rhs(self, d, pol):
        d = np.ascontiguousarray(d, float)
        pol = np.ascontiguousarray(pol, float)
        g = np.zeros(self.ndof, np.complex128)
        self._L.orc_rhs(self.h, _d(d), _d(pol), _d(g.view(np.float64)))
        return g

    def gmres(self, b, use_fmm=True, restart=1500, tol=1e-8, maxit=5000):
        b = _cz(b)
        x = np.zeros_like(b)
        its = np.zeros(1, np.int32)
        res = np.zeros(1)
        rc = self._L.orc_gmres(self.h, int(use_fmm), _d(b.view(np.float64)), _d(x.view(np.float64)), restart, tol,
                               maxit, _i(its), _d(res))
        return x, int(its[0]), float(res[0]), rc

    def far_field(self, coef, dirs):
        coef = _cz(coef)
        dirs = np.ascontiguousarray(dirs, float).reshape(-1, 3)
        out = np.zeros((dirs.shape[0], 3), np.complex128)
        self._L.orc_far_field(self.h, _d(coef.view(np.float64)), dirs.shape[0], _d(dirs), _d(out.view(np.float64)))
        return out

    def rhs_dipole(self, x0, p0):
        x0 = np.ascontiguousarray(x0, float)
        p0 = np.ascontiguousarray(p0, float)
        g = np.zeros(self.ndof, np.complex128)
        self._L.orc_rhs_dipole(self.h, _d(x0), _d(p0), _d(g.view(np.float64)))
        return g

    def exterior_field(self, coef, pts):
        coef = _cz(coef)
        pts = np.ascontiguousarray(pts, float).reshape(-1, 3)
        out = np.zeros((pts.shape[0], 3), np.complex128)
        self._L.orc_exterior_field(self.h, _d(coef.view(np.float64)), pts.shape[0], _d(pts), _d(out.view(np.float64)))
        return out

    def div_integral(self, coef):
        coef = _cz(coef)
        out = np.zeros(2)
        self._L.orc_div_integral(self.h, _d(coef.view(np.float64)), _d(out))
        return complex(out[0], out[1])

    def area(self):
        return self._L.orc_area(self.h)

    def mie_l2(self, coef, radius=1.0):
        coef = _cz(coef)
        out = np.zeros(2)
        self._L.orc_mie_l2(self.h, _d(coef.view(np.float64)), radius, _d(out))
        return out[0], out[1]
