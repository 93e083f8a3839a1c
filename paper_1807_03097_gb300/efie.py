"""Thin ctypes binding of the C ABI in include/efie.h (argument marshalling only).

Every numerical step runs in the CUDA library ``_build/libefie.so``; importing this module
without the compiled library raises, there is no CPU fallback.  Host arrays are numpy
complex128 / float64; device arrays are torch CUDA tensors (complex128), passed by pointer.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libefie.so")

EFIE_OK = 0
EFIE_NOT_CONVERGED = 1
EFIE_PENDING = 2
EFIE_FP64 = 0
EFIE_MIXED_FP32 = 1
EFIE_PTR_HOST = 0
EFIE_PTR_DEVICE = 1

# every symbol declared in include/efie.h
ABI_SYMBOLS = (
    "efie_default_options", "efie_create", "efie_set_geometry", "efie_setup", "efie_num_dofs",
    "efie_matvec", "efie_rhs_plane_waves", "efie_solve", "efie_solve_plane_waves", "efie_far_field",
    "efie_block_counts", "efie_export_blocks", "efie_export_near_blocks", "efie_matvec_superspace",
    "efie_matvec_superspace_batch", "efie_device_bytes", "efie_setup_timings", "efie_near_apply",
    "efie_last_timings", "efie_launch_count", "efie_destroy", "efie_status_string", "efie_last_error", "efie_check_device_waits", "efie_exterior_field",
    "efie_rhs_dipole",
    "efie_far_field_noalloc",
    "efie_server_create", "efie_server_submit", "efie_server_poll", "efie_server_destroy",
    "efie_setup_many", "efie_group_create", "efie_group_solve", "efie_group_stats", "efie_group_last_error",
    "efie_group_destroy",
)


class EfieOptions(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("level_m", ctypes.c_int), ("kappa", ctypes.c_double), ("q", ctypes.c_int),
                ("eta", ctypes.c_double), ("precision", ctypes.c_int), ("quad_regular", ctypes.c_int),
                ("quad_singular", ctypes.c_int), ("gmres_restart", ctypes.c_int), ("gmres_tol", ctypes.c_double),
                ("gmres_maxit", ctypes.c_int), ("tol_is_relative", ctypes.c_int), ("m2l_store", ctypes.c_int),
                ("m2l_batch", ctypes.c_int), ("leaf_dense", ctypes.c_int), ("m2l_pairs", ctypes.c_int)]


class EfieSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("residual", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double)]


class EfieRequest(ctypes.Structure):
    _fields_ = [("n_patches", ctypes.c_int), ("deg", ctypes.c_void_p), ("ncp", ctypes.c_void_p),
                ("knots", ctypes.c_void_p), ("cp", ctypes.c_void_p), ("w", ctypes.c_void_p), ("opt", EfieOptions),
                ("nrhs", ctypes.c_int), ("dir", ctypes.c_void_p), ("pol", ctypes.c_void_p), ("ndir", ctypes.c_int),
                ("ff_dirs", ctypes.c_void_p), ("w_out", ctypes.c_void_p), ("e_inf_out", ctypes.c_void_p)]


class EfieResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("residual", ctypes.c_double),
                ("ndof", ctypes.c_int64), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("footprint_bytes", ctypes.c_int64), ("device_peak_bytes", ctypes.c_int64)]


class EfieError(RuntimeError):
    def __init__(self, status, where, lib, handle=None):
        self.status = status
        msg = lib.efie_status_string(status).decode()
        detail = lib.efie_last_error(handle).decode() if handle else ""
        super().__init__(f"{where}: status {status} ({msg})" + (f": {detail}" if detail else ""))


_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    P, D, I, I64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), \
        ctypes.POINTER(ctypes.c_int64)
    c_int = ctypes.c_int
    sig = {
        "efie_default_options": (c_int, [ctypes.POINTER(EfieOptions)]),
        "efie_create": (c_int, [ctypes.POINTER(P), ctypes.POINTER(EfieOptions), P]),
        "efie_set_geometry": (c_int, [P, c_int, I, I, D, D, D]),
        "efie_setup": (c_int, [P]),
        "efie_num_dofs": (c_int, [P, I64]),
        "efie_matvec": (c_int, [P, c_int, P, P, c_int]),
        "efie_rhs_plane_waves": (c_int, [P, c_int, D, D, P, c_int]),
        "efie_solve": (c_int, [P, c_int, P, P, c_int, ctypes.POINTER(EfieSolveInfo)]),
        "efie_solve_plane_waves": (c_int, [P, c_int, D, D, P, c_int, ctypes.POINTER(EfieSolveInfo)]),
        "efie_far_field": (c_int, [P, c_int, P, c_int, D, P, c_int]),
        "efie_block_counts": (c_int, [P, I64, I64, I64, I64]),
        "efie_export_blocks": (c_int, [P, I, I]),
        "efie_export_near_blocks": (c_int, [P, D]),
        "efie_matvec_superspace": (c_int, [P, P, P, c_int]),
        "efie_matvec_superspace_batch": (c_int, [P, c_int, P, P, c_int]),
        "efie_device_bytes": (c_int, [P, I64, I64]),
        "efie_setup_timings": (c_int, [P, D, c_int]),
        "efie_near_apply": (c_int, [P, P, P, c_int]),
        "efie_last_timings": (c_int, [P, D, c_int]),
        "efie_launch_count": (ctypes.c_int64, [P]),
        "efie_far_field_noalloc": (c_int, [P, P, c_int, P, P]),
        "efie_server_create": (c_int, [ctypes.POINTER(P), ctypes.c_size_t, c_int]),
        "efie_server_submit": (c_int, [P, ctypes.POINTER(EfieRequest), ctypes.POINTER(ctypes.c_uint64)]),
        "efie_server_poll": (c_int, [P, ctypes.c_uint64, ctypes.POINTER(EfieResult)]),
        "efie_server_destroy": (c_int, [P]),
        "efie_destroy": (c_int, [P]),
        "efie_status_string": (ctypes.c_char_p, [c_int]),
        "efie_last_error": (ctypes.c_char_p, [P]),
        "efie_check_device_waits": (c_int, [P, ctypes.c_longlong]),
        "efie_exterior_field": (c_int, [P, c_int, P, c_int, P, P, c_int]),
        "efie_rhs_dipole": (c_int, [P, c_int, P, P, P, c_int]),
        "efie_setup_many": (c_int, [ctypes.POINTER(P), c_int, c_int, I]),
        "efie_group_create": (c_int, [ctypes.POINTER(P), ctypes.POINTER(P), c_int]),
        "efie_group_solve": (c_int, [P, ctypes.POINTER(P), ctypes.POINTER(P), c_int, I, D, I]),
        "efie_group_stats": (c_int, [P, D, c_int]),
        "efie_group_last_error": (ctypes.c_char_p, [P]),
        "efie_group_destroy": (c_int, [P]),
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


def _ptr(a):
    """(pointer, kind) of a numpy array (host) or a torch CUDA tensor (device)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data), EFIE_PTR_HOST
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), EFIE_PTR_DEVICE
    raise TypeError("expected a numpy array or a CUDA tensor")


def options(**kw) -> EfieOptions:
    L = load()
    o = EfieOptions()
    L.efie_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Solver:
    """One EFIE context: geometry + discretisation resident on the current CUDA device."""

    def __init__(self, patches=None, stream=None, **opts):
        self._L = load()
        self.opts = options(**opts)
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        self._check(self._L.efie_create(ctypes.byref(h), ctypes.byref(self.opts), st), "efie_create")
        self.h = h
        self.ndof = None
        if patches is not None:
            self.set_geometry(patches)
            self.setup()

    def _check(self, st, where):
        if st < 0:
            raise EfieError(st, where, self._L, getattr(self, "h", None))
        return st

    def close(self):
        if getattr(self, "h", None):
            self._L.efie_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, patches):
        from workloads.geometry import flatten

        deg, ncp, knots, cp, w = flatten(patches)
        self._check(self._L.efie_set_geometry(self.h, len(patches), _i(deg), _i(ncp), _d(knots), _d(cp), _d(w)),
                    "efie_set_geometry")

    def setup(self):
        self._check(self._L.efie_setup(self.h), "efie_setup")
        self._read_counts()

    def _read_counts(self):
        n = ctypes.c_int64()
        self._check(self._L.efie_num_dofs(self.h, ctypes.byref(n)), "efie_num_dofs")
        self.ndof = int(n.value)
        a, b, c, d = (ctypes.c_int64() for _ in range(4))
        self._check(self._L.efie_block_counts(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                              ctypes.byref(d)), "efie_block_counts")
        self.nfar, self.nnear, self.ncl, self.nsup = int(a.value), int(b.value), int(c.value), int(d.value)
        self.nb = 2 * (self.opts.p + 1) ** 2

    def matvec(self, x, out=None):
        """y = A x for x of shape (ndof,) or (nrhs, ndof); numpy (host) or CUDA tensor (device)."""
        nrhs = 1 if x.ndim == 1 else x.shape[0]
        if out is None:
            out = np.empty_like(x) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
        px, kx = _ptr(x)
        py, ky = _ptr(out)
        if kx != ky:
            raise ValueError("x and out must both be host or both be device arrays")
        self._check(self._L.efie_matvec(self.h, nrhs, px, py, kx), "efie_matvec")
        return out

    def matvec_superspace(self, xs, out=None):
        """ys = (N + F) xs for xs of shape (nsup,) or (nrhs, nsup) (several right-hand sides in
        one batched pass)."""
        if out is None:
            out = np.empty_like(xs) if isinstance(xs, np.ndarray) else xs.new_empty(xs.shape)
        px, kx = _ptr(xs)
        py, _ = _ptr(out)
        if xs.ndim == 2:
            self._check(self._L.efie_matvec_superspace_batch(self.h, xs.shape[0], px, py, kx),
                        "efie_matvec_superspace_batch")
        else:
            self._check(self._L.efie_matvec_superspace(self.h, px, py, kx), "efie_matvec_superspace")
        return out

    def near_apply(self, xs, out=None):
        """ys = N xs (the near-field blocks alone) on one superspace vector."""
        if out is None:
            out = np.empty_like(xs) if isinstance(xs, np.ndarray) else xs.new_empty(xs.shape)
        px, kx = _ptr(xs)
        py, _ = _ptr(out)
        self._check(self._L.efie_near_apply(self.h, px, py, kx), "efie_near_apply")
        return out

    def device_bytes(self):
        """(live, peak) bytes of device memory this context has allocated."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._L.efie_device_bytes(self.h, ctypes.byref(a), ctypes.byref(b)), "efie_device_bytes")
        return int(a.value), int(b.value)

    def rhs(self, dirs, pols, out=None):
        dirs = np.ascontiguousarray(dirs, float).reshape(-1, 3)
        pols = np.ascontiguousarray(pols, float).reshape(-1, 3)
        if out is None:
            out = np.zeros((dirs.shape[0], self.ndof), np.complex128)
        po, k = _ptr(out)
        self._check(self._L.efie_rhs_plane_waves(self.h, dirs.shape[0], _d(dirs), _d(pols), po, k),
                    "efie_rhs_plane_waves")
        return out

    def solve(self, b, out=None):
        nrhs = 1 if b.ndim == 1 else b.shape[0]
        if out is None:
            out = np.zeros_like(b) if isinstance(b, np.ndarray) else b.new_zeros(b.shape)
        pb, kb = _ptr(b)
        px, _ = _ptr(out)
        info = EfieSolveInfo()
        st = self._check(self._L.efie_solve(self.h, nrhs, pb, px, kb, ctypes.byref(info)), "efie_solve")
        return out, info, st

    def solve_plane_waves(self, dirs, pols, out=None):
        dirs = np.ascontiguousarray(dirs, float).reshape(-1, 3)
        pols = np.ascontiguousarray(pols, float).reshape(-1, 3)
        if out is None:
            out = np.zeros((dirs.shape[0], self.ndof), np.complex128)
        po, k = _ptr(out)
        info = EfieSolveInfo()
        st = self._check(self._L.efie_solve_plane_waves(self.h, dirs.shape[0], _d(dirs), _d(pols), po, k,
                                                        ctypes.byref(info)), "efie_solve_plane_waves")
        return out, info, st

    def far_field(self, w, dirs, out=None):
        dirs = np.ascontiguousarray(dirs, float).reshape(-1, 3)
        nrhs = 1 if w.ndim == 1 else w.shape[0]
        if out is None:
            out = np.zeros((nrhs, dirs.shape[0], 3), np.complex128) if isinstance(w, np.ndarray) else \
                w.new_zeros((nrhs, dirs.shape[0], 3))
        pw, kw = _ptr(w)
        po, _ = _ptr(out)
        self._check(self._L.efie_far_field(self.h, nrhs, pw, dirs.shape[0], _d(dirs), po, kw), "efie_far_field")
        return out

    def exterior_field(self, w, pts, out=None):
        """Scattered field (eq. ESLP) at points [npts][3] well away from the surface."""
        pts = np.ascontiguousarray(pts, float).reshape(-1, 3)
        nrhs = 1 if w.ndim == 1 else w.shape[0]
        if out is None:
            out = np.zeros((nrhs, pts.shape[0], 3), np.complex128) if isinstance(w, np.ndarray) else \
                w.new_zeros((nrhs, pts.shape[0], 3))
        pw, kw = _ptr(w)
        po, _ = _ptr(out)
        self._check(self._L.efie_exterior_field(self.h, nrhs, pw, pts.shape[0], _d(pts), po, kw),
                    "efie_exterior_field")
        return out

    def rhs_dipole(self, x0, p0, out=None):
        """Right-hand side for the incident field -DP_{x0,p0} (scattered field = the dipole)."""
        x0 = np.ascontiguousarray(x0, float).reshape(-1, 3)
        p0 = np.ascontiguousarray(p0, float).reshape(-1, 3)
        if out is None:
            out = np.zeros((x0.shape[0], self.ndof), np.complex128)
        po, k = _ptr(out)
        self._check(self._L.efie_rhs_dipole(self.h, x0.shape[0], _d(x0), _d(p0), po, k), "efie_rhs_dipole")
        return out

    def far_field_noalloc(self, w, dirs, out):
        """Far field of one right-hand side without device allocation; w, dirs ([ndir, 3]) and
        out ([ndir, 3] complex) must be CUDA tensors."""
        pw, kw = _ptr(w)
        pd, kd = _ptr(dirs)
        po, ko = _ptr(out)
        if not (kw == kd == ko == EFIE_PTR_DEVICE):
            raise ValueError("far_field_noalloc takes device tensors only")
        self._check(self._L.efie_far_field_noalloc(self.h, pw, dirs.shape[0], pd, po), "efie_far_field_noalloc")
        return out

    def blocks(self):
        far = np.zeros((self.nfar, 3), np.int32)
        near = np.zeros((self.nnear, 2), np.int32)
        self._check(self._L.efie_export_blocks(self.h, _i(far), _i(near)), "efie_export_blocks")
        return far, near

    def near_blocks(self):
        nb = 2 * (self.opts.p + 1) ** 2
        out = np.zeros((self.nnear, nb, nb), np.complex128)
        self._check(self._L.efie_export_near_blocks(self.h, _d(out.view(np.float64))), "efie_export_near_blocks")
        return out

    def launch_count(self):
        return int(self._L.efie_launch_count(self.h))

    def check_device_waits(self, cycles=1 << 20):
        """Run one bounded device wait that cannot complete; returns the status (expected
        EFIE_ETIMEOUT = -6) and efie_last_error's detail, without raising."""
        st = self._L.efie_check_device_waits(self.h, int(cycles))
        return st, self._L.efie_last_error(self.h).decode()

    def setup_timings(self):
        """Figures of the last setup: wall ms; touching-pair quadrature kernel ms, its quadrature
        points and pairs; separated-pair kernel ms and pairs; autotuned M2L times (ordered,
        unordered pairs) and the kernel kept (0 ordered, 1 unordered)."""
        out = np.zeros(9)
        n = self._L.efie_setup_timings(self.h, _d(out), 9)
        return dict(zip(["setup_ms", "near_quad_ms", "near_quad_points", "near_quad_pairs", "near_sep_ms",
                         "near_sep_pairs", "m2l_ordered_ms", "m2l_pairs_ms", "m2l_kept"], out[:n]))

    def last_timings(self):
        out = np.zeros(7)
        n = self._L.efie_last_timings(self.h, _d(out), 7)
        return dict(zip(["total", "gather", "near", "moments_m2m", "m2l", "l2l_eval", "scatter"], out[:n]))


def setup_many(solvers, nthreads=8):
    """efie_setup of several solvers (geometry set) on `nthreads` host threads; their device
    work overlaps on the GPU.  Raises on the first failure."""
    L = load()
    n = len(solvers)
    arr = (ctypes.c_void_p * n)(*[s.h.value for s in solvers])
    st = np.zeros(n, np.int32)
    rc = L.efie_setup_many(arr, n, int(nthreads), _i(st))
    for k, s in enumerate(solvers):
        if st[k] < 0:
            raise EfieError(int(st[k]), f"efie_setup_many (problem {k})", L, s.h)
        s._read_counts()
    if rc < 0:
        raise EfieError(rc, "efie_setup_many", L)
    return solvers


class Group:
    """Independent problems (set-up solvers on one device) solved in lockstep: one CUDA-graph
    launch of all products per GMRES step, batched Arnoldi/Givens work."""

    STATS = ("steps", "graph_captures", "kernels", "solve_ms", "product_graph_kernels", "chunks", "pre_ms",
             "products_ms", "post_ms")

    def __init__(self, solvers):
        self._L = load()
        self.solvers = list(solvers)
        n = len(self.solvers)
        arr = (ctypes.c_void_p * n)(*[s.h.value for s in self.solvers])
        h = ctypes.c_void_p()
        st = self._L.efie_group_create(ctypes.byref(h), arr, n)
        if st < 0:
            raise EfieError(st, "efie_group_create", self._L)
        self.h = h

    def solve(self, bs, xs=None):
        """Solve A_i x_i = b_i for every solver i; bs: list of (ndof_i,) numpy arrays or CUDA
        tensors.  Returns (xs, iterations, residuals, converged, status)."""
        n = len(self.solvers)
        if len(bs) != n:
            raise ValueError("one right-hand side per problem")
        if xs is None:
            xs = [np.empty_like(b) if isinstance(b, np.ndarray) else b.new_empty(b.shape) for b in bs]
        pb = [_ptr(b) for b in bs]
        px = [_ptr(x) for x in xs]
        kinds = {k for _, k in pb} | {k for _, k in px}
        if len(kinds) != 1:
            raise ValueError("all vectors must be host arrays or all CUDA tensors")
        for b, s in zip(bs, self.solvers):
            if b.shape[-1] != s.ndof:
                raise ValueError("right-hand side size differs from the problem's DOFs")
        ab = (ctypes.c_void_p * n)(*[p.value for p, _ in pb])
        ax = (ctypes.c_void_p * n)(*[p.value for p, _ in px])
        its = np.zeros(n, np.int32)
        res = np.zeros(n)
        conv = np.zeros(n, np.int32)
        st = self._L.efie_group_solve(self.h, ab, ax, kinds.pop(), _i(its), _d(res), _i(conv))
        if st < 0:
            raise RuntimeError(f"efie_group_solve: status {st}: {self._L.efie_group_last_error(self.h).decode()}")
        return xs, its, res, conv, st

    def stats(self):
        out = np.zeros(len(self.STATS))
        k = self._L.efie_group_stats(self.h, _d(out), len(out))
        return dict(zip(self.STATS, out[:k]))

    def close(self):
        if getattr(self, "h", None):
            self._L.efie_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop of the library: submit scattering requests, poll for results."""

    def __init__(self, hbm_budget_bytes, max_slots):
        self._L = load()
        h = ctypes.c_void_p()
        st = self._L.efie_server_create(ctypes.byref(h), int(hbm_budget_bytes), int(max_slots))
        if st < 0:
            raise EfieError(st, "efie_server_create", self._L)
        self.h = h
        self._keep = {}

    def submit(self, patches, dirs, pols, ff_dirs=None, **opts):
        """Queue a request; returns a ticket.  Output arrays are allocated here and returned
        by poll()."""
        from workloads.geometry import flatten

        deg, ncp, knots, cp, w = flatten(patches)
        o = options(**opts)
        dirs = np.ascontiguousarray(dirs, float).reshape(-1, 3)
        pols = np.ascontiguousarray(pols, float).reshape(-1, 3)
        n = 1 << o.level_m
        ndof = 2 * len(patches) * (n + o.p - 1) ** 2
        w_out = np.zeros((dirs.shape[0], ndof), np.complex128)
        ff = None if ff_dirs is None else np.ascontiguousarray(ff_dirs, float).reshape(-1, 3)
        e_out = None if ff is None else np.zeros((dirs.shape[0], ff.shape[0], 3), np.complex128)
        req = EfieRequest(len(patches), deg.ctypes.data, ncp.ctypes.data, knots.ctypes.data, cp.ctypes.data,
                          w.ctypes.data, o, dirs.shape[0], dirs.ctypes.data, pols.ctypes.data,
                          0 if ff is None else ff.shape[0], None if ff is None else ff.ctypes.data,
                          w_out.ctypes.data, None if e_out is None else e_out.ctypes.data)
        t = ctypes.c_uint64()
        st = self._L.efie_server_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st < 0:
            raise EfieError(st, "efie_server_submit", self._L)
        self._keep[t.value] = (w_out, e_out)
        return t.value

    def poll(self, ticket):
        """None while pending, else (result struct, w [nrhs][ndof], e_inf or None)."""
        r = EfieResult()
        st = self._L.efie_server_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r))
        if st == EFIE_PENDING:
            return None
        if st < 0:
            raise EfieError(st, "efie_server_poll", self._L)
        w_out, e_out = self._keep.pop(ticket)
        return r, w_out, e_out

    def wait(self, ticket, poll_s=0.002):
        import time

        while True:
            out = self.poll(ticket)
            if out is not None:
                return out
            time.sleep(poll_s)

    def close(self):
        if getattr(self, "h", None):
            self._L.efie_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
