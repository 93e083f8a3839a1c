"""Seeded, synthetic NURBS geometries used as inputs by both the CUDA path and the oracle.

This module only builds control nets (knots, control points, weights) of multipatch NURBS
surfaces.  It contains none of the boundary-element arithmetic; both the library and the
oracle evaluate the patches with their own code.

A patch is a dict with keys
  deg   (d0, d1)            polynomial degrees in s1 and s2
  knots (k0, k1)            p-open knot vectors on [0, 1]
  cp    [ncp1][ncp0][3]     control points (s1 index fastest)
  w     [ncp1][ncp0]        positive weights
Every patch factory returns patches oriented so that d_{s1}F x d_{s2}F points out of the
enclosed volume, as the boundary-element formulation requires.
"""
from __future__ import annotations

import math

import numpy as np


def _bezier_knots(d: int) -> np.ndarray:
    return np.array([0.0] * (d + 1) + [1.0] * (d + 1))


def _bernstein_matrix(d: int, t: np.ndarray) -> np.ndarray:
    """B[i, a] = binom(d, a) t_i^a (1 - t_i)^(d - a)."""
    t = np.asarray(t, dtype=np.float64)
    return np.stack([math.comb(d, a) * t ** a * (1.0 - t) ** (d - a) for a in range(d + 1)], axis=1)


def _fit_rational_bezier(fn, d: int):
    """Exact tensor rational Bezier form of a map whose homogeneous coordinates are
    tensor polynomials of bidegree (d, d).

    fn(u, v) -> (X, Y, Z, W) homogeneous polynomial values on a grid.  The Bernstein
    coefficients are recovered by inverting the (well conditioned) Bernstein collocation
    matrix on d+1 points per direction; the result is exact up to rounding because the
    input is a polynomial of that bidegree.
    """
    t = (np.arange(d + 1) + 0.5) / (d + 1)
    B = _bernstein_matrix(d, t)
    Binv = np.linalg.inv(B)
    U, V = np.meshgrid(t, t, indexing="xy")  # U varies along axis 1 (s1), V along axis 0 (s2)
    X, Y, Z, W = fn(U, V)
    coef = [Binv @ H @ Binv.T for H in (X, Y, Z, W)]  # [b(s2)][a(s1)]
    w = coef[3]
    cp = np.stack([coef[0] / w, coef[1] / w, coef[2] / w], axis=-1)
    return cp, w


def _patch(deg, cp, w, knots=None):
    d0, d1 = deg
    if knots is None:
        knots = (_bezier_knots(d0), _bezier_knots(d1))
    return {"deg": (int(d0), int(d1)), "knots": (np.asarray(knots[0], float), np.asarray(knots[1], float)),
            "cp": np.ascontiguousarray(cp, dtype=np.float64), "w": np.ascontiguousarray(w, dtype=np.float64)}


# proper rotations taking the +x axis to each cube-face normal
_FACE_ROT = [
    np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], float),     # +x
    np.array([[-1, 0, 0], [0, -1, 0], [0, 0, 1]], float),   # -x
    np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], float),    # +y
    np.array([[0, 1, 0], [-1, 0, 0], [0, 0, 1]], float),    # -y
    np.array([[0, 0, -1], [0, 1, 0], [1, 0, 0]], float),    # +z
    np.array([[0, 0, 1], [0, 1, 0], [-1, 0, 0]], float),    # -z
]


def _sphere_face_homogeneous(U, V):
    """Homogeneous coordinates of the +x face of the cube sphere.

    Q: a rational biquadratic map of the unit square onto the region of the plane that
    stereographic projection (from the pole (-1, 0, 0)) sends to the +x cube face; its
    four boundary curves are exact rational-quadratic circular arcs.  P: the inverse
    stereographic projection (s, t) -> ((1 - s^2 - t^2), 2s, 2t) / (1 + s^2 + t^2).
    Composing P with Q = (Xq, Yq) / Wq gives a rational map of bidegree (4, 4):
        ((Wq^2 - Xq^2 - Yq^2), 2 Xq Wq, 2 Yq Wq) / (Wq^2 + Xq^2 + Yq^2).
    """
    c = (math.sqrt(3.0) - 1.0) / 2.0           # corner (1,1,1)/sqrt(3) in the plane
    th = math.pi / 12.0                        # half opening angle of each boundary arc
    dmid = math.sqrt(2.0) / math.cos(th) - 1.0  # middle control point of each arc
    wm = math.cos(th)
    P = np.array([[[-c, -c], [0.0, -dmid], [c, -c]],
                  [[-dmid, 0.0], [0.0, 0.0], [dmid, 0.0]],
                  [[-c, c], [0.0, dmid], [c, c]]])           # [b][a][xy]
    Wt = np.array([[1.0, wm, 1.0], [wm, wm * wm, wm], [1.0, wm, 1.0]])
    Bu = [math.comb(2, a) * U ** a * (1 - U) ** (2 - a) for a in range(3)]
    Bv = [math.comb(2, b) * V ** b * (1 - V) ** (2 - b) for b in range(3)]
    Xq = sum(Bu[a] * Bv[b] * Wt[b, a] * P[b, a, 0] for a in range(3) for b in range(3))
    Yq = sum(Bu[a] * Bv[b] * Wt[b, a] * P[b, a, 1] for a in range(3) for b in range(3))
    Wq = sum(Bu[a] * Bv[b] * Wt[b, a] for a in range(3) for b in range(3))
    return (Wq * Wq - Xq * Xq - Yq * Yq, 2.0 * Xq * Wq, 2.0 * Yq * Wq, Wq * Wq + Xq * Xq + Yq * Yq)


def sphere(radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Exact sphere as 6 rational Bezier patches of bidegree (4, 4) (cube-sphere layout)."""
    cp0, w0 = _fit_rational_bezier(_sphere_face_homogeneous, 4)
    out = []
    for R in _FACE_ROT:
        cp = (cp0 @ R.T) * radius + np.asarray(center, float)
        out.append(_patch((4, 4), cp, w0.copy()))
    return out


def cube(side: float = 2.0, center=(0.0, 0.0, 0.0)):
    """Cube as 6 bilinear patches; face +x is (h, (2u-1)h, (2v-1)h), h = side/2."""
    h = side / 2.0
    cp0 = np.array([[[h, -h, -h], [h, h, -h]], [[h, -h, h], [h, h, h]]], float)
    out = []
    for R in _FACE_ROT:
        out.append(_patch((1, 1), cp0 @ R.T + np.asarray(center, float), np.ones((2, 2))))
    return out


def _quarter_arcs(radius: float, center2=(0.0, 0.0)):
    """Four rational quadratic quarter circles: list of (ctrl[3][2], w[3]) for angles
    [k pi/2, (k+1) pi/2]."""
    arcs = []
    for k in range(4):
        a0, a1 = k * math.pi / 2, (k + 1) * math.pi / 2
        p0 = np.array([math.cos(a0), math.sin(a0)])
        p2 = np.array([math.cos(a1), math.sin(a1)])
        p1 = p0 + p2
        ctrl = np.stack([p0, p1, p2]) * radius + np.asarray(center2, float)
        arcs.append((ctrl, np.array([1.0, math.sqrt(0.5), 1.0])))
    return arcs


def torus(R: float = 2.0, r: float = 0.5):
    """Exact torus as 16 rational biquadratic patches: s1 runs around the z axis (angle
    theta), s2 around the tube (angle phi).  Surface of revolution of the tube circle."""
    rev = _quarter_arcs(1.0)
    prof = _quarter_arcs(r, (R, 0.0))  # (rho, z) of the tube circle
    out = []
    for (pc, pw) in prof:            # s2 direction
        for (rc, rw) in rev:         # s1 direction
            cp = np.zeros((3, 3, 3))
            w = np.zeros((3, 3))
            for b in range(3):
                for a in range(3):
                    cp[b, a] = [pc[b, 0] * rc[a, 0], pc[b, 0] * rc[a, 1], pc[b, 1]]
                    w[b, a] = pw[b] * rw[a]
            out.append(_patch((2, 2), cp, w))
    return out


def _split_quadratic(ctrl, parts):
    """Split a quadratic Bezier curve (ctrl[3][2], polynomial) into `parts` equal parameter
    pieces by de Casteljau subdivision; returns the pieces' control points."""
    out = []
    for k in range(parts):
        t0, t1 = k / parts, (k + 1) / parts

        def at(t):
            return (1 - t) ** 2 * ctrl[0] + 2 * t * (1 - t) * ctrl[1] + t * t * ctrl[2]

        def d(t):
            return 2 * (1 - t) * (ctrl[1] - ctrl[0]) + 2 * t * (ctrl[2] - ctrl[1])

        p0, p2 = at(t0), at(t1)
        p1 = p0 + d(t0) * (t1 - t0) / 2.0
        out.append(np.stack([p0, p1, p2]))
    return out


def multicell(cells: int = 9, length: float = 1.0, r_eq: float = 0.9, r_iris: float = 0.35, r_in: float = 0.2,
              split: int = 2):
    """Synthetic many-patch surface of revolution (stand-in for multi-cell cavities): a closed
    profile in the (rho, z) half-plane, traversed counterclockwise, revolved about the z axis in
    four rational quarter turns.  The outer wall is `cells` bulges, each two quadratic arcs
    iris -> equator -> iris (horizontal tangent at the irises, vertical at the equator), then
    a flat end, a straight inner wall at rho = r_in and the other flat end; every profile piece
    (the bulge arcs split in `split` parts) gives 4 patches of bidegree (2, 2).  The default
    has 4 (2 cells split + 2 cells + 4) = 232 patches."""
    segs = []
    for c in range(cells):
        z0 = c * length
        up = np.array([[r_iris, z0], [r_eq, z0], [r_eq, z0 + length / 2]])
        down = np.array([[r_eq, z0 + length / 2], [r_eq, z0 + length], [r_iris, z0 + length]])
        segs += _split_quadratic(up, split) + _split_quadratic(down, split)

    def line(a, b, parts):
        a, b = np.asarray(a, float), np.asarray(b, float)
        return _split_quadratic(np.stack([a, (a + b) / 2, b]), parts)

    top = cells * length
    segs += line((r_iris, top), (r_in, top), 2)
    segs += line((r_in, top), (r_in, 0.0), 2 * cells)
    segs += line((r_in, 0.0), (r_iris, 0.0), 2)
    rev = _quarter_arcs(1.0)
    out = []
    for pc in segs:                  # s2 direction: the profile piece
        for (rc, rw) in rev:         # s1 direction: a quarter turn
            cp = np.zeros((3, 3, 3))
            w = np.zeros((3, 3))
            for b in range(3):
                for a in range(3):
                    cp[b, a] = [pc[b, 0] * rc[a, 0], pc[b, 0] * rc[a, 1], pc[b, 1]]
                    w[b, a] = rw[a]
            out.append(_patch((2, 2), cp, w))
    return out


def plane_waves(n: int, seed: int):
    """n seeded incident directions, uniform on S^2 (normalised Gaussians), each with a
    seeded random unit polarisation orthogonal to it."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = rng.standard_normal((n, 3))
    v -= np.sum(v * d, axis=1, keepdims=True) * d
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return d, v


def flatten(patches):
    """Pack a patch list into flat arrays (the layout both C interfaces take):
    deg[N][2], ncp[N][2], knots (concatenated k0 then k1 per patch), cp, w."""
    deg = np.array([p["deg"] for p in patches], dtype=np.int32).reshape(-1, 2)
    ncp = np.array([[p["cp"].shape[1], p["cp"].shape[0]] for p in patches], dtype=np.int32).reshape(-1, 2)
    knots = np.concatenate([np.concatenate([p["knots"][0], p["knots"][1]]) for p in patches]).astype(np.float64)
    cp = np.concatenate([p["cp"].reshape(-1) for p in patches]).astype(np.float64)
    w = np.concatenate([p["w"].reshape(-1) for p in patches]).astype(np.float64)
    return deg, ncp, knots, cp, w
