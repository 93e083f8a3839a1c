// Device evaluation of NURBS patch maps F_j: [0,1]^2 -> R^3 (Sec. 3.1, eq. def::geom) and
// of the Bernstein basis of the superspace (Sec. 4.1).  FP64 throughout.
#pragma once

#include "efie_internal.h"

namespace efie {

// All loops below run to compile-time bounds (kMaxGeoDeg, kMaxP1) and are predicated on the
// runtime degree, so that every small array stays in registers.  (A form with runtime loop
// bounds over the same local arrays produced wrong derivatives in some kernels; the
// evaluator is pinned against the oracle by the parity tests.)

// Values and first derivatives of the deg+1 B-splines that do not vanish at x; returns the
// knot span k (functions k-deg .. k).  Triangular Cox-de Boor scheme; the derivative uses
// the degree deg-1 values: b_f' = deg (b_f^{deg-1}/(t_{f+deg}-t_f) -
// b_{f+1}^{deg-1}/(t_{f+deg+1}-t_{f+1})).  inv holds the reciprocal knot differences
// inv[(d-1) nk + f] = 1 / (t_{f+d} - t_f) (0 where the difference is 0), nk = ncp + deg + 1,
// so that no division is evaluated here.  Loops run to the compile-time bound GD >= deg.
template <int GD>
__device__ inline int dev_bspline(const double *kn, const double *inv, int deg, int ncp, double x, double *N,
                                  double *dN) {
  int k;
  if (x >= kn[ncp]) {
    k = ncp - 1;
  } else {
    int lo = deg, hi = ncp;  // kn[lo] <= x < kn[hi]
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (x >= kn[mid]) lo = mid; else hi = mid;
    }
    k = lo;
  }
  const int nk = ncp + deg + 1;
  double cur[GD + 1], prev[GD + 1];
#pragma unroll
  for (int i = 0; i <= GD; ++i) {
    cur[i] = 0.0;
    prev[i] = 0.0;
  }
  cur[0] = 1.0;
#pragma unroll
  for (int d = 1; d <= GD; ++d) {
    if (d <= deg) {
#pragma unroll
      for (int i = 0; i <= GD; ++i) prev[i] = cur[i];
      const double *iv = inv + (d - 1) * nk;
#pragma unroll
      for (int i = 0; i <= GD; ++i) {
        if (i <= d) {
          int f = k - d + i;
          double v = 0.0;
          if (i >= 1) v += (x - kn[f]) * iv[f] * prev[i - 1];
          if (i < d) v += (kn[f + d + 1] - x) * iv[f + 1] * prev[i];
          cur[i] = v;
        }
      }
    }
  }
  const double *iv = inv + (deg - 1) * nk;
#pragma unroll
  for (int i = 0; i <= GD; ++i) {
    N[i] = cur[i];
    double v = 0.0;
    if (i <= deg) {
      int f = k - deg + i;
      if (i >= 1) v += deg * prev[i - 1] * iv[f];
      if (i < deg) v -= deg * prev[i] * iv[f + 1];
    }
    dN[i] = v;
  }
  return k;
}

// F(s), d1F(s), d2F(s) of one patch (rational, quotient rule); the patch degrees must not
// exceed GD.
template <int GD = kMaxGeoDeg>
__device__ inline void dev_patch_eval(const PatchDesc &Pg, const double *knots, const double4 *cpw, double s1,
                                      double s2, double X[3], double D1[3], double D2[3]) {
  const PatchDesc P = Pg;
  double Nu[GD + 1], dNu[GD + 1], Nv[GD + 1], dNv[GD + 1];
  int ku = dev_bspline<GD>(knots + P.kofs[0], knots + P.iofs[0], P.deg[0], P.ncp[0], s1, Nu, dNu);
  int kv = dev_bspline<GD>(knots + P.kofs[1], knots + P.iofs[1], P.deg[1], P.ncp[1], s2, Nv, dNv);
  // contraction in two stages: along s1 for each of the deg[1]+1 rows, then along s2
  double A[4] = {0, 0, 0, 0}, Au[4] = {0, 0, 0, 0}, Av[4] = {0, 0, 0, 0};
#pragma unroll
  for (int b = 0; b <= GD; ++b) {
    if (b <= P.deg[1]) {
      int r = kv - P.deg[1] + b;
      double R[4] = {0, 0, 0, 0}, Ru[4] = {0, 0, 0, 0};
#pragma unroll
      for (int a = 0; a <= GD; ++a) {
        if (a <= P.deg[0]) {
          double4 h = cpw[P.cofs + r * P.ncp[0] + ku - P.deg[0] + a];
          double c4[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            R[t] += Nu[a] * c4[t];
            Ru[t] += dNu[a] * c4[t];
          }
        }
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        A[t] += Nv[b] * R[t];
        Au[t] += Nv[b] * Ru[t];
        Av[t] += dNv[b] * R[t];
      }
    }
  }
  double iw = 1.0 / A[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    X[t] = A[t] * iw;
    D1[t] = (Au[t] - X[t] * Au[3]) * iw;
    D2[t] = (Av[t] - X[t] * Av[3]) * iw;
  }
}

// Bernstein values B_a^p(t) and derivatives, a = 0..p (p < kMaxP1).
__device__ inline void dev_bernstein(int p, double t, double *B, double *dB) {
  double lo[kMaxP1 + 1];
#pragma unroll
  for (int a = 0; a <= kMaxP1; ++a) lo[a] = 0.0;
  lo[0] = 1.0;  // degree 0
#pragma unroll
  for (int d = 1; d < kMaxP1; ++d) {
    if (d < p) {  // raise to degree d: B^d_a = (1-t) B^{d-1}_a + t B^{d-1}_{a-1}
#pragma unroll
      for (int a = kMaxP1 - 1; a >= 1; --a)
        if (a <= d) lo[a] = (1.0 - t) * lo[a] + t * lo[a - 1];
      lo[0] = (1.0 - t) * lo[0];
    }
  }
  // lo holds degree p-1 values (zero beyond index p-1)
#pragma unroll
  for (int a = 0; a < kMaxP1; ++a) {
    if (a <= p) {
      double l = a >= 1 ? lo[a - 1] : 0.0, r = a <= p - 1 ? lo[a] : 0.0;
      B[a] = (1.0 - t) * r + t * l;
      dB[a] = p * (l - r);
    } else {
      B[a] = 0.0;
      dB[a] = 0.0;
    }
  }
}

}  // namespace efie
