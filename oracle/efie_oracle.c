/* Oracle: plain serial FP64 implementation of the isogeometric EFIE with the
 * interpolation-based FMM of Doelz, Kurz, Schoeps, Wolf (arXiv 1807.03097).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the CPU
 * baseline of the benchmark; never by the library.  Every routine follows a passage of
 * the paper (cited by section / equation / algorithm) or a textbook definition, written
 * out without blocking or fusion so that it can be checked by eye.
 */
#include "efie_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------ */
/* 1-D building blocks                                                                  */
/* ------------------------------------------------------------------------------------ */

/* Gauss-Legendre rule on [0,1] (Newton iteration on the Legendre polynomial P_g). */
void orc_gauss01(int g, double *x, double *w) {
  for (int i = 0; i < g; ++i) {
    double t = cos(M_PI * (i + 0.75) / (g + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= g; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (g == 1) { p1 = t; p0 = 1.0; }
      dp = g * (t * p1 - p0) / (t * t - 1.0);
      double dt = p1 / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= g; ++k) {
        double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (g == 1) { p1 = t; p0 = 1.0; }
      dp = g * (t * p1 - p0) / (t * t - 1.0);
    }
    x[i] = 0.5 * (1.0 - t);
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
}

/* Chebyshev points of the first kind on [0,1], ascending (q+1 points, degree q). */
void orc_cheb01(int q, double *x) {
  for (int i = 0; i <= q; ++i) x[i] = 0.5 * (1.0 - cos((2.0 * i + 1.0) * M_PI / (2.0 * q + 2.0)));
}

/* Lagrange basis polynomial L_m of the nodes x[0..q] (Sec. 4.2). */
static double lagrange(int q, const double *xn, int m, double t) {
  double v = 1.0;
  for (int k = 0; k <= q; ++k)
    if (k != m) v *= (t - xn[k]) / (xn[m] - xn[k]);
  return v;
}

static double binom(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

/* Bernstein polynomials of degree p on [0,1] and their derivatives (local basis of the
 * discontinuous superspace S*_{p,m}, Sec. 4.1). */
static double bern(int p, int a, double t) {
  if (a < 0 || a > p) return 0.0;
  return binom(p, a) * pow(t, a) * pow(1.0 - t, p - a);
}
static double bern_d(int p, int a, double t) {
  if (p == 0) return 0.0;
  return p * (bern(p - 1, a - 1, t) - bern(p - 1, a, t));
}

/* B-spline b_j^p by the recursion of Def. "B-Splines" (Sec. 3.1), with chi on
 * half-open intervals; the right end of [0,1] belongs to the last non-empty interval. */
static double bspline(const double *kn, int nkn, int j, int p, double x) {
  if (p == 0) {
    if (x >= kn[j] && x < kn[j + 1]) return 1.0;
    if (x == kn[nkn - 1] && kn[j + 1] == x && kn[j] < x) return 1.0;
    return 0.0;
  }
  double v = 0.0;
  double d1 = kn[j + p] - kn[j];
  double d2 = kn[j + p + 1] - kn[j + 1];
  if (d1 > 0.0) v += (x - kn[j]) / d1 * bspline(kn, nkn, j, p - 1, x);
  if (d2 > 0.0) v += (kn[j + p + 1] - x) / d2 * bspline(kn, nkn, j + 1, p - 1, x);
  return v;
}
static double bspline_d(const double *kn, int nkn, int j, int p, double x) {
  if (p == 0) return 0.0;
  double v = 0.0;
  double d1 = kn[j + p] - kn[j];
  double d2 = kn[j + p + 1] - kn[j + 1];
  if (d1 > 0.0) v += p / d1 * bspline(kn, nkn, j, p - 1, x);
  if (d2 > 0.0) v -= p / d2 * bspline(kn, nkn, j + 1, p - 1, x);
  return v;
}

/* Solve a small dense real system A x = b in place (Gaussian elimination, pivoting). */
static void solve_small(int n, double *A, double *b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        double t = A[c * n + k];
        A[c * n + k] = A[piv * n + k];
        A[piv * n + k] = t;
      }
      double t = b[c];
      b[c] = b[piv];
      b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
}

static int morton(int i1, int i2) {
  int k = 0;
  for (int b = 0; b < 15; ++b) {
    k |= ((i1 >> b) & 1) << (2 * b);
    k |= ((i2 >> b) & 1) << (2 * b + 1);
  }
  return k;
}
static void demorton(int k, int *i1, int *i2) {
  int a = 0, c = 0;
  for (int b = 0; b < 15; ++b) {
    a |= ((k >> (2 * b)) & 1) << b;
    c |= ((k >> (2 * b + 1)) & 1) << b;
  }
  *i1 = a;
  *i2 = c;
}

/* ------------------------------------------------------------------------------------ */
/* Problem                                                                              */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  int deg[2], ncp[2];
  double *kn[2];
  double *cp; /* [ncp1][ncp0][3] */
  double *w;  /* [ncp1][ncp0] */
} Patch;

struct orc_problem {
  int leaf_dense; /* leaf-level variant of Algorithm 1 (see build_bct) */
  int np;
  Patch *pat;
  int p, m, n, q, nI, greg, gsing;
  double kappa, eta, scale, tol;
  int nE, nsup, nloc, nA, ndof;
  int *ldof;
  double *lsgn;
  int nbr[4096][3]; /* per (patch*4 + edge): neighbour patch, neighbour edge, reversed */
  double *Cp, *Cq;  /* extraction tables [n][p+1 (a)][p+1 (r)] */
  int nT;
  int *Trow, *Tcol;
  double *Tval;
  int ncl, nlev;
  int *cl_off; /* level offsets */
  double *ball; /* [ncl][4] */
  int nfar, capfar, nnear, capnear;
  int *far, *near;
  cplx *nblk;
  int nblk_done;
  double *chebx;
  double *Mt, *Mdt; /* moment tables [lev][2^(m-l)][nI1][p+1] */
  double *cgeo;     /* per cluster node: x[3], d1[3], d2[3] => 9 doubles */
  int rc_g;          /* regular-rule geometry cache: Gauss order and [nE][g*g][9] */
  double *rc_geo;
  int status;
  char msg[256];
};

static int nb_of(const orc_problem *P) { return 2 * (P->p + 1) * (P->p + 1); }

/* NURBS patch map F_j and its parameter derivatives (Sec. 3.1, eq. def::geom), by
 * direct summation over all control points; derivatives by the quotient rule. */
static void patch_eval(const Patch *pt, double s1, double s2, double X[3], double D1[3],
                       double D2[3]) {
  int n0 = pt->ncp[0], n1 = pt->ncp[1];
  int nk0 = n0 + pt->deg[0] + 1, nk1 = n1 + pt->deg[1] + 1;
  double bu[64], dbu[64], bv[64], dbv[64];
  for (int i1 = 0; i1 < n0; ++i1) {
    bu[i1] = bspline(pt->kn[0], nk0, i1, pt->deg[0], s1);
    dbu[i1] = bspline_d(pt->kn[0], nk0, i1, pt->deg[0], s1);
  }
  for (int i2 = 0; i2 < n1; ++i2) {
    bv[i2] = bspline(pt->kn[1], nk1, i2, pt->deg[1], s2);
    dbv[i2] = bspline_d(pt->kn[1], nk1, i2, pt->deg[1], s2);
  }
  double N[3] = {0, 0, 0}, N1[3] = {0, 0, 0}, N2[3] = {0, 0, 0}, W = 0, W1 = 0, W2 = 0;
  for (int i2 = 0; i2 < n1; ++i2) {
    if (bv[i2] == 0.0 && dbv[i2] == 0.0) continue;
    for (int i1 = 0; i1 < n0; ++i1) {
      double wt = pt->w[i2 * n0 + i1];
      const double *c = pt->cp + 3 * (i2 * n0 + i1);
      double b = bu[i1] * bv[i2] * wt, b1 = dbu[i1] * bv[i2] * wt, b2 = bu[i1] * dbv[i2] * wt;
      W += b;
      W1 += b1;
      W2 += b2;
      for (int k = 0; k < 3; ++k) {
        N[k] += c[k] * b;
        N1[k] += c[k] * b1;
        N2[k] += c[k] * b2;
      }
    }
  }
  for (int k = 0; k < 3; ++k) {
    X[k] = N[k] / W;
    if (D1) D1[k] = (N1[k] - X[k] * W1) / W;
    if (D2) D2[k] = (N2[k] - X[k] * W2) / W;
  }
}

void orc_eval_patch(const orc_problem *P, int patch, int npts, const double *s, double *x,
                    double *d1, double *d2) {
  for (int i = 0; i < npts; ++i)
    patch_eval(&P->pat[patch], s[2 * i], s[2 * i + 1], x + 3 * i, d1 ? d1 + 3 * i : NULL,
               d2 ? d2 + 3 * i : NULL);
}

static void elem_of(const orc_problem *P, int e, int *j, int *i1, int *i2) {
  int n2 = P->n * P->n;
  *j = e / n2;
  demorton(e % n2, i1, i2);
}

/* geometry at element-local coordinates sigma in [0,1]^2 (patch coordinates
 * s = (i + sigma)/n; derivatives are d/ds) */
static void elem_geo(const orc_problem *P, int e, const double sig[2], double X[3],
                     double D1[3], double D2[3]) {
  int j, i1, i2;
  elem_of(P, e, &j, &i1, &i2);
  patch_eval(&P->pat[j], (i1 + sig[0]) / P->n, (i2 + sig[1]) / P->n, X, D1, D2);
}

static double dist3(const double *a, const double *b) {
  double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
  return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

/* edge curves: 0 W (s1=0), 1 E (s1=1), 2 S (s2=0), 3 N (s2=1) */
static void edge_point(const Patch *pt, int k, double t, double X[3]) {
  double s1 = 0, s2 = 0;
  if (k == 0) { s1 = 0; s2 = t; }
  if (k == 1) { s1 = 1; s2 = t; }
  if (k == 2) { s1 = t; s2 = 0; }
  if (k == 3) { s1 = t; s2 = 1; }
  patch_eval(pt, s1, s2, X, NULL, NULL);
}

static int edge_sigma(int k) { return (k == 1 || k == 3) ? 1 : -1; }

static int loc_index(const orc_problem *P, int alpha, int i1, int i2) {
  int n = P->n, p = P->p;
  if (alpha == 0) return i2 * (n + p) + i1;
  return P->nA + i2 * (n + p - 1) + i1;
}

static void set_err(orc_problem *P, int code, const char *m) {
  if (P->status == 0) {
    P->status = code;
    snprintf(P->msg, sizeof P->msg, "%s", m);
  }
}

/* Interface matching (Sec. 3.1: F_j(.,1) = F_i(.,0) up to orientation) by comparing the
 * edge curves at five parameter values in both orientations. */
static void match_edges(orc_problem *P) {
  const double ts[5] = {0.0, 0.25, 0.5, 0.75, 1.0};
  for (int a = 0; a < 4 * P->np; ++a) P->nbr[a][0] = -1;
  for (int j = 0; j < P->np; ++j)
    for (int k = 0; k < 4; ++k) {
      int found = 0;
      double A[5][3];
      for (int t = 0; t < 5; ++t) edge_point(&P->pat[j], k, ts[t], A[t]);
      for (int j2 = 0; j2 < P->np; ++j2)
        for (int k2 = 0; k2 < 4; ++k2) {
          if (j2 == j && k2 == k) continue;
          double B[5][3];
          for (int t = 0; t < 5; ++t) edge_point(&P->pat[j2], k2, ts[t], B[t]);
          for (int rev = 0; rev < 2; ++rev) {
            double dmax = 0;
            for (int t = 0; t < 5; ++t) {
              double d = dist3(A[t], B[rev ? 4 - t : t]);
              if (d > dmax) dmax = d;
            }
            if (dmax < P->tol) {
              P->nbr[4 * j + k][0] = j2;
              P->nbr[4 * j + k][1] = k2;
              P->nbr[4 * j + k][2] = rev;
              ++found;
            }
          }
        }
      if (found != 1) set_err(P, -3, "patch edge without exactly one matching neighbour edge");
    }
}

/* Global S^1 numbering (Sec. 3.2, multipatch spline complex): patch-major, component,
 * i2, i1; the normal-trace functions of an interface are identified pairwise, with the
 * sign that makes the outward flux of one patch the inward flux of the other. */
static void build_dofs(orc_problem *P) {
  int n = P->n, p = P->p;
  P->nA = (n + p) * (n + p - 1);
  P->nloc = 2 * P->nA;
  P->ldof = malloc(sizeof(int) * P->np * P->nloc);
  P->lsgn = malloc(sizeof(double) * P->np * P->nloc);
  for (int i = 0; i < P->np * P->nloc; ++i) P->ldof[i] = -1;
  int nd = 0;
  for (int j = 0; j < P->np; ++j)
    for (int alpha = 0; alpha < 2; ++alpha) {
      int n1 = alpha == 0 ? n + p : n + p - 1;
      int n2 = alpha == 0 ? n + p - 1 : n + p;
      for (int i2 = 0; i2 < n2; ++i2)
        for (int i1 = 0; i1 < n1; ++i1) {
          int li = loc_index(P, alpha, i1, i2);
          if (P->ldof[j * P->nloc + li] >= 0) continue;
          P->ldof[j * P->nloc + li] = nd;
          P->lsgn[j * P->nloc + li] = 1.0;
          int k = -1, pos = 0;
          if (alpha == 0 && i1 == 0) { k = 0; pos = i2; }
          if (alpha == 0 && i1 == n + p - 1) { k = 1; pos = i2; }
          if (alpha == 1 && i2 == 0) { k = 2; pos = i1; }
          if (alpha == 1 && i2 == n + p - 1) { k = 3; pos = i1; }
          if (k >= 0 && P->nbr[4 * j + k][0] >= 0) {
            int j2 = P->nbr[4 * j + k][0], k2 = P->nbr[4 * j + k][1], rev = P->nbr[4 * j + k][2];
            int pp = rev ? (n + p - 2 - pos) : pos;
            int l2;
            if (k2 < 2) l2 = loc_index(P, 0, k2 == 0 ? 0 : n + p - 1, pp);
            else l2 = loc_index(P, 1, pp, k2 == 2 ? 0 : n + p - 1);
            P->ldof[j2 * P->nloc + l2] = nd;
            P->lsgn[j2 * P->nloc + l2] = -(double)(edge_sigma(k) * edge_sigma(k2));
          }
          ++nd;
        }
    }
  P->ndof = nd;
}

/* Bezier extraction by collocation: on element k, the B-spline of degree deg (knot
 * vector kn) with index k+r equals sum_a C[k][a][r] B_a^p on the element (for
 * deg = p-1 this is also the degree elevation to p). */
static void extraction(const orc_problem *P, const double *kn, int nkn, int deg, double *C) {
  int n = P->n, p = P->p, np1 = p + 1;
  for (int k = 0; k < n; ++k)
    for (int r = 0; r <= deg; ++r) {
      double A[64], b[8];
      for (int t = 0; t < np1; ++t) {
        double loc = (t + 0.5) / np1;
        for (int a = 0; a < np1; ++a) A[t * np1 + a] = bern(p, a, loc);
        b[t] = bspline(kn, nkn, k + r, deg, (k + loc) / n);
      }
      solve_small(np1, A, b);
      for (int a = 0; a < np1; ++a) C[(k * np1 + a) * np1 + r] = fabs(b[a]) < 1e-14 ? 0.0 : b[a];
    }
}

/* Transformation T of eq. superspace (Sec. 4.1): patchwise extraction times the +-1
 * interface identification. */
static void build_T(orc_problem *P) {
  int n = P->n, p = P->p, np1 = p + 1;
  int nk = n + 2 * p + 1, nkq = n + 2 * p - 1;
  double *kn = malloc(sizeof(double) * nk), *knq = malloc(sizeof(double) * nkq);
  for (int i = 0; i < nk; ++i) {
    int v = i - p;
    kn[i] = v <= 0 ? 0.0 : (v >= n ? 1.0 : (double)v / n);
  }
  for (int i = 0; i < nkq; ++i) knq[i] = kn[i + 1];
  P->Cp = calloc((size_t)n * np1 * np1, sizeof(double));
  P->Cq = calloc((size_t)n * np1 * np1, sizeof(double));
  extraction(P, kn, nk, p, P->Cp);
  extraction(P, knq, nkq, p - 1, P->Cq);
  int cap = P->nE * 2 * np1 * np1 * np1 * np1;
  P->Trow = malloc(sizeof(int) * cap);
  P->Tcol = malloc(sizeof(int) * cap);
  P->Tval = malloc(sizeof(double) * cap);
  int nT = 0;
  for (int e = 0; e < P->nE; ++e) {
    int j, i1e, i2e;
    elem_of(P, e, &j, &i1e, &i2e);
    for (int alpha = 0; alpha < 2; ++alpha) {
      int d1 = alpha == 0 ? p : p - 1, d2 = alpha == 0 ? p - 1 : p;
      const double *C1 = alpha == 0 ? P->Cp : P->Cq;
      const double *C2 = alpha == 0 ? P->Cq : P->Cp;
      for (int b = 0; b < np1; ++b)
        for (int a = 0; a < np1; ++a) {
          int row = ((e * 2 + alpha) * np1 + b) * np1 + a;
          for (int r2 = 0; r2 <= d2; ++r2)
            for (int r1 = 0; r1 <= d1; ++r1) {
              double c = C1[(i1e * np1 + a) * np1 + r1] * C2[(i2e * np1 + b) * np1 + r2];
              if (c == 0.0) continue;
              int li = loc_index(P, alpha, i1e + r1, i2e + r2);
              P->Trow[nT] = row;
              P->Tcol[nT] = P->ldof[j * P->nloc + li];
              P->Tval[nT] = c * P->lsgn[j * P->nloc + li];
              ++nT;
            }
        }
    }
  }
  P->nT = nT;
  free(kn);
  free(knq);
}

/* ---- cluster tree (Sec. 4.1, quadtree of the uniform refinement) ---- */
static int cl_id(const orc_problem *P, int l, int j, int K) {
  return P->cl_off[l] + j * (1 << (2 * l)) + K;
}

/* Bounding ball of a cluster: centre F(box centre), radius the largest distance of a 9x9
 * parameter grid (corners included) from the centre. */
static void cluster_ball(const orc_problem *P, int l, int j, int K, double out[4]) {
  int k1, k2;
  demorton(K, &k1, &k2);
  double hl = 1.0 / (1 << l);
  double c[3];
  patch_eval(&P->pat[j], (k1 + 0.5) * hl, (k2 + 0.5) * hl, c, NULL, NULL);
  double r = 0.0;
  for (int a = 0; a <= 8; ++a)
    for (int b = 0; b <= 8; ++b) {
      double X[3];
      patch_eval(&P->pat[j], (k1 + a / 8.0) * hl, (k2 + b / 8.0) * hl, X, NULL, NULL);
      double d = dist3(X, c);
      if (d > r) r = d;
    }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = r;
}

/* Admissibility, eq. admissibility: max(diam) <= eta dist, diam = 2r,
 * dist = |c - c'| - r - r' (must be positive). */
static int admissible(const orc_problem *P, int id1, int id2) {
  const double *b1 = P->ball + 4 * id1, *b2 = P->ball + 4 * id2;
  double dist = dist3(b1, b2) - b1[3] - b2[3];
  double diam = 2.0 * (b1[3] > b2[3] ? b1[3] : b2[3]);
  return dist > 0.0 && diam <= P->eta * dist;
}

static void push_far(orc_problem *P, int l, int t, int s) {
  if (P->nfar == P->capfar) {
    P->capfar = P->capfar ? 2 * P->capfar : 1024;
    P->far = realloc(P->far, sizeof(int) * 3 * P->capfar);
  }
  P->far[3 * P->nfar] = l;
  P->far[3 * P->nfar + 1] = t;
  P->far[3 * P->nfar + 2] = s;
  ++P->nfar;
}
static void push_near(orc_problem *P, int e, int e2) {
  if (P->nnear == P->capnear) {
    P->capnear = P->capnear ? 2 * P->capnear : 1024;
    P->near = realloc(P->near, sizeof(int) * 2 * P->capnear);
  }
  P->near[2 * P->nnear] = e;
  P->near[2 * P->nnear + 1] = e2;
  ++P->nnear;
}

/* Algorithm 1, BuildBlockClusterTree.  Leaf-level variant (leaf_dense): an admissible pair
 * of two leaves (single elements) is kept as an element block integrated by quadrature instead
 * of being compressed, when an element carries fewer basis functions per component than a
 * cluster carries interpolation nodes ((p+1)^2 < (q+1)^2); the paper's tree is leaf_dense = 0. */
static void build_bct(orc_problem *P, int l, int j, int K, int j2, int K2) {
  int a = cl_id(P, l, j, K), b = cl_id(P, l, j2, K2);
  if (admissible(P, a, b)) {
    if (P->leaf_dense && l == P->m && (P->p + 1) * (P->p + 1) < P->nI) {
      int n2 = P->n * P->n;
      push_near(P, j * n2 + K, j2 * n2 + K2);
    } else {
      push_far(P, l, a, b);
    }
    return;
  }
  if (l == P->m) {
    int n2 = P->n * P->n;
    push_near(P, j * n2 + K, j2 * n2 + K2);
    return;
  }
  for (int c = 0; c < 4; ++c)
    for (int c2 = 0; c2 < 4; ++c2) build_bct(P, l + 1, j, 4 * K + c, j2, 4 * K2 + c2);
}

orc_problem *orc_create(int np, const int *deg, const int *ncp, const double *knots,
                        const double *cp, const double *w, int p, int m, double kappa,
                        int q, double eta, int g_reg, int g_sing) {
  return orc_create_variant(np, deg, ncp, knots, cp, w, p, m, kappa, q, eta, g_reg, g_sing, 0);
}

orc_problem *orc_create_variant(int np, const int *deg, const int *ncp, const double *knots,
                                const double *cp, const double *w, int p, int m, double kappa,
                                int q, double eta, int g_reg, int g_sing, int leaf_dense) {
  orc_problem *P = calloc(1, sizeof(orc_problem));
  if (!P) return NULL;
  P->leaf_dense = leaf_dense;
  if (np <= 0 || np > 1024 || p < 1 || p > 6 || m < 0 || m > 10 || q < 1 || q > 20 ||
      !(kappa > 0) || !(eta > 0) || g_reg < 1 || g_sing < 1 || g_reg > 60 || g_sing > 60) {
    set_err(P, -1, "invalid argument");
    return P;
  }
  P->np = np;
  P->p = p;
  P->m = m;
  P->n = 1 << m;
  P->q = q;
  P->nI = (q + 1) * (q + 1);
  P->kappa = kappa;
  P->eta = eta;
  P->greg = g_reg;
  P->gsing = g_sing;
  P->pat = calloc(np, sizeof(Patch));
  size_t ko = 0, co = 0;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int j = 0; j < np; ++j) {
    Patch *pt = &P->pat[j];
    for (int d = 0; d < 2; ++d) {
      pt->deg[d] = deg[2 * j + d];
      pt->ncp[d] = ncp[2 * j + d];
      int nk = pt->ncp[d] + pt->deg[d] + 1;
      pt->kn[d] = malloc(sizeof(double) * nk);
      memcpy(pt->kn[d], knots + ko, sizeof(double) * nk);
      ko += nk;
    }
    if (pt->ncp[0] > 64 || pt->ncp[1] > 64 || pt->deg[0] < 1 || pt->deg[1] < 1) set_err(P, -1, "patch control net larger than 64 or degree < 1");
    int nc = pt->ncp[0] * pt->ncp[1];
    pt->cp = malloc(sizeof(double) * 3 * nc);
    pt->w = malloc(sizeof(double) * nc);
    memcpy(pt->cp, cp + 3 * co, sizeof(double) * 3 * nc);
    memcpy(pt->w, w + co, sizeof(double) * nc);
    for (int i = 0; i < nc; ++i)
      for (int k = 0; k < 3; ++k) {
        if (pt->cp[3 * i + k] < lo[k]) lo[k] = pt->cp[3 * i + k];
        if (pt->cp[3 * i + k] > hi[k]) hi[k] = pt->cp[3 * i + k];
      }
    co += nc;
  }
  if (P->status) return P;
  P->scale = dist3(lo, hi);
  P->tol = 1e-9 * P->scale;
  P->nE = np * P->n * P->n;
  P->nsup = P->nE * 2 * (p + 1) * (p + 1);
  match_edges(P);
  if (P->status) return P;
  build_dofs(P);
  build_T(P);
  /* clusters */
  P->nlev = m + 1;
  P->cl_off = malloc(sizeof(int) * (m + 2));
  int off = 0;
  for (int l = 0; l <= m; ++l) {
    P->cl_off[l] = off;
    off += np * (1 << (2 * l));
  }
  P->cl_off[m + 1] = off;
  P->ncl = off;
  P->ball = malloc(sizeof(double) * 4 * off);
  for (int l = 0; l <= m; ++l)
    for (int j = 0; j < np; ++j)
      for (int K = 0; K < (1 << (2 * l)); ++K) cluster_ball(P, l, j, K, P->ball + 4 * cl_id(P, l, j, K));
  for (int j = 0; j < np; ++j)
    for (int j2 = 0; j2 < np; ++j2) build_bct(P, 0, j, 0, j2, 0);
  /* interpolation nodes and direct (non-nested) moment tables */
  P->chebx = malloc(sizeof(double) * (q + 1));
  orc_cheb01(q, P->chebx);
  {
    int np1 = p + 1, q1 = q + 1;
    int ng = (q + p) / 2 + 2;
    double gx[64], gw[64];
    orc_gauss01(ng, gx, gw);
    size_t tot = 0;
    for (int l = 0; l <= m; ++l) tot += (size_t)(1 << (m - l)) * q1 * np1;
    P->Mt = calloc(tot, sizeof(double));
    P->Mdt = calloc(tot, sizeof(double));
    size_t o = 0;
    for (int l = 0; l <= m; ++l) {
      int no = 1 << (m - l);
      for (int oo = 0; oo < no; ++oo)
        for (int mi = 0; mi < q1; ++mi)
          for (int a = 0; a < np1; ++a) {
            double s = 0, sd = 0;
            for (int g = 0; g < ng; ++g) {
              double L = lagrange(q, P->chebx, mi, (oo + gx[g]) / no);
              s += gw[g] * L * bern(p, a, gx[g]);
              sd += gw[g] * L * bern_d(p, a, gx[g]);
            }
            P->Mt[o + ((size_t)oo * q1 + mi) * np1 + a] = s;
            P->Mdt[o + ((size_t)oo * q1 + mi) * np1 + a] = sd;
          }
      o += (size_t)no * q1 * np1;
    }
  }
  /* geometry at the interpolation nodes of every cluster */
  P->cgeo = malloc(sizeof(double) * 9 * (size_t)P->ncl * P->nI);
  for (int l = 0; l <= m; ++l)
    for (int j = 0; j < np; ++j)
      for (int K = 0; K < (1 << (2 * l)); ++K) {
        int k1, k2;
        demorton(K, &k1, &k2);
        double hl = 1.0 / (1 << l);
        int id = cl_id(P, l, j, K);
        for (int m2 = 0; m2 <= q; ++m2)
          for (int m1 = 0; m1 <= q; ++m1) {
            double *g = P->cgeo + 9 * ((size_t)id * P->nI + m2 * (q + 1) + m1);
            patch_eval(&P->pat[j], (k1 + P->chebx[m1]) * hl, (k2 + P->chebx[m2]) * hl, g, g + 3,
                       g + 6);
          }
      }
  return P;
}

void orc_destroy(orc_problem *P) {
  if (!P) return;
  for (int j = 0; j < P->np && P->pat; ++j) {
    free(P->pat[j].kn[0]);
    free(P->pat[j].kn[1]);
    free(P->pat[j].cp);
    free(P->pat[j].w);
  }
  free(P->pat);
  free(P->ldof);
  free(P->lsgn);
  free(P->Cp);
  free(P->Cq);
  free(P->Trow);
  free(P->Tcol);
  free(P->Tval);
  free(P->cl_off);
  free(P->ball);
  free(P->far);
  free(P->near);
  free(P->nblk);
  free(P->chebx);
  free(P->Mt);
  free(P->Mdt);
  free(P->cgeo);
  free(P->rc_geo);
  free(P);
}

int orc_status(const orc_problem *P, char *msg, int msglen) {
  if (msg && msglen > 0) snprintf(msg, msglen, "%s", P->msg);
  return P->status;
}
int orc_num_dofs(const orc_problem *P) { return P->ndof; }
int orc_num_elements(const orc_problem *P) { return P->nE; }
int orc_superspace_size(const orc_problem *P) { return P->nsup; }
int orc_num_clusters(const orc_problem *P) { return P->ncl; }
int orc_num_far(const orc_problem *P) { return P->nfar; }
int orc_num_near(const orc_problem *P) { return P->nnear; }
void orc_far_pairs(const orc_problem *P, int *out) { memcpy(out, P->far, sizeof(int) * 3 * P->nfar); }
void orc_near_pairs(const orc_problem *P, int *out) { memcpy(out, P->near, sizeof(int) * 2 * P->nnear); }
void orc_cluster_balls(const orc_problem *P, double *out) { memcpy(out, P->ball, sizeof(double) * 4 * P->ncl); }

int orc_T_coo(const orc_problem *P, int cap, int *row, int *col, double *val) {
  for (int i = 0; i < P->nT && i < cap; ++i) {
    row[i] = P->Trow[i];
    col[i] = P->Tcol[i];
    val[i] = P->Tval[i];
  }
  return P->nT;
}

static void apply_T(const orc_problem *P, const cplx *x, cplx *xs) {
  for (int i = 0; i < P->nsup; ++i) xs[i] = 0;
  for (int k = 0; k < P->nT; ++k) xs[P->Trow[k]] += P->Tval[k] * x[P->Tcol[k]];
}
static void apply_Tt(const orc_problem *P, const cplx *ys, cplx *y) {
  for (int i = 0; i < P->ndof; ++i) y[i] = 0;
  for (int k = 0; k < P->nT; ++k) y[P->Tcol[k]] += P->Tval[k] * ys[P->Trow[k]];
}

/* ------------------------------------------------------------------------------------ */
/* Element-pair quadrature                                                              */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  double s[2], t[2], w;
} QP;

/* symmetry of the unit square: optional swap of the two coordinates, then optional
 * reflections x -> 1-x, y -> 1-y */
static void sym_apply(int r, const double u[2], double out[2]) {
  double a = (r & 1) ? u[1] : u[0];
  double b = (r & 1) ? u[0] : u[1];
  if (r & 2) a = 1.0 - a;
  if (r & 4) b = 1.0 - b;
  out[0] = a;
  out[1] = b;
}
static int sym_find(int cP, int cQ) {
  for (int r = 0; r < 8; ++r) {
    double o[2], u0[2] = {0, 0}, u1[2] = {1, 0};
    sym_apply(r, u0, o);
    if ((int)o[0] + 2 * (int)o[1] != cP) continue;
    if (cQ < 0) return r;
    sym_apply(r, u1, o);
    if ((int)(o[0] + 0.5) + 2 * (int)(o[1] + 0.5) == cQ) return r;
  }
  return -1;
}

static void elem_corners(const orc_problem *P, int e, double C[4][3]) {
  for (int c = 0; c < 4; ++c) {
    double sig[2] = {(double)(c & 1), (double)(c >> 1)};
    elem_geo(P, e, sig, C[c], NULL, NULL);
  }
}

/* tolerance-aware lexicographic order of two points (role-independent choice of the
 * shared-edge direction) */
static int lex_less(const double *a, const double *b, double tol) {
  for (int k = 0; k < 3; ++k) {
    if (fabs(a[k] - b[k]) > tol) return a[k] < b[k];
  }
  return 0;
}

/* Classify an element pair by shared corners and return the square symmetries that put
 * the shared vertex at (0,0) / the shared edge on {x2 = 0} in both elements.
 * 3 identical, 2 common edge, 1 common vertex, 0 separated, -1 invalid. */
static int classify(const orc_problem *P, int e, int e2, int *r1, int *r2) {
  *r1 = 0;
  *r2 = 0;
  if (e == e2) return 3;
  double A[4][3], B[4][3];
  elem_corners(P, e, A);
  elem_corners(P, e2, B);
  int ca[4], cb[4], ns = 0;
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k)
      if (dist3(A[i], B[k]) < P->tol) {
        ca[ns] = i;
        cb[ns] = k;
        ++ns;
      }
  if (ns == 0) return 0;
  if (ns == 1) {
    *r1 = sym_find(ca[0], -1);
    *r2 = sym_find(cb[0], -1);
    return 1;
  }
  if (ns == 2) {
    int first = lex_less(A[ca[1]], A[ca[0]], P->tol) ? 1 : 0;
    int second = 1 - first;
    *r1 = sym_find(ca[first], ca[second]);
    *r2 = sym_find(cb[first], cb[second]);
    if (*r1 < 0 || *r2 < 0) return -1;
    return 2;
  }
  return -1;
}

int orc_pair_kind(const orc_problem *P, int e, int e2) {
  int r1, r2;
  return classify(P, e, e2, &r1, &r2);
}

/* Quadrature points of one element pair in element-local coordinates.  Separated pairs:
 * tensor Gauss.  Touching pairs: the Sauter-Schwab singularity-removing substitutions
 * [SS97] derived for the unit square: relative coordinates z = t - s, then a Duffy
 * split of the singular coordinates (identical: 8 parts, common edge: 6, common vertex:
 * 4), each part a tensor Gauss rule on [0,1]^4. */
static int pair_rule(const orc_problem *P, int e, int e2, int greg, int gsing, QP **out) {
  int r1, r2;
  int kind = classify(P, e, e2, &r1, &r2);
  if (kind < 0) {
    *out = NULL;
    return -1;
  }
  int g = kind == 0 ? greg : gsing;
  double gx[64], gw[64];
  orc_gauss01(g, gx, gw);
  int g4 = g * g * g * g;
  int nparts = kind == 0 ? 1 : (kind == 3 ? 8 : (kind == 2 ? 6 : 4));
  QP *Q = malloc(sizeof(QP) * (size_t)g4 * nparts);
  int nq = 0;
  for (int part = 0; part < nparts; ++part)
    for (int i0 = 0; i0 < g; ++i0)
      for (int i1 = 0; i1 < g; ++i1)
        for (int i2 = 0; i2 < g; ++i2)
          for (int i3 = 0; i3 < g; ++i3) {
            double W = gw[i0] * gw[i1] * gw[i2] * gw[i3];
            double sh[2], th[2];
            if (kind == 0) {
              sh[0] = gx[i0];
              sh[1] = gx[i1];
              th[0] = gx[i2];
              th[1] = gx[i3];
            } else if (kind == 3) {
              double xi = gx[i0], eta = gx[i1], u[2] = {gx[i2], gx[i3]};
              int q1 = (part & 1) ? -1 : 1, q2 = (part & 2) ? -1 : 1, tri = part >> 2;
              double z[2] = {tri == 0 ? xi : xi * eta, tri == 0 ? xi * eta : xi};
              int qs[2] = {q1, q2};
              for (int d = 0; d < 2; ++d) {
                sh[d] = (qs[d] < 0 ? z[d] : 0.0) + (1.0 - z[d]) * u[d];
                th[d] = sh[d] + qs[d] * z[d];
              }
              W *= xi * (1.0 - z[0]) * (1.0 - z[1]);
            } else if (kind == 2) {
              double xi = gx[i0], e1 = gx[i1], e2v = gx[i2], u = gx[i3];
              int qq = (part & 1) ? -1 : 1, pyr = part >> 1;
              double zeta, a2, b2;
              if (pyr == 0) { zeta = xi; a2 = xi * e1; b2 = xi * e2v; }
              else if (pyr == 1) { a2 = xi; zeta = xi * e1; b2 = xi * e2v; }
              else { b2 = xi; zeta = xi * e1; a2 = xi * e2v; }
              sh[0] = (qq < 0 ? zeta : 0.0) + (1.0 - zeta) * u;
              th[0] = sh[0] + qq * zeta;
              sh[1] = a2;
              th[1] = b2;
              W *= xi * xi * (1.0 - zeta);
            } else {
              double xi = gx[i0], et[3] = {gx[i1], gx[i2], gx[i3]}, v[4];
              int k = 0;
              for (int d = 0; d < 4; ++d) v[d] = (d == part) ? xi : xi * et[k++];
              sh[0] = v[0];
              sh[1] = v[1];
              th[0] = v[2];
              th[1] = v[3];
              W *= xi * xi * xi;
            }
            sym_apply(r1, sh, Q[nq].s);
            sym_apply(r2, th, Q[nq].t);
            Q[nq].w = W;
            ++nq;
          }
  *out = Q;
  return nq;
}

static int classify_kind(const orc_problem *P, int e, int e2) {
  int r1, r2;
  return classify(P, e, e2, &r1, &r2);
}

/* geometry at the tensor Gauss points of every element (pure cache of patch_eval) */
static void regular_cache(orc_problem *P, int g) {
  if (P->rc_geo && P->rc_g == g) return;
  free(P->rc_geo);
  double gx[64], gw[64];
  orc_gauss01(g, gx, gw);
  P->rc_geo = malloc(sizeof(double) * 9 * (size_t)P->nE * g * g);
  P->rc_g = g;
  for (int e = 0; e < P->nE; ++e)
    for (int i = 0; i < g; ++i)
      for (int j = 0; j < g; ++j) {
        double sig[2] = {gx[i], gx[j]};
        double *o = P->rc_geo + 9 * ((size_t)e * g * g + i * g + j);
        elem_geo(P, e, sig, o, o + 3, o + 6);
      }
}

static cplx helmholtz(double kappa, double r) { return cexp(I * kappa * r) / (4.0 * M_PI * r); }

/* Element-pair block of V* (eq. Vkh written in patch coordinates, sigma the element-local
 * coordinate, s = (i + sigma)/n): rows index (alpha, b, a) of e, columns (beta, b', a')
 * of e2:
 *   h^4 int int G <d_alpha F(s), d_beta F(t)> psi(sigma) psi'(tau)
 *   - kappa^-2 h^2 int int G d_alpha psi(sigma) d_beta psi'(tau). */
static int pair_block(const orc_problem *P, int e, int e2, int greg, int gsing, cplx *blk) {
  int p = P->p, np1 = p + 1, nb = nb_of(P);
  double h = 1.0 / P->n, h2 = h * h, h4 = h2 * h2, ik2 = 1.0 / (P->kappa * P->kappa);
  QP *Q;
  int nq = pair_rule(P, e, e2, greg, gsing, &Q);
  if (nq < 0) return -1;
  for (int i = 0; i < nb * nb; ++i) blk[i] = 0;
  double *vs = malloc(sizeof(double) * nb * 4), *vt = malloc(sizeof(double) * nb * 4);
  const double *rc = (P->rc_geo && P->rc_g == greg && nq == greg * greg * greg * greg &&
                      classify_kind(P, e, e2) == 0) ? P->rc_geo : NULL;
  int gg = greg * greg;
  for (int k = 0; k < nq; ++k) {
    double X[3], D[2][3], Y[3], E[2][3];
    if (rc) { /* tensor rule: point k = ((i0*g + i1)*g + i2)*g + i3 */
      const double *a = rc + 9 * ((size_t)e * gg + k / gg), *c = rc + 9 * ((size_t)e2 * gg + k % gg);
      for (int t = 0; t < 3; ++t) {
        X[t] = a[t]; D[0][t] = a[3 + t]; D[1][t] = a[6 + t];
        Y[t] = c[t]; E[0][t] = c[3 + t]; E[1][t] = c[6 + t];
      }
    } else {
      elem_geo(P, e, Q[k].s, X, D[0], D[1]);
      elem_geo(P, e2, Q[k].t, Y, E[0], E[1]);
    }
    cplx G = helmholtz(P->kappa, dist3(X, Y)) * Q[k].w;
    /* vs[r*4 + c] = d_alpha F(s)[c] psi_r (c<3), vs[r*4+3] = d_alpha psi_r */
    for (int alpha = 0; alpha < 2; ++alpha)
      for (int b = 0; b < np1; ++b)
        for (int a = 0; a < np1; ++a) {
          int r = (alpha * np1 + b) * np1 + a;
          double ps = bern(p, a, Q[k].s[0]) * bern(p, b, Q[k].s[1]);
          double dps = alpha == 0 ? bern_d(p, a, Q[k].s[0]) * bern(p, b, Q[k].s[1])
                                  : bern(p, a, Q[k].s[0]) * bern_d(p, b, Q[k].s[1]);
          double pt = bern(p, a, Q[k].t[0]) * bern(p, b, Q[k].t[1]);
          double dpt = alpha == 0 ? bern_d(p, a, Q[k].t[0]) * bern(p, b, Q[k].t[1])
                                  : bern(p, a, Q[k].t[0]) * bern_d(p, b, Q[k].t[1]);
          for (int c = 0; c < 3; ++c) {
            vs[r * 4 + c] = D[alpha][c] * ps;
            vt[r * 4 + c] = E[alpha][c] * pt;
          }
          vs[r * 4 + 3] = dps;
          vt[r * 4 + 3] = dpt;
        }
    for (int r = 0; r < nb; ++r)
      for (int c = 0; c < nb; ++c) {
        double dot = vs[r * 4] * vt[c * 4] + vs[r * 4 + 1] * vt[c * 4 + 1] + vs[r * 4 + 2] * vt[c * 4 + 2];
        blk[r * nb + c] += G * (h4 * dot - ik2 * h2 * vs[r * 4 + 3] * vt[c * 4 + 3]);
      }
  }
  free(vs);
  free(vt);
  free(Q);
  return 0;
}

void orc_pair_block(const orc_problem *P, int e, int e2, int g_reg, int g_sing, double *out) {
  pair_block(P, e, e2, g_reg, g_sing, (cplx *)out);
}

void orc_pair_scalar(const orc_problem *P, int e, int e2, int g_reg, int g_sing, double kappa,
                     double *out2) {
  QP *Q;
  int nq = pair_rule(P, e, e2, g_reg, g_sing, &Q);
  cplx s = 0;
  double h2 = 1.0 / ((double)P->n * P->n);
  for (int k = 0; k < nq; ++k) {
    double X[3], D[2][3], Y[3], E[2][3];
    elem_geo(P, e, Q[k].s, X, D[0], D[1]);
    elem_geo(P, e2, Q[k].t, Y, E[0], E[1]);
    double n1[3] = {D[0][1] * D[1][2] - D[0][2] * D[1][1], D[0][2] * D[1][0] - D[0][0] * D[1][2],
                    D[0][0] * D[1][1] - D[0][1] * D[1][0]};
    double n2[3] = {E[0][1] * E[1][2] - E[0][2] * E[1][1], E[0][2] * E[1][0] - E[0][0] * E[1][2],
                    E[0][0] * E[1][1] - E[0][1] * E[1][0]};
    double z[3] = {0, 0, 0};
    double tau1 = dist3(n1, z), tau2 = dist3(n2, z);
    s += Q[k].w * helmholtz(kappa, dist3(X, Y)) * tau1 * tau2 * h2 * h2;
  }
  free(Q);
  out2[0] = creal(s);
  out2[1] = cimag(s);
}

static void ensure_near_blocks(orc_problem *P) {
  if (P->nblk_done) return;
  regular_cache(P, P->greg);
  int nb = nb_of(P);
  P->nblk = malloc(sizeof(cplx) * (size_t)P->nnear * nb * nb);
  /* independent pairs: the optional OpenMP loop changes no arithmetic */
#pragma omp parallel for schedule(dynamic, 4)
  for (int k = 0; k < P->nnear; ++k) {
    if (pair_block(P, P->near[2 * k], P->near[2 * k + 1], P->greg, P->gsing,
                   P->nblk + (size_t)k * nb * nb) < 0)
      set_err(P, -3, "invalid element pair (overlapping elements)");
  }
  P->nblk_done = 1;
}

void orc_near_blocks(orc_problem *P, double *out) {
  ensure_near_blocks(P);
  int nb = nb_of(P);
  memcpy(out, P->nblk, sizeof(cplx) * (size_t)P->nnear * nb * nb);
}

void orc_dense_superspace(const orc_problem *P, double *out) {
  regular_cache((orc_problem *)P, P->greg);
  int nb = nb_of(P);
  int S = P->nsup;
  cplx *V = (cplx *)out;
  cplx *blk = malloc(sizeof(cplx) * nb * nb);
  for (int e = 0; e < P->nE; ++e)
    for (int e2 = 0; e2 < P->nE; ++e2) {
      pair_block(P, e, e2, P->greg, P->gsing, blk);
      for (int r = 0; r < nb; ++r)
        for (int c = 0; c < nb; ++c) V[(size_t)(e * nb + r) * S + e2 * nb + c] = blk[r * nb + c];
    }
  free(blk);
}

void orc_dense_matvec(const orc_problem *P, int nrhs, const double *x, double *y) {
  int S = P->nsup;
  cplx *V = malloc(sizeof(cplx) * (size_t)S * S);
  orc_dense_superspace(P, (double *)V);
  cplx *xs = malloc(sizeof(cplx) * S), *ys = malloc(sizeof(cplx) * S);
  for (int r = 0; r < nrhs; ++r) {
    apply_T(P, (const cplx *)x + (size_t)r * P->ndof, xs);
    for (int i = 0; i < S; ++i) {
      cplx s = 0;
      for (int k = 0; k < S; ++k) s += V[(size_t)i * S + k] * xs[k];
      ys[i] = s;
    }
    apply_Tt(P, ys, (cplx *)y + (size_t)r * P->ndof);
  }
  free(V);
  free(xs);
  free(ys);
}

/* ------------------------------------------------------------------------------------ */
/* Interpolation FMM, non-nested (Sec. 4.2, eq. FMMlr)                                  */
/* ------------------------------------------------------------------------------------ */

static const double *mom_table(const orc_problem *P, int deriv, int l) {
  size_t o = 0;
  int q1 = P->q + 1, np1 = P->p + 1;
  for (int ll = 0; ll < l; ++ll) o += (size_t)(1 << (P->m - ll)) * q1 * np1;
  return (deriv ? P->Mdt : P->Mt) + o;
}

/* moments of every cluster, computed directly from its elements:
 * mu_beta(m) = sum_e sum_ab [int L_m psi_ab] x*_{e,beta,ab},
 * nu(m) = sum_e sum_beta sum_ab [int L_m d_beta psi_ab] x*_{e,beta,ab} */
static cplx *direct_moments(const orc_problem *P, const cplx *xs) {
  int p = P->p, np1 = p + 1, q1 = P->q + 1, nI = P->nI;
  double h = 1.0 / P->n, h2 = h * h;
  cplx *mom = calloc((size_t)P->ncl * 3 * nI, sizeof(cplx));
  for (int l = 0; l <= P->m; ++l) {
    const double *M = mom_table(P, 0, l), *Md = mom_table(P, 1, l);
    int sh = P->m - l;
    for (int e = 0; e < P->nE; ++e) {
      int j, i1, i2;
      elem_of(P, e, &j, &i1, &i2);
      int id = cl_id(P, l, j, morton(i1 >> sh, i2 >> sh));
      int o1 = i1 - ((i1 >> sh) << sh), o2 = i2 - ((i2 >> sh) << sh);
      cplx *mu = mom + (size_t)id * 3 * nI;
      for (int m2 = 0; m2 < q1; ++m2)
        for (int m1 = 0; m1 < q1; ++m1)
          for (int beta = 0; beta < 2; ++beta)
            for (int b = 0; b < np1; ++b)
              for (int a = 0; a < np1; ++a) {
                cplx xv = xs[((size_t)(e * 2 + beta) * np1 + b) * np1 + a];
                double Ma = M[(o1 * q1 + m1) * np1 + a], Mb = M[(o2 * q1 + m2) * np1 + b];
                double Dda = Md[(o1 * q1 + m1) * np1 + a], Ddb = Md[(o2 * q1 + m2) * np1 + b];
                mu[beta * nI + m2 * q1 + m1] += h2 * Ma * Mb * xv;
                mu[2 * nI + m2 * q1 + m1] += h * (beta == 0 ? Dda * Mb : Ma * Ddb) * xv;
              }
    }
  }
  return mom;
}

/* one admissible block (eq. FMMlr): with K1^(alpha,beta) = G <d_alpha F(x_m), d_beta F(x_m')>
 * and K2 = -kappa^-2 G at the interpolation nodes, lo += [K1 mu ; K2 nu] */
static void far_block(const orc_problem *P, int t, int s, const cplx *mom, cplx *loc) {
  int nI = P->nI;
  double ik2 = 1.0 / (P->kappa * P->kappa);
  const cplx *mu = mom + (size_t)s * 3 * nI;
  cplx *lo = loc + (size_t)t * 3 * nI;
  for (int mi = 0; mi < nI; ++mi) {
    const double *gt = P->cgeo + 9 * ((size_t)t * nI + mi);
    for (int mj = 0; mj < nI; ++mj) {
      const double *gs = P->cgeo + 9 * ((size_t)s * nI + mj);
      cplx G = helmholtz(P->kappa, dist3(gt, gs));
      for (int alpha = 0; alpha < 2; ++alpha)
        for (int beta = 0; beta < 2; ++beta) {
          const double *da = gt + 3 + 3 * alpha, *db = gs + 3 + 3 * beta;
          double dot = da[0] * db[0] + da[1] * db[1] + da[2] * db[2];
          lo[alpha * nI + mi] += G * dot * mu[beta * nI + mj];
        }
      lo[2 * nI + mi] += -ik2 * G * mu[2 * nI + mj];
    }
  }
}

/* evaluation of the local fields of the level-l cluster containing e at its test functions */
static void eval_local(const orc_problem *P, int l, int e, const cplx *loc, cplx *ye) {
  int p = P->p, np1 = p + 1, q1 = P->q + 1, nI = P->nI;
  double h = 1.0 / P->n, h2 = h * h;
  const double *M = mom_table(P, 0, l), *Md = mom_table(P, 1, l);
  int sh = P->m - l;
  int j, i1, i2;
  elem_of(P, e, &j, &i1, &i2);
  int id = cl_id(P, l, j, morton(i1 >> sh, i2 >> sh));
  int o1 = i1 - ((i1 >> sh) << sh), o2 = i2 - ((i2 >> sh) << sh);
  const cplx *lo = loc + (size_t)id * 3 * nI;
  for (int alpha = 0; alpha < 2; ++alpha)
    for (int b = 0; b < np1; ++b)
      for (int a = 0; a < np1; ++a) {
        cplx acc = 0;
        for (int m2 = 0; m2 < q1; ++m2)
          for (int m1 = 0; m1 < q1; ++m1) {
            double Ma = M[(o1 * q1 + m1) * np1 + a], Mb = M[(o2 * q1 + m2) * np1 + b];
            double Dda = Md[(o1 * q1 + m1) * np1 + a], Ddb = Md[(o2 * q1 + m2) * np1 + b];
            acc += h2 * Ma * Mb * lo[alpha * nI + m2 * q1 + m1];
            acc += h * (alpha == 0 ? Dda * Mb : Ma * Ddb) * lo[2 * nI + m2 * q1 + m1];
          }
        ye[(alpha * np1 + b) * np1 + a] += acc;
      }
}

/* y* = (N + F) x* in superspace coordinates. */
static void fmm_superspace(orc_problem *P, const cplx *xs, cplx *ys) {
  ensure_near_blocks(P);
  int nb = nb_of(P), nI = P->nI;
  for (int i = 0; i < P->nsup; ++i) ys[i] = 0;
  /* near field */
  for (int k = 0; k < P->nnear; ++k) {
    int e = P->near[2 * k], e2 = P->near[2 * k + 1];
    const cplx *B = P->nblk + (size_t)k * nb * nb;
    for (int r = 0; r < nb; ++r) {
      cplx s = 0;
      for (int c = 0; c < nb; ++c) s += B[r * nb + c] * xs[(size_t)e2 * nb + c];
      ys[(size_t)e * nb + r] += s;
    }
  }
  cplx *mom = direct_moments(P, xs);
  cplx *loc = calloc((size_t)P->ncl * 3 * nI, sizeof(cplx));
  for (int f = 0; f < P->nfar; ++f) far_block(P, P->far[3 * f + 1], P->far[3 * f + 2], mom, loc);
  for (int l = 0; l <= P->m; ++l)
    for (int e = 0; e < P->nE; ++e) eval_local(P, l, e, loc, ys + (size_t)e * nb);
  free(mom);
  free(loc);
}

/* rows of y* = (N + F) x* for selected elements only: near blocks integrated on demand
 * (with_near = 1, else the near part is left out), far field restricted to the blocks whose
 * target cluster contains the element */
static void fmm_rows(orc_problem *P, const double *xsd, int nrows, const int *elems, double *out, int with_near) {
  const cplx *xs = (const cplx *)xsd;
  int nb = nb_of(P), nI = P->nI;
  cplx *o = (cplx *)out;
  regular_cache(P, P->greg);
  cplx *mom = direct_moments(P, xs);
  cplx *loc = calloc((size_t)P->ncl * 3 * nI, sizeof(cplx));
  cplx *blk = malloc(sizeof(cplx) * nb * nb);
  for (int r = 0; r < nrows; ++r) {
    int e = elems[r];
    cplx *ye = o + (size_t)r * nb;
    for (int i = 0; i < nb; ++i) ye[i] = 0;
    for (int k = 0; with_near && k < P->nnear; ++k) {
      if (P->near[2 * k] != e) continue;
      int e2 = P->near[2 * k + 1];
      pair_block(P, e, e2, P->greg, P->gsing, blk);
      for (int i = 0; i < nb; ++i) {
        cplx s = 0;
        for (int c = 0; c < nb; ++c) s += blk[i * nb + c] * xs[(size_t)e2 * nb + c];
        ye[i] += s;
      }
    }
    int j, i1, i2;
    elem_of(P, e, &j, &i1, &i2);
    for (int l = 0; l <= P->m; ++l) {
      int sh = P->m - l, id = cl_id(P, l, j, morton(i1 >> sh, i2 >> sh));
      memset(loc + (size_t)id * 3 * nI, 0, sizeof(cplx) * 3 * nI);
      for (int f = 0; f < P->nfar; ++f)
        if (P->far[3 * f + 1] == id) far_block(P, id, P->far[3 * f + 2], mom, loc);
      eval_local(P, l, e, loc, ye);
    }
  }
  free(blk);
  free(mom);
  free(loc);
}

void orc_fmm_rows(orc_problem *P, const double *xs, int nrows, const int *elems, double *out) {
  fmm_rows(P, xs, nrows, elems, out, 1);
}

void orc_fmm_rows_far(orc_problem *P, const double *xs, int nrows, const int *elems, double *out) {
  fmm_rows(P, xs, nrows, elems, out, 0);
}

void orc_fmm_matvec_superspace(orc_problem *P, const double *xs, double *ys) {
  fmm_superspace(P, (const cplx *)xs, (cplx *)ys);
}

void orc_fmm_matvec(orc_problem *P, int nrhs, const double *x, double *y) {
  cplx *xs = malloc(sizeof(cplx) * P->nsup), *ys = malloc(sizeof(cplx) * P->nsup);
  for (int r = 0; r < nrhs; ++r) {
    apply_T(P, (const cplx *)x + (size_t)r * P->ndof, xs);
    fmm_superspace(P, xs, ys);
    apply_Tt(P, ys, (cplx *)y + (size_t)r * P->ndof);
  }
  free(xs);
  free(ys);
}

/* ------------------------------------------------------------------------------------ */
/* Right-hand side, GMRES, far field, diagnostics                                       */
/* ------------------------------------------------------------------------------------ */

/* g = -T^T g*, g*_{e,alpha,ab} = int_e e_i(F(s)) . d_alpha F(s) psi_ab ds, the tested
 * incident field of eq. linsys (dot-product form of eq. MSLtested). */
void orc_rhs(const orc_problem *P, const double *dir, const double *pol, double *g) {
  int p = P->p, np1 = p + 1, gq = P->greg;
  double gx[64], gw[64], h2 = 1.0 / ((double)P->n * P->n);
  orc_gauss01(gq, gx, gw);
  cplx *gs = calloc(P->nsup, sizeof(cplx));
  for (int e = 0; e < P->nE; ++e)
    for (int u = 0; u < gq; ++u)
      for (int v = 0; v < gq; ++v) {
        double sig[2] = {gx[u], gx[v]}, X[3], D[2][3];
        elem_geo(P, e, sig, X, D[0], D[1]);
        cplx ph = cexp(I * P->kappa * (dir[0] * X[0] + dir[1] * X[1] + dir[2] * X[2]));
        for (int alpha = 0; alpha < 2; ++alpha) {
          double pd = pol[0] * D[alpha][0] + pol[1] * D[alpha][1] + pol[2] * D[alpha][2];
          for (int b = 0; b < np1; ++b)
            for (int a = 0; a < np1; ++a)
              gs[((size_t)(e * 2 + alpha) * np1 + b) * np1 + a] -=
                  gw[u] * gw[v] * h2 * ph * pd * bern(p, a, sig[0]) * bern(p, b, sig[1]);
        }
      }
  apply_Tt(P, gs, (cplx *)g);
  free(gs);
}

static void op_apply(orc_problem *P, int use_fmm, const cplx *x, cplx *y, cplx *Vd) {
  if (use_fmm) {
    orc_fmm_matvec(P, 1, (const double *)x, (double *)y);
  } else {
    int N = P->ndof;
    for (int i = 0; i < N; ++i) {
      cplx s = 0;
      for (int k = 0; k < N; ++k) s += Vd[(size_t)i * N + k] * x[k];
      y[i] = s;
    }
  }
}

static double vnorm(int n, const cplx *v) {
  double s = 0;
  for (int i = 0; i < n; ++i) s += creal(v[i] * conj(v[i]));
  return sqrt(s);
}

/* Restarted complex GMRES (Saad, Alg. 6.9) with modified Gram-Schmidt Arnoldi and
 * Givens rotations, zero initial guess, relative residual ||r|| <= tol ||b||. */
int orc_gmres(orc_problem *P, int use_fmm, const double *bd, double *xd, int restart, double tol,
              int maxit, int *its_out, double *relres) {
  int N = P->ndof, k = restart;
  const cplx *b = (const cplx *)bd;
  cplx *x = (cplx *)xd;
  cplx *Vd = NULL;
  if (!use_fmm) {
    /* dense Galerkin matrix A = T^T V* T of eq. superspace */
    int S = P->nsup;
    cplx *Vs = malloc(sizeof(cplx) * (size_t)S * S);
    orc_dense_superspace(P, (double *)Vs);
    cplx *VT = calloc((size_t)S * N, sizeof(cplx)); /* V* T */
    for (int t = 0; t < P->nT; ++t)
      for (int i = 0; i < S; ++i) VT[(size_t)i * N + P->Tcol[t]] += Vs[(size_t)i * S + P->Trow[t]] * P->Tval[t];
    Vd = calloc((size_t)N * N, sizeof(cplx));
    for (int t = 0; t < P->nT; ++t)
      for (int j = 0; j < N; ++j) Vd[(size_t)P->Tcol[t] * N + j] += P->Tval[t] * VT[(size_t)P->Trow[t] * N + j];
    free(Vs);
    free(VT);
  }
  cplx *V = malloc(sizeof(cplx) * (size_t)(k + 1) * N);
  cplx *H = calloc((size_t)(k + 1) * k, sizeof(cplx));
  double *cs = malloc(sizeof(double) * k);
  cplx *sn = malloc(sizeof(cplx) * k), *gv = malloc(sizeof(cplx) * (k + 1)), *yv = malloc(sizeof(cplx) * k);
  cplx *w = malloc(sizeof(cplx) * N), *r = malloc(sizeof(cplx) * N);
  double bn = vnorm(N, b);
  int its = 0, conv = 0;
  for (int i = 0; i < N; ++i) x[i] = 0;
  double res = bn;
  if (bn == 0.0) conv = 1;
  while (!conv && its < maxit) {
    op_apply(P, use_fmm, x, w, Vd);
    for (int i = 0; i < N; ++i) r[i] = b[i] - w[i];
    double beta = vnorm(N, r);
    res = beta;
    if (beta <= tol * bn) {
      conv = 1;
      break;
    }
    for (int i = 0; i < N; ++i) V[i] = r[i] / beta;
    for (int i = 0; i <= k; ++i) gv[i] = 0;
    gv[0] = beta;
    int j = 0;
    for (; j < k && its < maxit; ++j) {
      op_apply(P, use_fmm, V + (size_t)j * N, w, Vd);
      ++its;
      for (int i = 0; i <= j; ++i) {
        cplx hij = 0;
        for (int t = 0; t < N; ++t) hij += conj(V[(size_t)i * N + t]) * w[t];
        H[i * k + j] = hij;
        for (int t = 0; t < N; ++t) w[t] -= hij * V[(size_t)i * N + t];
      }
      double hn = vnorm(N, w);
      H[(j + 1) * k + j] = hn;
      for (int t = 0; t < N; ++t) V[(size_t)(j + 1) * N + t] = hn > 0 ? w[t] / hn : 0;
      for (int i = 0; i < j; ++i) {
        cplx a = H[i * k + j], c = H[(i + 1) * k + j];
        H[i * k + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * k + j] = -conj(sn[i]) * a + cs[i] * c;
      }
      cplx a = H[j * k + j];
      double bb = hn, aa = cabs(a), tt = sqrt(aa * aa + bb * bb);
      if (aa == 0.0) {
        cs[j] = 0.0;
        sn[j] = 1.0;
      } else {
        cs[j] = aa / tt;
        sn[j] = (a / aa) * bb / tt;
      }
      H[j * k + j] = cs[j] * a + sn[j] * bb;
      H[(j + 1) * k + j] = 0;
      gv[j + 1] = -conj(sn[j]) * gv[j];
      gv[j] = cs[j] * gv[j];
      res = cabs(gv[j + 1]);
      if (res <= tol * bn) {
        ++j;
        break;
      }
    }
    for (int i = j - 1; i >= 0; --i) {
      cplx s = gv[i];
      for (int t = i + 1; t < j; ++t) s -= H[i * k + t] * yv[t];
      yv[i] = s / H[i * k + i];
    }
    for (int i = 0; i < j; ++i)
      for (int t = 0; t < N; ++t) x[t] += yv[i] * V[(size_t)i * N + t];
    if (res <= tol * bn) {
      op_apply(P, use_fmm, x, w, Vd);
      for (int i = 0; i < N; ++i) r[i] = b[i] - w[i];
      res = vnorm(N, r);
      if (res <= tol * bn * 1.01) conv = 1;
    }
  }
  if (its_out) *its_out = its;
  if (relres) *relres = bn > 0 ? res / bn : 0.0;
  free(V);
  free(H);
  free(cs);
  free(sn);
  free(gv);
  free(yv);
  free(w);
  free(r);
  free(Vd);
  return conv ? 0 : 1;
}

/* Far field of the electric single-layer potential (eq. ESLP): with
 * W(d) = int w(y) exp(-i kappa d.y) dsigma_y, E_inf(d) = (1/4pi) (W - d (d.W)).  On the
 * patch, w dsigma = dF w_hat ds (Piola transform iota_1). */
void orc_far_field(const orc_problem *P, const double *coef, int ndir, const double *dirs,
                   double *out) {
  int p = P->p, np1 = p + 1, gq = P->greg;
  double gx[64], gw[64], h2 = 1.0 / ((double)P->n * P->n);
  orc_gauss01(gq, gx, gw);
  cplx *xs = malloc(sizeof(cplx) * P->nsup);
  apply_T(P, (const cplx *)coef, xs);
  cplx *o = (cplx *)out;
  for (int dd = 0; dd < ndir; ++dd) {
    const double *d = dirs + 3 * dd;
    cplx W[3] = {0, 0, 0};
    for (int e = 0; e < P->nE; ++e)
      for (int u = 0; u < gq; ++u)
        for (int v = 0; v < gq; ++v) {
          double sig[2] = {gx[u], gx[v]}, X[3], D[2][3];
          elem_geo(P, e, sig, X, D[0], D[1]);
          cplx ph = cexp(-I * P->kappa * (d[0] * X[0] + d[1] * X[1] + d[2] * X[2])) * gw[u] * gw[v] * h2;
          for (int alpha = 0; alpha < 2; ++alpha) {
            cplx wa = 0;
            for (int b = 0; b < np1; ++b)
              for (int a = 0; a < np1; ++a)
                wa += xs[((size_t)(e * 2 + alpha) * np1 + b) * np1 + a] * bern(p, a, sig[0]) * bern(p, b, sig[1]);
            for (int c = 0; c < 3; ++c) W[c] += ph * D[alpha][c] * wa;
          }
        }
    cplx dw = d[0] * W[0] + d[1] * W[1] + d[2] * W[2];
    for (int c = 0; c < 3; ++c) o[3 * dd + c] = (W[c] - d[c] * dw) / (4.0 * M_PI);
  }
  free(xs);
}

/* Hertz dipole at x0 with moment p0 (Sec. 5.2, "The Electric Field as a Quantity of
 * Interest", after Jackson (9.18) without the 1/(4 pi eps0) factor):
 *   E(x) = e^{i kappa r} ( kappa^2/r (n x p0) x n + (1/r^3 - i kappa/r^2)(3 n (n.p0) - p0) ),
 * r = |x - x0|, n = (x - x0)/r.  It solves curl curl E - kappa^2 E = 0 away from x0. */
static void dipole_at(double kappa, const double *x0, const double *p0, const double *x, cplx *E) {
  double d[3] = {x[0] - x0[0], x[1] - x0[1], x[2] - x0[2]};
  double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double n[3] = {d[0] / r, d[1] / r, d[2] / r};
  double np = n[0] * p0[0] + n[1] * p0[1] + n[2] * p0[2];
  /* (n x p0) x n = p0 - n (n.p0) */
  cplx ph = cexp(I * kappa * r);
  cplx a = kappa * kappa / r, b = 1.0 / (r * r * r) - I * kappa / (r * r);
  for (int c = 0; c < 3; ++c) E[c] = ph * (a * (p0[c] - n[c] * np) + b * (3.0 * n[c] * np - p0[c]));
}

void orc_dipole_field(double kappa, const double *x0, const double *p0, int npts, const double *x, double *out) {
  cplx *o = (cplx *)out;
  for (int k = 0; k < npts; ++k) dipole_at(kappa, x0, p0, x + 3 * k, o + 3 * k);
}

/* Right-hand side for the incident field e_i = -DP_{x0,p0}: g = -T^T int e_i . phi, i.e.
 * +T^T int DP . phi, so that the scattered field outside is the dipole field itself (the
 * manufactured solution of Sec. 5.2; the dipole sits inside the scatterer). */
void orc_rhs_dipole(const orc_problem *P, const double *x0, const double *p0, double *g) {
  int p = P->p, np1 = p + 1, gq = P->greg;
  double gx[64], gw[64], h2 = 1.0 / ((double)P->n * P->n);
  orc_gauss01(gq, gx, gw);
  cplx *gs = calloc(P->nsup, sizeof(cplx));
  for (int e = 0; e < P->nE; ++e)
    for (int u = 0; u < gq; ++u)
      for (int v = 0; v < gq; ++v) {
        double sig[2] = {gx[u], gx[v]}, X[3], D[2][3];
        cplx E[3];
        elem_geo(P, e, sig, X, D[0], D[1]);
        dipole_at(P->kappa, x0, p0, X, E);
        for (int alpha = 0; alpha < 2; ++alpha) {
          cplx ed = E[0] * D[alpha][0] + E[1] * D[alpha][1] + E[2] * D[alpha][2];
          for (int b = 0; b < np1; ++b)
            for (int a = 0; a < np1; ++a)
              gs[((size_t)(e * 2 + alpha) * np1 + b) * np1 + a] +=
                  gw[u] * gw[v] * h2 * ed * bern(p, a, sig[0]) * bern(p, b, sig[1]);
        }
      }
  apply_Tt(P, gs, (cplx *)g);
  free(gs);
}

/* Electric single-layer potential (eq. ESLP) at points off the surface:
 *   E(x) = int G(x-y) w(y) dsigma_y + kappa^-2 grad_x int G(x-y) div_Gamma w(y) dsigma_y,
 * G of eq. HelmholtzGreen, grad_x G(x-y) = G(x-y) (i kappa - 1/R) (x-y)/R, R = |x-y|.  On a
 * patch w dsigma = dF w_hat ds and div_Gamma w dsigma = div w_hat ds (Piola transforms);
 * tensor Gauss with quad_regular points per element direction (the points are assumed well
 * separated from the surface).  out [npts][3] complex. */
void orc_exterior_field(const orc_problem *P, const double *coef, int npts, const double *xp, double *out) {
  int p = P->p, np1 = p + 1, gq = P->greg;
  double gx[64], gw[64], h = 1.0 / P->n, h2 = h * h;
  orc_gauss01(gq, gx, gw);
  cplx *xs = malloc(sizeof(cplx) * P->nsup);
  apply_T(P, (const cplx *)coef, xs);
  cplx *o = (cplx *)out;
  double k2 = P->kappa * P->kappa;
  for (int k = 0; k < npts; ++k) {
    const double *x = xp + 3 * k;
    cplx Ev[3] = {0, 0, 0}, Ed[3] = {0, 0, 0};
    for (int e = 0; e < P->nE; ++e)
      for (int u = 0; u < gq; ++u)
        for (int v = 0; v < gq; ++v) {
          double sig[2] = {gx[u], gx[v]}, X[3], D[2][3];
          elem_geo(P, e, sig, X, D[0], D[1]);
          double d[3] = {x[0] - X[0], x[1] - X[1], x[2] - X[2]};
          double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
          cplx G = cexp(I * P->kappa * R) / (4.0 * M_PI * R);
          cplx w[2] = {0, 0}, dv = 0;
          for (int alpha = 0; alpha < 2; ++alpha)
            for (int b = 0; b < np1; ++b)
              for (int a = 0; a < np1; ++a) {
                cplx c = xs[((size_t)(e * 2 + alpha) * np1 + b) * np1 + a];
                w[alpha] += c * bern(p, a, sig[0]) * bern(p, b, sig[1]);
                dv += c * (alpha == 0 ? bern_d(p, a, sig[0]) * bern(p, b, sig[1])
                                      : bern(p, a, sig[0]) * bern_d(p, b, sig[1]));
              }
          /* vector part: h^2 ds weight; divergence part: div in patch coordinates is (1/h)
           * times the element-local derivative, times h^2 */
          cplx gv = gw[u] * gw[v] * h2 * G, gd = gw[u] * gw[v] * h * G * (I * P->kappa - 1.0 / R) / R;
          for (int c = 0; c < 3; ++c) {
            Ev[c] += gv * (D[0][c] * w[0] + D[1][c] * w[1]);
            Ed[c] += gd * d[c] * dv;
          }
        }
    for (int c = 0; c < 3; ++c) o[3 * k + c] = Ev[c] + Ed[c] / k2;
  }
  free(xs);
}

/* int_Gamma div_Gamma w dsigma = sum_e int_e div w_hat ds (iota_2 cancels tau). */
void orc_div_integral(const orc_problem *P, const double *coef, double *out2) {
  int p = P->p, np1 = p + 1, gq = P->greg;
  double gx[64], gw[64], h = 1.0 / P->n;
  orc_gauss01(gq, gx, gw);
  cplx *xs = malloc(sizeof(cplx) * P->nsup);
  apply_T(P, (const cplx *)coef, xs);
  cplx s = 0;
  for (int e = 0; e < P->nE; ++e)
    for (int u = 0; u < gq; ++u)
      for (int v = 0; v < gq; ++v)
        for (int alpha = 0; alpha < 2; ++alpha)
          for (int b = 0; b < np1; ++b)
            for (int a = 0; a < np1; ++a) {
              double d = alpha == 0 ? bern_d(p, a, gx[u]) * bern(p, b, gx[v]) : bern(p, a, gx[u]) * bern_d(p, b, gx[v]);
              s += gw[u] * gw[v] * h * d * xs[((size_t)(e * 2 + alpha) * np1 + b) * np1 + a];
            }
  out2[0] = creal(s);
  out2[1] = cimag(s);
  free(xs);
}

double orc_area(const orc_problem *P) {
  int gq = P->greg;
  double gx[64], gw[64], h2 = 1.0 / ((double)P->n * P->n), A = 0;
  orc_gauss01(gq, gx, gw);
  for (int e = 0; e < P->nE; ++e)
    for (int u = 0; u < gq; ++u)
      for (int v = 0; v < gq; ++v) {
        double sig[2] = {gx[u], gx[v]}, X[3], D[2][3];
        elem_geo(P, e, sig, X, D[0], D[1]);
        double nx = D[0][1] * D[1][2] - D[0][2] * D[1][1], ny = D[0][2] * D[1][0] - D[0][0] * D[1][2],
               nz = D[0][0] * D[1][1] - D[0][1] * D[1][0];
        A += gw[u] * gw[v] * h2 * sqrt(nx * nx + ny * ny + nz * nz);
      }
  return A;
}

/* ------------------------------------------------------------------------------------ */
/* Mie series for the PEC sphere (textbook vector spherical harmonics expansion with     */
/* time convention exp(-i omega t); incident field x exp(i kappa z))                     */
/* ------------------------------------------------------------------------------------ */

/* spherical Bessel j_n (downward recurrence normalised by j_0) and y_n (upward) */
static void sph_bessel(int nmax, double x, double *j, double *y) {
  int start = nmax + 40 + (int)x;
  double *f = malloc(sizeof(double) * (start + 2));
  f[start + 1] = 0.0;
  f[start] = 1e-300;
  for (int k = start; k >= 1; --k) {
    f[k - 1] = (2.0 * k + 1.0) / x * f[k] - f[k + 1];
    if (fabs(f[k - 1]) > 1e250) {
      for (int t = k - 1; t <= start + 1; ++t) f[t] *= 1e-250;
    }
  }
  double j0 = sin(x) / x, sc = j0 / f[0];
  for (int k = 0; k <= nmax; ++k) j[k] = f[k] * sc;
  free(f);
  y[0] = -cos(x) / x;
  if (nmax >= 1) y[1] = -cos(x) / (x * x) - sin(x) / x;
  for (int k = 1; k < nmax; ++k) y[k + 1] = (2.0 * k + 1.0) / x * y[k] - y[k - 1];
}

void orc_mie_field(double kappa, double radius, int which, int npts, const double *xp,
                   double *out) {
  cplx *o = (cplx *)out;
  double xa = kappa * radius;
  for (int ip = 0; ip < npts; ++ip) {
    const double *P = xp + 3 * ip;
    double r = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    double ct = P[2] / r, st = sqrt(fmax(0.0, 1.0 - ct * ct)), ph = atan2(P[1], P[0]);
    double cp = cos(ph), sp = sin(ph);
    double rho = which == 4 ? kappa : kappa * r;
    /* scattering coefficients vanish super-exponentially beyond n ~ kappa a; the
     * incident expansion at radius r needs n ~ kappa r terms */
    int nsca = (int)(xa + 4.0 * cbrt(xa) + 20.0);
    int nmax = which == 4 ? nsca : (int)(fmax(rho, xa) + 4.0 * cbrt(fmax(rho, xa)) + 20.0);
    if (which == 1 && nmax > nsca) nmax = nsca;
    double *jr = malloc(sizeof(double) * (nmax + 2)), *yr = malloc(sizeof(double) * (nmax + 2));
    double *ja = malloc(sizeof(double) * (nsca + 2)), *ya = malloc(sizeof(double) * (nsca + 2));
    sph_bessel(nmax + 1, rho, jr, yr);
    sph_bessel(nsca + 1, xa, ja, ya);
    cplx Er = 0, Et = 0, Ep = 0; /* components in (r, theta, phi) */
    double pi_nm1 = 0.0, pi_n = 1.0; /* pi_0, pi_1 (angular functions pi_n = P_n^1 / sin) */
    for (int n = 1; n <= nmax; ++n) {
      if (n >= 2) {
        double nxt = (2.0 * n - 1.0) / (n - 1.0) * ct * pi_n - (double)n / (n - 1.0) * pi_nm1;
        pi_nm1 = pi_n;
        pi_n = nxt;
      }
      double tau_n = n * ct * pi_n - (n + 1.0) * pi_nm1;
      cplx En = cpow(I, n) * (2.0 * n + 1.0) / (n * (n + 1.0));
      /* radial functions at r: z = j (type 1) or h = j + i y (type 3) */
      cplx z1 = jr[n], z3 = jr[n] + I * yr[n];
      cplx dz1 = (rho * jr[n - 1] - n * jr[n]) / rho;
      cplx dz3 = (rho * (jr[n - 1] + I * yr[n - 1]) - n * (jr[n] + I * yr[n])) / rho;
      cplx an = 0, bn = 0;
      if (n <= nsca) {
        cplx hA = ja[n] + I * ya[n];
        cplx dxjA = xa * ja[n - 1] - n * ja[n];
        cplx dxhA = xa * (ja[n - 1] + I * ya[n - 1]) - n * hA;
        an = dxjA / dxhA;
        bn = ja[n] / hA;
      }
      /* M_o1n, M_e1n, N_o1n, N_e1n in (r, theta, phi) */
      cplx Mo1[3] = {0, cp * pi_n * z1, -sp * tau_n * z1};
      cplx Me1[3] = {0, -sp * pi_n * z1, -cp * tau_n * z1};
      cplx No1[3] = {sp * n * (n + 1.0) * st * pi_n * z1 / rho, sp * tau_n * dz1, cp * pi_n * dz1};
      cplx Ne1[3] = {cp * n * (n + 1.0) * st * pi_n * z1 / rho, cp * tau_n * dz1, -sp * pi_n * dz1};
      cplx Mo3[3] = {0, cp * pi_n * z3, -sp * tau_n * z3};
      cplx Me3[3] = {0, -sp * pi_n * z3, -cp * tau_n * z3};
      cplx No3[3] = {sp * n * (n + 1.0) * st * pi_n * z3 / rho, sp * tau_n * dz3, cp * pi_n * dz3};
      cplx Ne3[3] = {cp * n * (n + 1.0) * st * pi_n * z3 / rho, cp * tau_n * dz3, -sp * pi_n * dz3};
      if (which == 4) {
        /* far-field amplitude: h_n(rho) ~ (-i)^(n+1) e^{i rho}/rho and
         * [rho h_n]'/rho ~ (-i)^n e^{i rho}/rho, radial parts decay faster */
        cplx zf = cpow(-I, n + 1) / kappa, dzf = cpow(-I, n) / kappa;
        cplx Mo[3] = {0, cp * pi_n * zf, -sp * tau_n * zf};
        cplx Ne[3] = {0, cp * tau_n * dzf, -sp * pi_n * dzf};
        for (int c = 0; c < 3; ++c) {
          cplx v = En * (I * an * Ne[c] - bn * Mo[c]);
          if (c == 1) Et += v;
          if (c == 2) Ep += v;
        }
        continue;
      }
      cplx F[3] = {0, 0, 0};
      for (int c = 0; c < 3; ++c) {
        cplx inc = Mo1[c] - I * Ne1[c];
        cplx sca = I * an * Ne3[c] - bn * Mo3[c];
        cplx cinc = kappa * (No1[c] - I * Me1[c]);
        cplx csca = kappa * (I * an * Me3[c] - bn * No3[c]);
        if (which == 0) F[c] = inc;
        else if (which == 1) F[c] = sca;
        else F[c] = cinc + csca;
      }
      Er += En * F[0];
      Et += En * F[1];
      Ep += En * F[2];
    }
    free(jr);
    free(yr);
    free(ja);
    free(ya);
    if (which == 3) { /* n x (curl E) with n = r_hat: r x theta = phi, r x phi = -theta */
      cplx t = Et;
      Et = -Ep;
      Ep = t;
      Er = 0;
    }
    double rh[3] = {st * cp, st * sp, ct}, th[3] = {ct * cp, ct * sp, -st}, phv[3] = {-sp, cp, 0};
    for (int c = 0; c < 3; ++c) o[3 * ip + c] = Er * rh[c] + Et * th[c] + Ep * phv[c];
  }
}

/* L2 error of the density against the Mie current (the error measure of the Mie
 * experiment, Sec. 5.1): w_h = dF w_hat / tau on the patch. */
void orc_mie_l2(const orc_problem *P, const double *coef, double radius, double *out) {
  int p = P->p, np1 = p + 1, gq = P->greg;
  double gx[64], gw[64], h2 = 1.0 / ((double)P->n * P->n);
  orc_gauss01(gq, gx, gw);
  cplx *xs = malloc(sizeof(cplx) * P->nsup);
  apply_T(P, (const cplx *)coef, xs);
  double err = 0, nrm = 0;
  for (int e = 0; e < P->nE; ++e)
    for (int u = 0; u < gq; ++u)
      for (int v = 0; v < gq; ++v) {
        double sig[2] = {gx[u], gx[v]}, X[3], D[2][3];
        elem_geo(P, e, sig, X, D[0], D[1]);
        double nx = D[0][1] * D[1][2] - D[0][2] * D[1][1], ny = D[0][2] * D[1][0] - D[0][0] * D[1][2],
               nz = D[0][0] * D[1][1] - D[0][1] * D[1][0];
        double tau = sqrt(nx * nx + ny * ny + nz * nz);
        cplx wa[2] = {0, 0};
        for (int alpha = 0; alpha < 2; ++alpha)
          for (int b = 0; b < np1; ++b)
            for (int a = 0; a < np1; ++a)
              wa[alpha] += xs[((size_t)(e * 2 + alpha) * np1 + b) * np1 + a] * bern(p, a, sig[0]) * bern(p, b, sig[1]);
        double ex[6];
        orc_mie_field(P->kappa, radius, 3, 1, X, ex);
        cplx wm[3] = {ex[0] + I * ex[1], ex[2] + I * ex[3], ex[4] + I * ex[5]};
        double wt = gw[u] * gw[v] * h2 * tau;
        for (int c = 0; c < 3; ++c) {
          cplx wh = (D[0][c] * wa[0] + D[1][c] * wa[1]) / tau;
          err += wt * creal((wh - wm[c]) * conj(wh - wm[c]));
          nrm += wt * creal(wm[c] * conj(wm[c]));
        }
      }
  out[0] = sqrt(err);
  out[1] = sqrt(nrm);
  free(xs);
}
