// Host-side index structures of the GB300 EFIE library: the multipatch S^1 DOF map and the
// superspace transformation T (Sec. 3.2, Sec. 4.1 eq. superspace), the quadtree cluster
// tree and the block-cluster tree of Algorithm 1 (Sec. 4.2), and the classification of
// near-field element pairs for the singular quadrature.  No floating-point work of the
// operator itself happens here; geometry values come from the device evaluator.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "efie_internal.h"

namespace efie {

// ---------------------------------------------------------------------------------------
// small 1-D tools

// Gauss-Legendre nodes / weights on [0,1]: Newton iteration on P_g started from the
// asymptotic guess, derivative from the standard identity (1 - t^2) P_g' = g (P_{g-1} - t P_g).
void gauss_legendre01(int g, std::vector<double> &x, std::vector<double> &w) {
  x.assign(g, 0.0);
  w.assign(g, 0.0);
  for (int i = 0; i < g; ++i) {
    double t = std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * g + 2.0));
    double Pg = 0, Pm = 0;
    for (int it = 0; it < 60; ++it) {
      double a = 1.0, b = t;  // P_0, P_1
      if (g == 1) { Pm = 1.0; Pg = t; }
      for (int k = 2; k <= g; ++k) {
        double c2 = ((2 * k - 1) * t * b - (k - 1) * a) / k;
        a = b;
        b = c2;
      }
      if (g >= 2) { Pm = a; Pg = b; }
      double dP = g * (Pm - t * Pg) / (1.0 - t * t);
      double step = Pg / dP;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    double a = 1.0, b = t;
    for (int k = 2; k <= g; ++k) {
      double c2 = ((2 * k - 1) * t * b - (k - 1) * a) / k;
      a = b;
      b = c2;
    }
    if (g == 1) { a = 1.0; b = t; }
    double dP = g * (a - t * b) / (1.0 - t * t);
    // node on [0,1] in ascending order
    x[i] = 0.5 * (1.0 - t);
    w[i] = 1.0 / ((1.0 - t * t) * dP * dP);
  }
}

static double bernstein(int p, int a, double t) {
  double c = 1.0;
  for (int i = 0; i < a; ++i) c = c * (p - i) / (i + 1);
  double v = c;
  for (int i = 0; i < a; ++i) v *= t;
  for (int i = 0; i < p - a; ++i) v *= (1.0 - t);
  return v;
}
static double bernstein_d(int p, int a, double t) {
  if (p == 0) return 0.0;
  double l = a >= 1 ? bernstein(p - 1, a - 1, t) : 0.0;
  double r = a <= p - 1 ? bernstein(p - 1, a, t) : 0.0;
  return p * (l - r);
}

// The deg+1 B-splines that do not vanish on knot span [kn[span], kn[span+1]), evaluated
// at x by the triangular Cox-de Boor scheme; N[i] belongs to function span - deg + i.
static void bspline_nonzero(const std::vector<double> &kn, int deg, int span, double x, double *N) {
  double cur[16], nxt[16];
  cur[0] = 1.0;
  for (int d = 1; d <= deg; ++d) {
    for (int i = 0; i <= d; ++i) {
      int f = span - d + i;
      double v = 0.0;
      if (i >= 1) {
        double den = kn[f + d] - kn[f];
        if (den > 0) v += (x - kn[f]) / den * cur[i - 1];
      }
      if (i <= d - 1) {
        double den = kn[f + d + 1] - kn[f + 1];
        if (den > 0) v += (kn[f + d + 1] - x) / den * cur[i];
      }
      nxt[i] = v;
    }
    for (int i = 0; i <= d; ++i) cur[i] = nxt[i];
  }
  for (int i = 0; i <= deg; ++i) N[i] = cur[i];
}

// Chebyshev nodes of the first kind on [0,1] (ascending) and Lagrange basis.
static double lagr(const std::vector<double> &xs, int m, double t) {
  double v = 1.0;
  for (size_t k = 0; k < xs.size(); ++k)
    if ((int)k != m) v *= (t - xs[k]) / (xs[m] - xs[k]);
  return v;
}

void host_tables(Ctx *c) {
  Tables &T = c->tab;
  int q1 = c->q1, p1 = c->p1, p = c->p;
  T.xcheb.resize(q1);
  for (int i = 0; i < q1; ++i) T.xcheb[i] = 0.5 - 0.5 * std::cos(M_PI * (2 * i + 1) / (2.0 * q1));
  // moments are polynomials of degree q + p: exact with ceil((q+p+1)/2) + 1 points
  std::vector<double> gx, gw;
  gauss_legendre01((c->q + p + 2) / 2 + 1, gx, gw);
  T.M.assign(q1 * p1, 0.0);
  T.Md.assign(q1 * p1, 0.0);
  for (int mi = 0; mi < q1; ++mi)
    for (int a = 0; a < p1; ++a) {
      double s = 0, sd = 0;
      for (size_t k = 0; k < gx.size(); ++k) {
        double L = lagr(T.xcheb, mi, gx[k]);
        s += gw[k] * L * bernstein(p, a, gx[k]);
        sd += gw[k] * L * bernstein_d(p, a, gx[k]);
      }
      T.M[mi * p1 + a] = s;
      T.Md[mi * p1 + a] = sd;
    }
  T.E.assign(2 * q1 * q1, 0.0);
  for (int ch = 0; ch < 2; ++ch)
    for (int mi = 0; mi < q1; ++mi)
      for (int mj = 0; mj < q1; ++mj) T.E[(ch * q1 + mi) * q1 + mj] = lagr(T.xcheb, mi, 0.5 * (ch + T.xcheb[mj]));
  gauss_legendre01(c->gr, T.gx, T.gw);
  gauss_legendre01(c->gs, T.sx, T.sw);
}

// ---------------------------------------------------------------------------------------
// DOF map and T

static int edge_sign(int k) { return (k == 1 || k == 3) ? 1 : -1; }  // W,E,S,N = 0,1,2,3

static double pdist(const double *a, const double *b) {
  double s = 0;
  for (int k = 0; k < 3; ++k) s += (a[k] - b[k]) * (a[k] - b[k]);
  return std::sqrt(s);
}

static double geometry_tolerance(const Ctx *c) {
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (size_t i = 0; i < c->cpw.size() / 4; ++i)
    for (int k = 0; k < 3; ++k) {
      double v = c->cpw[4 * i + k] / c->cpw[4 * i + 3];
      lo[k] = std::min(lo[k], v);
      hi[k] = std::max(hi[k], v);
    }
  return 1e-9 * pdist(lo, hi);
}

// edge_pts: [np][4 edges][5 samples][3] at t = 0, 1/4, 1/2, 3/4, 1 along W(s1=0),
// E(s1=1), S(s2=0), N(s2=1), parametrised by the free coordinate.
efie_status host_build_space(Ctx *c, const std::vector<double> &edge_pts, const std::vector<double> & /*corner*/) {
  const int np = c->np, n = c->n, p = c->p, p1 = c->p1;
  const double tol = geometry_tolerance(c);
  c->edge_nbr.assign(np * 4 * 3, -1);
  for (int a = 0; a < np * 4; ++a) {
    int hits = 0;
    for (int b = 0; b < np * 4; ++b) {
      if (a == b) continue;
      for (int rev = 0; rev < 2; ++rev) {
        bool ok = true;
        for (int t = 0; t < 5 && ok; ++t)
          ok = pdist(&edge_pts[(a * 5 + t) * 3], &edge_pts[(b * 5 + (rev ? 4 - t : t)) * 3]) < tol;
        if (ok) {
          c->edge_nbr[a * 3] = b / 4;
          c->edge_nbr[a * 3 + 1] = b % 4;
          c->edge_nbr[a * 3 + 2] = rev;
          ++hits;
        }
      }
    }
    if (hits != 1) {
      c->err = "patch " + std::to_string(a / 4) + " edge " + std::to_string(a % 4) +
               " has " + std::to_string(hits) + " matching neighbour edges (need exactly 1)";
      return EFIE_EGEOMETRY;
    }
  }
  // consistent orientation: a shared edge is traversed in opposite directions by the
  // counter-clockwise boundaries of the two patches (S, E: +t; N, W: -t)
  for (int a = 0; a < np * 4; ++a) {
    int k = a % 4, k2 = c->edge_nbr[a * 3 + 1], rev = c->edge_nbr[a * 3 + 2];
    int da = (k == 1 || k == 2) ? 1 : -1, db = (k2 == 1 || k2 == 2) ? 1 : -1;
    if (da * db * (rev ? -1 : 1) != -1) {
      c->err = "patches " + std::to_string(a / 4) + " and " + std::to_string(c->edge_nbr[a * 3]) +
               " are not consistently oriented";
      return EFIE_EGEOMETRY;
    }
  }

  // patch-local S^1 functions: component 0 has (n+p) x (n+p-1), component 1 (n+p-1) x (n+p)
  const int nA = (n + p) * (n + p - 1), nloc = 2 * nA;
  auto local = [&](int comp, int i1, int i2) {
    return comp == 0 ? i2 * (n + p) + i1 : nA + i2 * (n + p - 1) + i1;
  };
  // partner of an edge function: (flat index, sign) or (-1, 0)
  auto partner = [&](int j, int comp, int i1, int i2, int &sgn) -> int {
    int k = -1, pos = 0;
    if (comp == 0 && i1 == 0) { k = 0; pos = i2; }
    else if (comp == 0 && i1 == n + p - 1) { k = 1; pos = i2; }
    else if (comp == 1 && i2 == 0) { k = 2; pos = i1; }
    else if (comp == 1 && i2 == n + p - 1) { k = 3; pos = i1; }
    if (k < 0) return -1;
    const int *nb = &c->edge_nbr[(j * 4 + k) * 3];
    int j2 = nb[0], k2 = nb[1], pp = nb[2] ? (n + p - 2 - pos) : pos;
    sgn = -edge_sign(k) * edge_sign(k2);
    int l2 = (k2 < 2) ? local(0, k2 == 0 ? 0 : n + p - 1, pp) : local(1, pp, k2 == 2 ? 0 : n + p - 1);
    return j2 * nloc + l2;
  };
  std::vector<int> dof(np * nloc, -1);
  std::vector<signed char> sg(np * nloc, 1);
  int nd = 0;
  for (int j = 0; j < np; ++j)
    for (int comp = 0; comp < 2; ++comp) {
      int e1 = comp == 0 ? n + p : n + p - 1, e2 = comp == 0 ? n + p - 1 : n + p;
      for (int i2 = 0; i2 < e2; ++i2)
        for (int i1 = 0; i1 < e1; ++i1) {
          int self = j * nloc + local(comp, i1, i2);
          int s = 1;
          int other = partner(j, comp, i1, i2, s);
          if (other >= 0 && other < self) {  // numbered where it first occurred
            dof[self] = dof[other];
            sg[self] = (signed char)s;
          } else {
            dof[self] = nd++;
            sg[self] = 1;
          }
        }
    }
  c->ndof = nd;

  // Bezier extraction by L2 projection onto the Bernstein basis of each element:
  // G c = r with G_ab = int B_a B_b, r_a = int B_a b_f (exact Gauss with p+1 points).
  std::vector<double> kn(n + 2 * p + 1), knq(n + 2 * p - 1);
  for (int i = 0; i < (int)kn.size(); ++i) kn[i] = std::min(1.0, std::max(0.0, double(i - p) / n));
  for (int i = 0; i < (int)knq.size(); ++i) knq[i] = kn[i + 1];
  std::vector<double> gx, gw;
  gauss_legendre01(p1, gx, gw);
  auto extract = [&](const std::vector<double> &kv, int deg, std::vector<double> &C) {
    // C[(k * p1 + a) * p1 + r]: coefficient of B_a in function k + r on element k
    C.assign((size_t)n * p1 * p1, 0.0);
    for (int k = 0; k < n; ++k) {
      double G[kMaxP1 * kMaxP1] = {0}, R[kMaxP1 * kMaxP1] = {0};
      for (int g = 0; g < p1; ++g) {
        double N[16];
        bspline_nonzero(kv, deg, k + deg, (k + gx[g]) / n, N);
        for (int a = 0; a < p1; ++a) {
          double Ba = bernstein(p, a, gx[g]);
          for (int b = 0; b < p1; ++b) G[a * p1 + b] += gw[g] * Ba * bernstein(p, b, gx[g]);
          for (int r = 0; r <= deg; ++r) R[a * p1 + r] += gw[g] * Ba * N[r];
        }
      }
      // Cholesky-free solve: Gauss-Jordan on the small SPD Gram matrix
      for (int col = 0; col < p1; ++col) {
        double piv = G[col * p1 + col];
        for (int t = 0; t < p1; ++t) {
          G[col * p1 + t] /= piv;
          R[col * p1 + t] /= piv;
        }
        for (int row = 0; row < p1; ++row) {
          if (row == col) continue;
          double f = G[row * p1 + col];
          for (int t = 0; t < p1; ++t) {
            G[row * p1 + t] -= f * G[col * p1 + t];
            R[row * p1 + t] -= f * R[col * p1 + t];
          }
        }
      }
      for (int a = 0; a < p1; ++a)
        for (int r = 0; r <= deg; ++r) {
          double v = R[a * p1 + r];
          C[((size_t)k * p1 + a) * p1 + r] = std::fabs(v) < 1e-14 ? 0.0 : v;
        }
    }
  };
  std::vector<double> Cp, Cq;
  extract(kn, p, Cp);
  extract(knq, p - 1, Cq);

  std::vector<int> rows, cols;
  std::vector<double> vals;
  const int n2 = n * n;
  for (int e = 0; e < c->nE; ++e) {
    int j = e / n2, i1, i2;
    unmorton2(e % n2, i1, i2);
    for (int comp = 0; comp < 2; ++comp) {
      int d1 = comp == 0 ? p : p - 1, d2 = comp == 0 ? p - 1 : p;
      const std::vector<double> &C1 = comp == 0 ? Cp : Cq;
      const std::vector<double> &C2 = comp == 0 ? Cq : Cp;
      for (int b = 0; b < p1; ++b)
        for (int a = 0; a < p1; ++a) {
          int row = ((e * 2 + comp) * p1 + b) * p1 + a;
          for (int r2 = 0; r2 <= d2; ++r2)
            for (int r1 = 0; r1 <= d1; ++r1) {
              double v = C1[((size_t)i1 * p1 + a) * p1 + r1] * C2[((size_t)i2 * p1 + b) * p1 + r2];
              if (v == 0.0) continue;
              int fl = j * nloc + local(comp, i1 + r1, i2 + r2);
              rows.push_back(row);
              cols.push_back(dof[fl]);
              vals.push_back(v * sg[fl]);
            }
        }
    }
  }
  c->nT = (int)rows.size();
  // gather CSR (rows already ascending) and scatter CSR (transpose)
  std::vector<int> gptr(c->nsup + 1, 0), sptr(c->ndof + 1, 0);
  for (int r : rows) gptr[r + 1]++;
  for (int k = 0; k < c->nsup; ++k) gptr[k + 1] += gptr[k];
  for (int cl : cols) sptr[cl + 1]++;
  for (int k = 0; k < c->ndof; ++k) sptr[k + 1] += sptr[k];
  std::vector<int> scol(c->nT), fill(sptr.begin(), sptr.end() - 1);
  std::vector<double> sval(c->nT);
  for (int t = 0; t < c->nT; ++t) {
    int at = fill[cols[t]]++;
    scol[at] = rows[t];
    sval[at] = vals[t];
  }
  EFIE_TRY(dalloc(c, &c->d_tg_ptr, gptr.size()));
  EFIE_TRY(dalloc(c, &c->d_tg_col, cols.size()));
  EFIE_TRY(dalloc(c, &c->d_tg_val, vals.size()));
  EFIE_TRY(dalloc(c, &c->d_ts_ptr, sptr.size()));
  EFIE_TRY(dalloc(c, &c->d_ts_col, scol.size()));
  EFIE_TRY(dalloc(c, &c->d_ts_val, sval.size()));
  EFIE_CUDA(cudaMemcpyAsync(c->d_tg_ptr, gptr.data(), gptr.size() * 4, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(c->d_tg_col, cols.data(), cols.size() * 4, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(c->d_tg_val, vals.data(), vals.size() * 8, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(c->d_ts_ptr, sptr.data(), sptr.size() * 4, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(c->d_ts_col, scol.data(), scol.size() * 4, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(c->d_ts_val, sval.data(), sval.size() * 8, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  return EFIE_OK;
}

// ---------------------------------------------------------------------------------------
// block-cluster tree (Algorithm 1) with bounding-ball admissibility (eq. admissibility)

efie_status host_build_trees(Ctx *c) {
  const int np = c->np, m = c->m;
  auto id = [&](int l, int j, int K) { return c->lev_off[l] + j * (1 << (2 * l)) + K; };
  auto admissible = [&](int a, int b) {
    const double *A = &c->ball[4 * a], *B = &c->ball[4 * b];
    double d = pdist(A, B) - A[3] - B[3];
    return d > 0.0 && 2.0 * std::max(A[3], B[3]) <= c->eta * d;
  };
  c->far.clear();
  c->nearl.clear();
  struct Item { int l, j, K, j2, K2; };
  std::vector<Item> stack;
  for (int j = np - 1; j >= 0; --j)
    for (int j2 = np - 1; j2 >= 0; --j2) stack.push_back({0, j, 0, j2, 0});
  const int n2 = c->n * c->n;
  const bool leaf_dense = c->opt.leaf_dense != 0 && c->p1 * c->p1 < c->nI;
  while (!stack.empty()) {
    Item it = stack.back();
    stack.pop_back();
    // leaf-level variant (option leaf_dense): an admissible pair of two leaves (single
    // elements) becomes an element block integrated by quadrature instead of an M2L block,
    // when an element carries fewer Bernstein functions per component than a cluster carries
    // interpolation nodes ((p+1)^2 < (q+1)^2)
    int a = id(it.l, it.j, it.K), b = id(it.l, it.j2, it.K2);
    if (admissible(a, b) && !(leaf_dense && it.l == m)) {
      c->far.insert(c->far.end(), {it.l, a, b});
    } else if (it.l == m) {
      c->nearl.insert(c->nearl.end(), {it.j * n2 + it.K, it.j2 * n2 + it.K2});
    } else {
      for (int ch = 3; ch >= 0; --ch)
        for (int ch2 = 3; ch2 >= 0; --ch2) stack.push_back({it.l + 1, it.j, 4 * it.K + ch, it.j2, 4 * it.K2 + ch2});
    }
  }
  c->nfar = (int)c->far.size() / 3;
  // largest phase kappa (r - r0) of the FP32 M2L: |r - r0| <= |offset_t| + |offset_s|, the
  // offsets bounded by the ball radii (with a margin for the sampled radius)
  // and the largest distance kappa r, which bounds the FP32 rounding of a direct phase
  double maxph = 0.0, maxkr = 0.0;
  for (int f = 0; f < c->nfar; ++f) {
    const double *bt = &c->ball[4 * c->far[3 * f + 1]], *bs = &c->ball[4 * c->far[3 * f + 2]];
    maxph = std::max(maxph, c->kappa * 1.5 * (bt[3] + bs[3]));
    maxkr = std::max(maxkr, c->kappa * (pdist(bt, bs) + 1.5 * (bt[3] + bs[3])));
  }
  if (!(maxph < 100.0 * M_PI)) c->m2l_mode = 2;
  // direct phase when its rounding (a few units of 2^-24 relative in kappa r: about 4 kappa r
  // 2^-24 rad per entry) stays within 2e-5 rad; the product error, an average over many entries,
  // is then about 1e-6 or less (4.3e-7 at the 13k-DOF sphere, kappa r up to about 34)
  else if (maxkr * std::ldexp(1.0, -24) < 5e-6) c->m2l_mode = 0;
  else c->m2l_mode = 1;
  c->nnear = (int)c->nearl.size() / 2;

  // far pairs as CSR over target clusters (all levels in one list)
  std::vector<int> fptr(c->ncl + 1, 0), fsrc(c->nfar);
  for (int f = 0; f < c->nfar; ++f) fptr[c->far[3 * f + 1] + 1]++;
  for (int k = 0; k < c->ncl; ++k) fptr[k + 1] += fptr[k];
  {
    std::vector<int> fill(fptr.begin(), fptr.end() - 1);
    for (int f = 0; f < c->nfar; ++f) fsrc[fill[c->far[3 * f + 1]]++] = c->far[3 * f + 2];
  }
  std::vector<int> targets;
  for (int k = 0; k < c->ncl; ++k)
    if (fptr[k + 1] > fptr[k]) targets.push_back(k);
  // longest source lists first: the M2L kernels take targets in this order
  std::stable_sort(targets.begin(), targets.end(),
                   [&](int a, int b) { return fptr[a + 1] - fptr[a] > fptr[b + 1] - fptr[b]; });
  c->n_m2l_targets = (int)targets.size();
  std::vector<int> ftgt(std::max(c->nfar, 1), 0);
  for (int k = 0; k < c->ncl; ++k)
    for (int f = fptr[k]; f < fptr[k + 1]; ++f) ftgt[f] = k;
  EFIE_TRY(dalloc(c, &c->d_far_tgt, ftgt.size()));
  EFIE_CUDA(cudaMemcpyAsync(c->d_far_tgt, ftgt.data(), ftgt.size() * 4, cudaMemcpyHostToDevice, c->stream));
  EFIE_TRY(dalloc(c, &c->d_far_ptr, fptr.size()));
  EFIE_TRY(dalloc(c, &c->d_far_src, fsrc.size()));
  EFIE_TRY(dalloc(c, &c->d_m2l_targets, targets.size()));
  EFIE_CUDA(cudaMemcpyAsync(c->d_far_ptr, fptr.data(), fptr.size() * 4, cudaMemcpyHostToDevice, c->stream));
  if (c->nfar) EFIE_CUDA(cudaMemcpyAsync(c->d_far_src, fsrc.data(), fsrc.size() * 4, cudaMemcpyHostToDevice, c->stream));
  if (!targets.empty())
    EFIE_CUDA(cudaMemcpyAsync(c->d_m2l_targets, targets.data(), targets.size() * 4, cudaMemcpyHostToDevice, c->stream));

  // unordered far pairs (the list is symmetric: (t, s) and (s, t) are both admissible): owner
  // chosen to balance the owned counts, visiting pairs by decreasing level then ids
  {
    std::vector<std::array<int, 3>> up;  // (level, t, s) with t < s
    for (int f = 0; f < c->nfar; ++f)
      if (c->far[3 * f + 1] < c->far[3 * f + 2]) up.push_back({c->far[3 * f], c->far[3 * f + 1], c->far[3 * f + 2]});
    std::sort(up.begin(), up.end(), [](const std::array<int, 3> &a, const std::array<int, 3> &b) {
      if (a[0] != b[0]) return a[0] > b[0];
      if (a[1] != b[1]) return a[1] < b[1];
      return a[2] < b[2];
    });
    c->npairs = (int)up.size();
    std::vector<int> owned(c->ncl, 0), owner(up.size());
    for (size_t u = 0; u < up.size(); ++u) {
      const int a = up[u][1], b = up[u][2];
      owner[u] = owned[a] <= owned[b] ? a : b;
      ++owned[owner[u]];
    }
    std::vector<int> optr(c->ncl + 1, 0), osrc(up.size()), oslot(up.size());
    std::vector<int> pptr(c->ncl + 1, 0), pslot(up.size());
    for (size_t u = 0; u < up.size(); ++u) {
      optr[owner[u] + 1]++;
      pptr[(owner[u] == up[u][1] ? up[u][2] : up[u][1]) + 1]++;
    }
    for (int k = 0; k < c->ncl; ++k) {
      optr[k + 1] += optr[k];
      pptr[k + 1] += pptr[k];
    }
    std::vector<int> of(optr.begin(), optr.end() - 1), pf(pptr.begin(), pptr.end() - 1);
    for (size_t u = 0; u < up.size(); ++u) {
      const int o = owner[u], other = o == up[u][1] ? up[u][2] : up[u][1];
      osrc[of[o]] = other;
      oslot[of[o]++] = (int)u;
      pslot[pf[other]++] = (int)u;
    }
    std::vector<int> otg, red;
    for (int k = 0; k < c->ncl; ++k) {
      if (optr[k + 1] > optr[k]) otg.push_back(k);
      if (optr[k + 1] > optr[k] || pptr[k + 1] > pptr[k]) red.push_back(k);
    }
    std::stable_sort(otg.begin(), otg.end(),
                     [&](int a, int b) { return optr[a + 1] - optr[a] > optr[b + 1] - optr[b]; });
    c->n_own_targets = (int)otg.size();
    c->n_red = (int)red.size();
    EFIE_TRY(dalloc(c, &c->d_own_ptr, optr.size()));
    EFIE_TRY(dalloc(c, &c->d_own_src, std::max<size_t>(osrc.size(), 1)));
    EFIE_TRY(dalloc(c, &c->d_own_slot, std::max<size_t>(oslot.size(), 1)));
    EFIE_TRY(dalloc(c, &c->d_own_targets, std::max<size_t>(otg.size(), 1)));
    EFIE_TRY(dalloc(c, &c->d_par_ptr, pptr.size()));
    EFIE_TRY(dalloc(c, &c->d_par_slot, std::max<size_t>(pslot.size(), 1)));
    EFIE_TRY(dalloc(c, &c->d_red, std::max<size_t>(red.size(), 1)));
    EFIE_CUDA(cudaMemcpyAsync(c->d_own_ptr, optr.data(), optr.size() * 4, cudaMemcpyHostToDevice, c->stream));
    EFIE_CUDA(cudaMemcpyAsync(c->d_par_ptr, pptr.data(), pptr.size() * 4, cudaMemcpyHostToDevice, c->stream));
    if (!up.empty()) {
      EFIE_CUDA(cudaMemcpyAsync(c->d_own_src, osrc.data(), osrc.size() * 4, cudaMemcpyHostToDevice, c->stream));
      EFIE_CUDA(cudaMemcpyAsync(c->d_own_slot, oslot.data(), oslot.size() * 4, cudaMemcpyHostToDevice, c->stream));
      EFIE_CUDA(cudaMemcpyAsync(c->d_own_targets, otg.data(), otg.size() * 4, cudaMemcpyHostToDevice, c->stream));
      EFIE_CUDA(cudaMemcpyAsync(c->d_par_slot, pslot.data(), pslot.size() * 4, cudaMemcpyHostToDevice, c->stream));
      EFIE_CUDA(cudaMemcpyAsync(c->d_red, red.data(), red.size() * 4, cudaMemcpyHostToDevice, c->stream));
    }
    EFIE_CUDA(cudaStreamSynchronize(c->stream));
  }

  // near pairs as CSR over target elements; near_perm maps CSR slots to list entries
  std::vector<int> nptr(c->nE + 1, 0), nsrc(c->nnear);
  c->near_perm.assign(c->nnear, 0);
  for (int k = 0; k < c->nnear; ++k) nptr[c->nearl[2 * k] + 1]++;
  for (int k = 0; k < c->nE; ++k) nptr[k + 1] += nptr[k];
  {
    std::vector<int> fill(nptr.begin(), nptr.end() - 1);
    for (int k = 0; k < c->nnear; ++k) {
      int at = fill[c->nearl[2 * k]]++;
      nsrc[at] = c->nearl[2 * k + 1];
      c->near_perm[at] = k;
    }
  }
  EFIE_TRY(dalloc(c, &c->d_near_ptr, nptr.size()));
  EFIE_TRY(dalloc(c, &c->d_near_src, nsrc.size()));
  EFIE_CUDA(cudaMemcpyAsync(c->d_near_ptr, nptr.data(), nptr.size() * 4, cudaMemcpyHostToDevice, c->stream));
  if (c->nnear) EFIE_CUDA(cudaMemcpyAsync(c->d_near_src, nsrc.data(), nsrc.size() * 4, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  return EFIE_OK;
}

// ---------------------------------------------------------------------------------------
// near-pair classification for the Sauter-Schwab rules

// square symmetry: optional swap of the coordinates, then optional reflections
struct Sym { int swap, fx, fy; };
static void sym_map(const Sym &s, double u0, double u1, double &a, double &b) {
  a = s.swap ? u1 : u0;
  b = s.swap ? u0 : u1;
  if (s.fx) a = 1.0 - a;
  if (s.fy) b = 1.0 - b;
}
static int corner_of(const Sym &s, double u0, double u1) {
  double a, b;
  sym_map(s, u0, u1, a, b);
  return (int)std::lround(a) + 2 * (int)std::lround(b);
}
static int sym_code(const Sym &s) { return s.swap | (s.fx << 1) | (s.fy << 2); }

// corner_pts: [np][(n+1)^2][3] vertex grid of every patch.
efie_status host_classify_near(Ctx *c, const std::vector<double> &corner_pts, std::vector<NearPair> &pairs,
                               std::vector<int> &mirror) {
  const int n = c->n, n2 = n * n, nv = (n + 1) * (n + 1);
  const double tol = geometry_tolerance(c);
  auto corner = [&](int e, int cc) -> const double * {
    int j = e / n2, i1, i2;
    unmorton2(e % n2, i1, i2);
    int v1 = i1 + (cc & 1), v2 = i2 + (cc >> 1);
    return &corner_pts[((size_t)j * nv + v2 * (n + 1) + v1) * 3];
  };
  auto lex_smaller = [&](const double *u, const double *v) {  // tolerance-aware u < v
    for (int k = 0; k < 3; ++k)
      if (std::fabs(u[k] - v[k]) > tol) return u[k] < v[k];
    return false;
  };
  pairs.resize(c->nnear);
  for (int k = 0; k < c->nnear; ++k) {
    NearPair &P = pairs[k];
    P.e = c->nearl[2 * k];
    P.e2 = c->nearl[2 * k + 1];
    P.kind = 0;
    P.r1 = P.r2 = 0;
    if (P.e == P.e2) {
      P.kind = 3;
      continue;
    }
    int sa[4], sb[4], ns = 0;
    for (int i = 0; i < 4; ++i)
      for (int t = 0; t < 4; ++t)
        if (pdist(corner(P.e, i), corner(P.e2, t)) < tol) {
          if (ns < 4) {
            sa[ns] = i;
            sb[ns] = t;
          }
          ++ns;
        }
    if (ns == 0) continue;
    if (ns == 1) {  // shared vertex to the origin by reflections only
      P.kind = 1;
      P.r1 = sym_code({0, sa[0] & 1, sa[0] >> 1});
      P.r2 = sym_code({0, sb[0] & 1, sb[0] >> 1});
      continue;
    }
    if (ns == 2) {  // shared edge onto {x2 = 0}, from the lexicographically smaller end
      int f = lex_smaller(corner(P.e, sa[1]), corner(P.e, sa[0])) ? 1 : 0, g = 1 - f;
      int found = 0;
      for (int code = 0; code < 8; ++code) {
        Sym s{code & 1, (code >> 1) & 1, (code >> 2) & 1};
        if (corner_of(s, 0, 0) == sa[f] && corner_of(s, 1, 0) == sa[g]) { P.r1 = code; found |= 1; }
        if (corner_of(s, 0, 0) == sb[f] && corner_of(s, 1, 0) == sb[g]) { P.r2 = code; found |= 2; }
      }
      if (found == 3) {
        P.kind = 2;
        continue;
      }
    }
    c->err = "elements " + std::to_string(P.e) + " and " + std::to_string(P.e2) + " overlap or touch irregularly";
    return EFIE_EGEOMETRY;
  }
  // mirror partner of every pair (the near set is symmetric)
  std::unordered_map<int64_t, int> where;
  where.reserve(c->nnear * 2);
  for (int k = 0; k < c->nnear; ++k) where[(int64_t)pairs[k].e * c->nE + pairs[k].e2] = k;
  mirror.assign(c->nnear, -1);
  for (int k = 0; k < c->nnear; ++k) {
    auto it = where.find((int64_t)pairs[k].e2 * c->nE + pairs[k].e);
    if (it == where.end()) {
      c->err = "near field is not symmetric";
      return EFIE_EGEOMETRY;
    }
    mirror[k] = it->second;
  }
  return EFIE_OK;
}

}  // namespace efie
