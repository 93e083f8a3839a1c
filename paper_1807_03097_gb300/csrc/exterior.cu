// Electric field off the surface and the manufactured-solution right-hand side (Sec. 5.2).
//  * Electric single-layer potential (eq. ESLP) at points x off the surface:
//      E(x) = int G(x-y) w(y) dsigma_y + kappa^-2 grad_x int G(x-y) div_Gamma w(y) dsigma_y,
//    G of eq. HelmholtzGreen, grad_x G(x-y) = G(x-y) (i kappa - 1/R) (x-y)/R, R = |x-y|; on a
//    patch w dsigma = dF w_hat ds and div_Gamma w dsigma = div w_hat ds (Piola transforms).
//    Tensor Gauss rule with quad_regular points per element direction, so the points must be
//    well separated from the surface (the quadrature is not adapted to near points).
//  * Right-hand side for the incident field e_i = -DP_{x0,p0} (Hertz dipole, Sec. 5.2): the
//    scattered field outside is then DP itself, g = -T^T int e_i . phi = +T^T int DP . phi.
// One block per (element, point) or element, one thread per Gauss point; deterministic
// reductions in a fixed order.
#include <cmath>

#include "geom.cuh"

namespace efie {

efie_status dev_scatter(Ctx *c, const double2 *ys, double2 *y);
efie_status dev_gather(Ctx *c, const double2 *x, double2 *xs);

namespace {

__device__ inline void locate(int e, int n, int &j, int &i1, int &i2) {
  const int n2 = n * n, K = e % n2;
  j = e / n2;
  i1 = 0;
  i2 = 0;
  for (int b = 0; b < 15; ++b) {
    i1 |= ((K >> (2 * b)) & 1) << b;
    i2 |= ((K >> (2 * b + 1)) & 1) << b;
  }
}

// Hertz dipole DP_{x0,p0}(x) = e^{i kappa r} ( kappa^2/r (p0 - n (n.p0))
//                                              + (1/r^3 - i kappa/r^2)(3 n (n.p0) - p0) )
__device__ inline void dipole(double kappa, const double *x0, const double *p0, const double *x, double2 *E) {
  const double d0 = x[0] - x0[0], d1 = x[1] - x0[1], d2 = x[2] - x0[2];
  const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  const double n[3] = {d0 / r, d1 / r, d2 / r};
  const double np = n[0] * p0[0] + n[1] * p0[1] + n[2] * p0[2];
  double sn, cs;
  sincos(kappa * r, &sn, &cs);
  const double a = kappa * kappa / r, br = 1.0 / (r * r * r), bi = -kappa / (r * r);
  for (int c = 0; c < 3; ++c) {
    const double v1 = p0[c] - n[c] * np, v2 = 3.0 * n[c] * np - p0[c];
    const double re = a * v1 + br * v2, im = bi * v2;  // (a v1 + (br + i bi) v2)
    E[c] = make_double2(cs * re - sn * im, cs * im + sn * re);
  }
}

}  // namespace

// one block per element, one thread per Gauss point (g*g <= 256)
__global__ void k_rhs_dipole(const PatchDesc *patches, const double *knots, const double4 *cpw, int n, int p, int g,
                             const double *gx, const double *gw, double kappa, const double *x0p0,
                             double2 *gs) {
  const int e = blockIdx.x, P1 = p + 1, t = threadIdx.x;
  __shared__ double2 val[256][2];
  __shared__ double B[256][2][kMaxP1];
  int j, i1, i2;
  locate(e, n, j, i1, i2);
  const double h = 1.0 / n;
  if (t < g * g) {
    const double u = gx[t % g], v = gx[t / g];
    double X[3], D1[3], D2[3];
    dev_patch_eval(patches[j], knots, cpw, (i1 + u) * h, (i2 + v) * h, X, D1, D2);
    double2 E[3];
    dipole(kappa, x0p0, x0p0 + 3, X, E);
    const double wt = gw[t % g] * gw[t / g] * h * h;
    double2 a0 = make_double2(0, 0), a1 = make_double2(0, 0);
    for (int c = 0; c < 3; ++c) {
      a0.x += E[c].x * D1[c];
      a0.y += E[c].y * D1[c];
      a1.x += E[c].x * D2[c];
      a1.y += E[c].y * D2[c];
    }
    val[t][0] = make_double2(wt * a0.x, wt * a0.y);
    val[t][1] = make_double2(wt * a1.x, wt * a1.y);
    double Bu[kMaxP1], dBu[kMaxP1], Bv[kMaxP1], dBv[kMaxP1];
    dev_bernstein(p, u, Bu, dBu);
    dev_bernstein(p, v, Bv, dBv);
    for (int a = 0; a < P1; ++a) {
      B[t][0][a] = Bu[a];
      B[t][1][a] = Bv[a];
    }
  }
  __syncthreads();
  const int nout = 2 * P1 * P1;
  for (int o = t; o < nout; o += blockDim.x) {
    const int al = o / (P1 * P1), b = (o / P1) % P1, a = o % P1;
    double x = 0.0, y = 0.0;
    for (int k = 0; k < g * g; ++k) {
      const double f = B[k][0][a] * B[k][1][b];
      x += f * val[k][al].x;
      y += f * val[k][al].y;
    }
    gs[(size_t)e * nout + o] = make_double2(x, y);
  }
}

// partial field of element blockIdx.x at point blockIdx.y: part[(pt nE + e) 3 + k]
__global__ void k_ext_partial(const PatchDesc *patches, const double *knots, const double4 *cpw, int n, int p, int g,
                              const double *gx, const double *gw, double kappa, int nE, const double *pts,
                              const double2 *__restrict__ xs, double2 *part) {
  const int e = blockIdx.x, pt = blockIdx.y, P1 = p + 1, t = threadIdx.x;
  __shared__ double2 red[256][3];
  int j, i1, i2;
  locate(e, n, j, i1, i2);
  const double h = 1.0 / n;
  double2 C[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  if (t < g * g) {
    const double u = gx[t % g], v = gx[t / g];
    double X[3], D1[3], D2[3];
    dev_patch_eval(patches[j], knots, cpw, (i1 + u) * h, (i2 + v) * h, X, D1, D2);
    const double *x = pts + 3 * pt;
    const double d[3] = {x[0] - X[0], x[1] - X[1], x[2] - X[2]};
    const double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double sn, cs;
    sincos(kappa * R, &sn, &cs);
    const double gr = cs / (4.0 * M_PI * R), gi = sn / (4.0 * M_PI * R);  // G
    double Bu[kMaxP1], dBu[kMaxP1], Bv[kMaxP1], dBv[kMaxP1];
    dev_bernstein(p, u, Bu, dBu);
    dev_bernstein(p, v, Bv, dBv);
    const double2 *xe = xs + (size_t)e * 2 * P1 * P1;
    double2 w0 = make_double2(0, 0), w1 = make_double2(0, 0), dv = make_double2(0, 0);
    for (int b = 0; b < P1; ++b)
      for (int a = 0; a < P1; ++a) {
        const double2 c0 = xe[b * P1 + a], c1 = xe[(P1 + b) * P1 + a];
        const double f = Bu[a] * Bv[b], f0 = dBu[a] * Bv[b], f1 = Bu[a] * dBv[b];
        w0.x += f * c0.x;
        w0.y += f * c0.y;
        w1.x += f * c1.x;
        w1.y += f * c1.y;
        dv.x += f0 * c0.x + f1 * c1.x;
        dv.y += f0 * c0.y + f1 * c1.y;
      }
    const double wq = gw[t % g] * gw[t / g];
    // vector part: wq h^2 G (D1 w0 + D2 w1)
    const double sv = wq * h * h;
    // gradient part / kappa^2: wq h G (i kappa - 1/R) / R * d * dv
    const double sd = wq * h / (R * kappa * kappa);
    const double2 q = make_double2(-gr / R - gi * kappa, gr * kappa - gi / R);  // G (i kappa - 1/R)
    const double2 qd = make_double2(q.x * dv.x - q.y * dv.y, q.x * dv.y + q.y * dv.x);
    for (int k = 0; k < 3; ++k) {
      const double vx = D1[k] * w0.x + D2[k] * w1.x, vy = D1[k] * w0.y + D2[k] * w1.y;
      C[k] = make_double2(sv * (gr * vx - gi * vy) + sd * d[k] * qd.x, sv * (gr * vy + gi * vx) + sd * d[k] * qd.y);
    }
  }
  for (int k = 0; k < 3; ++k) red[t][k] = C[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s)
      for (int k = 0; k < 3; ++k) {
        red[t][k].x += red[t + s][k].x;
        red[t][k].y += red[t + s][k].y;
      }
    __syncthreads();
  }
  if (t == 0)
    for (int k = 0; k < 3; ++k) part[((size_t)pt * nE + e) * 3 + k] = red[0][k];
}

// out[pt][k] = sum over elements (fixed order) of part
__global__ void k_ext_final(int nE, const double2 *part, double2 *out) {
  const int pt = blockIdx.x, t = threadIdx.x;
  __shared__ double2 red[256][3];
  double2 W[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  for (int e = t; e < nE; e += blockDim.x)
    for (int k = 0; k < 3; ++k) {
      W[k].x += part[((size_t)pt * nE + e) * 3 + k].x;
      W[k].y += part[((size_t)pt * nE + e) * 3 + k].y;
    }
  for (int k = 0; k < 3; ++k) red[t][k] = W[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s)
      for (int k = 0; k < 3; ++k) {
        red[t][k].x += red[t + s][k].x;
        red[t][k].y += red[t + s][k].y;
      }
    __syncthreads();
  }
  if (t == 0)
    for (int k = 0; k < 3; ++k) out[3 * pt + k] = red[0][k];
}

static efie_status upload_rule(Ctx *c, DevTemp &tmp, double **d_rule) {
  if (c->gr * c->gr > 256) {
    c->err = "quad_regular must be <= 16";
    return EFIE_EINVAL;
  }
  EFIE_TRY(tmp.get(c, d_rule, 2 * (size_t)c->gr));
  EFIE_CUDA(cudaMemcpyAsync(*d_rule, c->tab.gx.data(), 8 * (size_t)c->gr, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(*d_rule + c->gr, c->tab.gw.data(), 8 * (size_t)c->gr, cudaMemcpyHostToDevice, c->stream));
  return EFIE_OK;
}

// g (device, ndof) for the incident field -DP_{x0,p0}; x0, p0 host arrays of 3
efie_status dev_rhs_dipole(Ctx *c, const double *x0, const double *p0, double2 *g) {
  DevTemp tmp;
  double *d_rule = nullptr, *d_xp = nullptr;
  EFIE_TRY(upload_rule(c, tmp, &d_rule));
  EFIE_TRY(tmp.get(c, &d_xp, 6));
  double xp[6] = {x0[0], x0[1], x0[2], p0[0], p0[1], p0[2]};
  EFIE_CUDA(cudaMemcpyAsync(d_xp, xp, sizeof(xp), cudaMemcpyHostToDevice, c->stream));
  k_rhs_dipole<<<c->nE, 256, 0, c->stream>>>(c->d_patches, c->d_knots, c->d_cpw, c->n, c->p, c->gr, d_rule,
                                             d_rule + c->gr, c->kappa, d_xp, c->d_ys); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_TRY(dev_scatter(c, c->d_ys, g));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  return EFIE_OK;
}

// out (device, [npts][3] complex) = eq. ESLP of the DOF vector w (device) at pts (host)
efie_status dev_exterior_field(Ctx *c, const double2 *w, int npts, const double *pts, double2 *out) {
  DevTemp tmp;
  double *d_rule = nullptr, *d_pts = nullptr;
  double2 *d_part = nullptr;
  EFIE_TRY(upload_rule(c, tmp, &d_rule));
  EFIE_TRY(tmp.get(c, &d_pts, 3 * (size_t)npts));
  EFIE_TRY(tmp.get(c, &d_part, 3 * (size_t)npts * c->nE));
  EFIE_CUDA(cudaMemcpyAsync(d_pts, pts, 24 * (size_t)npts, cudaMemcpyHostToDevice, c->stream));
  EFIE_TRY(dev_gather(c, w, c->d_xs));
  dim3 grid(c->nE, npts);
  k_ext_partial<<<grid, 256, 0, c->stream>>>(c->d_patches, c->d_knots, c->d_cpw, c->n, c->p, c->gr, d_rule,
                                             d_rule + c->gr, c->kappa, c->nE, d_pts, c->d_xs, d_part); ++c->launches;
  k_ext_final<<<npts, 256, 0, c->stream>>>(c->nE, d_part, out); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  return EFIE_OK;
}

}  // namespace efie
