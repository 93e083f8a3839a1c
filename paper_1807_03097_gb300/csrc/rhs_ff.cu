// Right-hand side (a12) and far field (a13).
//  a12: g*_{e,alpha,ab} = -int_e e_i(F(s)) . d_alpha F(s) psi_ab ds for the plane wave
//       e_i = pol exp(i kappa d.x) (eq. linsys with the dot-product pairing of eq. MSLtested),
//       then g = T^T g*.
//  a13: E_inf(d) = (W - d (d.W)) / 4pi with W = int w exp(-i kappa d.y) dsigma, the far field
//       of the electric single-layer potential (eq. ESLP); on a patch w dsigma = dF w_hat ds.
// Tensor Gauss rules with quad_regular points per direction; deterministic reductions.
#include <algorithm>
#include <cmath>

#include "geom.cuh"

namespace efie {

efie_status dev_scatter(Ctx *c, const double2 *ys, double2 *y);
efie_status dev_gather(Ctx *c, const double2 *x, double2 *xs);

__device__ inline void elem_locate(int e, int n, int &j, int &i1, int &i2) {
  int n2 = n * n;
  j = e / n2;
  int K = e % n2;
  i1 = 0;
  i2 = 0;
  for (int b = 0; b < 15; ++b) {
    i1 |= ((K >> (2 * b)) & 1) << b;
    i2 |= ((K >> (2 * b + 1)) & 1) << b;
  }
}

// one block per element, one thread per Gauss point (g*g <= 256)
__global__ void k_rhs(const PatchDesc *patches, const double *knots, const double4 *cpw, int n, int p, int g,
                      const double *gx, const double *gw, double kappa, double d0, double d1, double d2, double p0,
                      double pp1, double p2, double2 *gs) {
  int e = blockIdx.x;
  int P1 = p + 1;
  __shared__ double2 val[256][2];
  __shared__ double B[256][2][kMaxP1];
  int j, i1, i2;
  elem_locate(e, n, j, i1, i2);
  double h = 1.0 / n;
  int t = threadIdx.x;
  if (t < g * g) {
    double u = gx[t % g], v = gx[t / g];
    double X[3], D1[3], D2[3];
    dev_patch_eval(patches[j], knots, cpw, (i1 + u) * h, (i2 + v) * h, X, D1, D2);
    double sn, cs;
    sincos(kappa * (d0 * X[0] + d1 * X[1] + d2 * X[2]), &sn, &cs);
    double wt = gw[t % g] * gw[t / g] * h * h;
    double a0 = p0 * D1[0] + pp1 * D1[1] + p2 * D1[2];
    double a1 = p0 * D2[0] + pp1 * D2[1] + p2 * D2[2];
    val[t][0] = make_double2(-wt * a0 * cs, -wt * a0 * sn);
    val[t][1] = make_double2(-wt * a1 * cs, -wt * a1 * sn);
    double Bu[kMaxP1], dBu[kMaxP1], Bv[kMaxP1], dBv[kMaxP1];
    dev_bernstein(p, u, Bu, dBu);
    dev_bernstein(p, v, Bv, dBv);
    for (int a = 0; a < P1; ++a) {
      B[t][0][a] = Bu[a];
      B[t][1][a] = Bv[a];
    }
  }
  __syncthreads();
  int nout = 2 * P1 * P1;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    int al = o / (P1 * P1), b = (o / P1) % P1, a = o % P1;
    double x = 0.0, y = 0.0;
    for (int k = 0; k < g * g; ++k) {
      double f = B[k][0][a] * B[k][1][b];
      x += f * val[k][al].x;
      y += f * val[k][al].y;
    }
    gs[(size_t)e * nout + o] = make_double2(x, y);
  }
}

efie_status dev_rhs(Ctx *c, const double *dir, const double *pol, double2 *g) {
  if (c->gr * c->gr > 256) {
    c->err = "quad_regular must be <= 16";
    return EFIE_EINVAL;
  }
  DevTemp tmp;
  double *d_rule = nullptr;
  EFIE_TRY(tmp.get(c, &d_rule, 2 * (size_t)c->gr));
  EFIE_CUDA(cudaMemcpyAsync(d_rule, c->tab.gx.data(), 8 * (size_t)c->gr, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(d_rule + c->gr, c->tab.gw.data(), 8 * (size_t)c->gr, cudaMemcpyHostToDevice, c->stream));
  k_rhs<<<c->nE, 256, 0, c->stream>>>(c->d_patches, c->d_knots, c->d_cpw, c->n, c->p, c->gr, d_rule, d_rule + c->gr,
                                      c->kappa, dir[0], dir[1], dir[2], pol[0], pol[1], pol[2], c->d_ys); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_TRY(dev_scatter(c, c->d_ys, g));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  return EFIE_OK;
}

// Partial W of one element for every direction: part[(dir * nE + e) * 3 + k].  The block first
// evaluates, at each of the element's g x g Gauss points (one thread each), the point F(x) and
// the weighted surface current v = w h^2 (d1F w_1 + d2F w_2) from the element's superspace
// coefficients, once; then thread t sums e^{-i kappa d.F(x)} v over the points, in a fixed
// order, for the directions t, t + blockDim, ...
__global__ void k_ff_partial(const PatchDesc *patches, const double *knots, const double4 *cpw, int n, int p, int g,
                             const double *gx, const double *gw, double kappa, int nE, int ndir, const double *dirs,
                             const double2 *__restrict__ xs, double2 *part) {
  extern __shared__ double2 sff[];
  const int e = blockIdx.x, G2 = g * g, P1 = p + 1;
  double2 *sV = sff;                                        // [G2][3] (16-byte aligned)
  double *sX = reinterpret_cast<double *>(sff + 3 * G2);    // [G2][3]
  int j, i1, i2;
  elem_locate(e, n, j, i1, i2);
  const double h = 1.0 / n;
  for (int t = threadIdx.x; t < G2; t += blockDim.x) {
    const double u = gx[t % g], v = gx[t / g];
    double X[3], D1[3], D2[3];
    dev_patch_eval(patches[j], knots, cpw, (i1 + u) * h, (i2 + v) * h, X, D1, D2);
    const double wt = gw[t % g] * gw[t / g] * h * h;
    double Bu[kMaxP1], dBu[kMaxP1], Bv[kMaxP1], dBv[kMaxP1];
    dev_bernstein(p, u, Bu, dBu);
    dev_bernstein(p, v, Bv, dBv);
    double2 wa[2] = {make_double2(0, 0), make_double2(0, 0)};
    const double2 *xe = xs + (size_t)e * 2 * P1 * P1;
    for (int al = 0; al < 2; ++al)
      for (int b = 0; b < P1; ++b)
        for (int a = 0; a < P1; ++a) {
          const double f = Bu[a] * Bv[b];
          const double2 cf = xe[(al * P1 + b) * P1 + a];
          wa[al].x += f * cf.x;
          wa[al].y += f * cf.y;
        }
    for (int k = 0; k < 3; ++k) {
      sX[3 * t + k] = X[k];
      sV[3 * t + k] = make_double2(wt * (D1[k] * wa[0].x + D2[k] * wa[1].x), wt * (D1[k] * wa[0].y + D2[k] * wa[1].y));
    }
  }
  __syncthreads();
  for (int dd = threadIdx.x; dd < ndir; dd += blockDim.x) {
    const double d0 = dirs[3 * dd], d1 = dirs[3 * dd + 1], d2 = dirs[3 * dd + 2];
    double2 W[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int t = 0; t < G2; ++t) {
      double sn, cs;
      sincos(-kappa * (d0 * sX[3 * t] + d1 * sX[3 * t + 1] + d2 * sX[3 * t + 2]), &sn, &cs);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 v = sV[3 * t + k];
        W[k].x += cs * v.x - sn * v.y;
        W[k].y += cs * v.y + sn * v.x;
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) part[((size_t)dd * nE + e) * 3 + k] = W[k];
  }
}

__global__ void k_ff_final(int nE, const double *dirs, const double2 *part, double2 *out) {
  int dd = blockIdx.x;
  __shared__ double2 red[256][3];
  int t = threadIdx.x;
  double2 W[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  for (int e = t; e < nE; e += blockDim.x)
    for (int k = 0; k < 3; ++k) {
      W[k].x += part[((size_t)dd * nE + e) * 3 + k].x;
      W[k].y += part[((size_t)dd * nE + e) * 3 + k].y;
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
  if (t == 0) {
    const double *d = dirs + 3 * dd;
    double2 dw = make_double2(d[0] * red[0][0].x + d[1] * red[0][1].x + d[2] * red[0][2].x,
                              d[0] * red[0][0].y + d[1] * red[0][1].y + d[2] * red[0][2].y);
    const double f = 0.25 / M_PI;
    for (int k = 0; k < 3; ++k)
      out[3 * dd + k] = make_double2(f * (red[0][k].x - d[k] * dw.x), f * (red[0][k].y - d[k] * dw.y));
  }
}

efie_status dev_far_field(Ctx *c, const double2 *w, int ndir, const double *dirs, double2 *out) {
  if (c->gr * c->gr > 256) {
    c->err = "quad_regular must be <= 16";
    return EFIE_EINVAL;
  }
  DevTemp tmp;
  double *d_rule = nullptr, *d_dirs = nullptr;
  double2 *d_part = nullptr;
  EFIE_TRY(tmp.get(c, &d_rule, 2 * (size_t)c->gr));
  EFIE_TRY(tmp.get(c, &d_dirs, 3 * (size_t)ndir));
  EFIE_TRY(tmp.get(c, &d_part, 3 * (size_t)ndir * c->nE));
  EFIE_CUDA(cudaMemcpyAsync(d_rule, c->tab.gx.data(), 8 * (size_t)c->gr, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(d_rule + c->gr, c->tab.gw.data(), 8 * (size_t)c->gr, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(d_dirs, dirs, 24 * (size_t)ndir, cudaMemcpyHostToDevice, c->stream));
  EFIE_TRY(dev_gather(c, w, c->d_xs));
  const int G2 = c->gr * c->gr;
  const int thr = std::min(256, std::max(64, ((std::max(G2, ndir) + 31) / 32) * 32));
  k_ff_partial<<<c->nE, thr, sizeof(double) * 9 * G2, c->stream>>>(c->d_patches, c->d_knots, c->d_cpw, c->n, c->p,
                                                                     c->gr, d_rule, d_rule + c->gr, c->kappa, c->nE,
                                                                     ndir, d_dirs, c->d_xs, d_part);
  ++c->launches;
  k_ff_final<<<ndir, 256, 0, c->stream>>>(c->nE, d_dirs, d_part, out); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  return EFIE_OK;
}

}  // namespace efie
