// Far field by the interpolation-based H^2 scheme of Sec. 4.2 (eq. FMMlr) and the
// superspace transformation (eq. superspace):
//   a3  x* = T x                         (k_gather)
//   a4  leaf moments of the vector part M^box and of the div part M^{alpha,box}
//   a5  M2M: moments of a parent from its four children through the tensor transfer
//       E_c[m][m'] = L_m((c + x_m') / 2), exact re-expansion of degree-q polynomials
//   a6  M2L: for every admissible block, the kernel G_kappa at the tensor Chebyshev nodes
//       mapped through the patch maps, applied to 4 fields: the vector moments folded into
//       Cartesian form u = sum_beta d_beta F(x_m') mu_beta (so that K1^(alpha,beta) =
//       G <d_alpha F, d_beta F'> becomes G times a 3-vector dot product) and the div
//       moment (K2 = -kappa^-2 G)
//   a7  L2L: transpose of a5
//   a8  evaluation at the test functions of every leaf
//   a10 y = T^T y*                       (k_scatter)
#include <algorithm>
#include <cmath>

#include "efie_internal.h"

namespace efie {

efie_status dev_near_apply(Ctx *c, const double2 *xs, double2 *ysn, cudaStream_t st);

template <class R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };
template <class R> using C2 = typename Cx<R>::T;
template <class R> __device__ inline C2<R> mk(R a, R b) { C2<R> v; v.x = a; v.y = b; return v; }

// ------------------------------------------------------------------------ T and T^T
__global__ void k_gather(int nrow, const int *__restrict__ ptr, const int *__restrict__ col,
                         const double *__restrict__ val, const double2 *__restrict__ x, double2 *__restrict__ xs) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  double2 s = make_double2(0.0, 0.0);
  for (int k = ptr[r]; k < ptr[r + 1]; ++k) {
    double2 v = x[col[k]];
    s.x += val[k] * v.x;
    s.y += val[k] * v.y;
  }
  xs[r] = s;
}

__global__ void k_scatter(int ndof, const int *__restrict__ ptr, const int *__restrict__ row,
                          const double *__restrict__ val, const double2 *__restrict__ ys,
                          const double2 *__restrict__ ysn, double2 *__restrict__ y) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= ndof) return;
  double2 s = make_double2(0.0, 0.0);
  for (int k = ptr[d]; k < ptr[d + 1]; ++k) {
    double2 v = ys[row[k]];
    if (ysn) {
      double2 w = ysn[row[k]];
      v.x += w.x;
      v.y += w.y;
    }
    s.x += val[k] * v.x;
    s.y += val[k] * v.y;
  }
  y[d] = s;
}

__global__ void k_add(int n, double2 *a, const double2 *b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    a[i].x += b[i].x;
    a[i].y += b[i].y;
  }
}

// ------------------------------------------------------------------------ a4 leaf moments
// mu_beta(m) = h^2 sum_ab M[m1][a] M[m2][b] x*_{beta,b,a}
// nu(m)      = h sum_ab (Md[m1][a] M[m2][b] x*_{0,b,a} + M[m1][a] Md[m2][b] x*_{1,b,a})
template <class R>
__global__ void k_leaf_moments(int nE, int leaf_off, int p1, int q1, R h, const double *__restrict__ Mt,
                               const double *__restrict__ Mdt, const double2 *__restrict__ xs, C2<R> *__restrict__ mom) {
  int e = blockIdx.x;
  if (e >= nE) return;
  int nI = q1 * q1;
  __shared__ R sM[kMaxQ1 * kMaxP1], sMd[kMaxQ1 * kMaxP1];
  __shared__ C2<R> sx[2 * kMaxP1 * kMaxP1];
  __shared__ C2<R> T0[kMaxP1 * kMaxQ1], T1[kMaxP1 * kMaxQ1], Td[kMaxP1 * kMaxQ1];
  for (int i = threadIdx.x; i < q1 * p1; i += blockDim.x) {
    sM[i] = (R)Mt[i];
    sMd[i] = (R)Mdt[i];
  }
  for (int i = threadIdx.x; i < 2 * p1 * p1; i += blockDim.x) {
    double2 v = xs[(size_t)e * 2 * p1 * p1 + i];
    sx[i] = mk<R>((R)v.x, (R)v.y);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < p1 * q1; i += blockDim.x) {
    int b = i / q1, m1 = i % q1;
    C2<R> a0 = mk<R>(0, 0), a1 = mk<R>(0, 0), ad = mk<R>(0, 0);
    for (int a = 0; a < p1; ++a) {
      R M = sM[m1 * p1 + a], Md = sMd[m1 * p1 + a];
      C2<R> x0 = sx[b * p1 + a], x1 = sx[p1 * p1 + b * p1 + a];
      a0.x += M * x0.x; a0.y += M * x0.y;
      a1.x += M * x1.x; a1.y += M * x1.y;
      ad.x += Md * x0.x; ad.y += Md * x0.y;
    }
    T0[i] = a0;
    T1[i] = a1;
    Td[i] = ad;
  }
  __syncthreads();
  C2<R> *out = mom + (size_t)(leaf_off + e) * 3 * nI;
  R h2 = h * h;
  for (int mi = threadIdx.x; mi < nI; mi += blockDim.x) {
    int m1 = mi % q1, m2 = mi / q1;
    C2<R> u0 = mk<R>(0, 0), u1 = mk<R>(0, 0), v = mk<R>(0, 0);
    for (int b = 0; b < p1; ++b) {
      R M = sM[m2 * p1 + b], Md = sMd[m2 * p1 + b];
      C2<R> t0 = T0[b * q1 + m1], t1 = T1[b * q1 + m1], td = Td[b * q1 + m1];
      u0.x += M * t0.x; u0.y += M * t0.y;
      u1.x += M * t1.x; u1.y += M * t1.y;
      v.x += M * td.x + Md * t1.x; v.y += M * td.y + Md * t1.y;
    }
    out[mi] = mk<R>(h2 * u0.x, h2 * u0.y);
    out[nI + mi] = mk<R>(h2 * u1.x, h2 * u1.y);
    out[2 * nI + mi] = mk<R>(h * v.x, h * v.y);
  }
}

// ------------------------------------------------------------------------ a5 M2M
// parent(f, m2, m1) = sum_c sum_{m2'} E[c2][m2][m2'] sum_{m1'} E[c1][m1][m1'] child_c(f, m2', m1')
template <class R>
__global__ void k_m2m(int nparent, int par_off, int ch_off, int q1, const double *__restrict__ Et,
                      C2<R> *__restrict__ mom) {
  int pid = blockIdx.x;
  if (pid >= nparent) return;
  int nI = q1 * q1;
  extern __shared__ unsigned char smraw[];
  R *sE = (R *)smraw;                                      // [2][q1][q1]
  C2<R> *ch = (C2<R> *)(smraw + sizeof(double) * 2 * kMaxQ1 * kMaxQ1);  // [4][3][nI]
  C2<R> *T = ch + 12 * nI;                                 // [4][3][q1 (m2')][q1 (m1)]
  for (int i = threadIdx.x; i < 2 * q1 * q1; i += blockDim.x) sE[i] = (R)Et[i];
  // children of parent (patch j, K) at level l are 4K + c at level l + 1: contiguous
  const C2<R> *cm = mom + (size_t)(ch_off + 4 * pid) * 3 * nI;
  for (int i = threadIdx.x; i < 12 * nI; i += blockDim.x) ch[i] = cm[i];
  __syncthreads();
  for (int i = threadIdx.x; i < 12 * nI; i += blockDim.x) {
    int cf = i / nI, rem = i % nI, m2p = rem / q1, m1 = rem % q1;
    int cidx = cf / 3, c1 = cidx & 1;
    C2<R> s = mk<R>(0, 0);
    const C2<R> *src = ch + cf * nI + m2p * q1;
    for (int m1p = 0; m1p < q1; ++m1p) {
      R e = sE[(c1 * q1 + m1) * q1 + m1p];
      s.x += e * src[m1p].x;
      s.y += e * src[m1p].y;
    }
    T[i] = s;
  }
  __syncthreads();
  C2<R> *out = mom + (size_t)(par_off + pid) * 3 * nI;
  for (int i = threadIdx.x; i < 3 * nI; i += blockDim.x) {
    int f = i / nI, rem = i % nI, m2 = rem / q1, m1 = rem % q1;
    C2<R> s = mk<R>(0, 0);
    for (int cidx = 0; cidx < 4; ++cidx) {
      int c2 = cidx >> 1;
      const C2<R> *tt = T + (cidx * 3 + f) * nI;
      for (int m2p = 0; m2p < q1; ++m2p) {
        R e = sE[(c2 * q1 + m2) * q1 + m2p];
        s.x += e * tt[m2p * q1 + m1].x;
        s.y += e * tt[m2p * q1 + m1].y;
      }
    }
    out[i] = s;
  }
}

// ------------------------------------------------------------------------ fold / unfold
template <class R>
__global__ void k_fold(long long tot, int nI, const double *__restrict__ nodeD, const C2<R> *__restrict__ mom,
                       C2<R> *__restrict__ src) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  int id = (int)(t / nI), mi = (int)(t % nI);
  const double *D = nodeD + 6 * t;
  const C2<R> *mm = mom + (size_t)id * 3 * nI;
  C2<R> m0 = mm[mi], m1 = mm[nI + mi];
  C2<R> *s = src + (size_t)id * 4 * nI;
  for (int k = 0; k < 3; ++k) {
    R d1 = (R)D[k], d2 = (R)D[3 + k];
    s[k * nI + mi] = mk<R>(d1 * m0.x + d2 * m1.x, d1 * m0.y + d2 * m1.y);
  }
  s[3 * nI + mi] = mm[2 * nI + mi];
}

template <class R, class A>
__global__ void k_unfold(long long tot, int nI, R ik2, const double *__restrict__ nodeD, const A *__restrict__ acc,
                         C2<R> *__restrict__ loc) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  int id = (int)(t / nI), mi = (int)(t % nI);
  const double *D = nodeD + 6 * t;
  const A *a = acc + (size_t)id * 4 * nI;
  R l0x = 0, l0y = 0, l1x = 0, l1y = 0;
  for (int k = 0; k < 3; ++k) {
    A v = a[k * nI + mi];
    l0x += (R)D[k] * (R)v.x;
    l0y += (R)D[k] * (R)v.y;
    l1x += (R)D[3 + k] * (R)v.x;
    l1y += (R)D[3 + k] * (R)v.y;
  }
  C2<R> *l = loc + (size_t)id * 3 * nI;
  l[mi] = mk<R>(l0x, l0y);
  l[nI + mi] = mk<R>(l1x, l1y);
  A dv = a[3 * nI + mi];
  l[2 * nI + mi] = mk<R>(-ik2 * (R)dv.x, -ik2 * (R)dv.y);
}

// ------------------------------------------------------------------------ a6 M2L (FP64)
// acc_t(k, m) = (1/4pi) sum_{s in far(t)} sum_m' e^{i kappa r}/r src_s(k, m'),
// r = |F_t(x_m) - F_s(x_m')|.  One block per target cluster, one thread per target node.
__global__ void k_m2l_f64(const int *__restrict__ targets, const int *__restrict__ fptr, const int *__restrict__ fsrc,
                          int nI, double kappa, const double *__restrict__ nodeX, const double2 *__restrict__ src,
                          double2 *__restrict__ acc) {
  int t = targets[blockIdx.x];
  extern __shared__ double smd[];
  double *sX = smd;                               // [nI][3]
  double2 *sS = (double2 *)(smd + 3 * nI + (3 * nI & 1));  // [4][nI]
  int mi = threadIdx.x;
  double xt0 = 0, xt1 = 0, xt2 = 0;
  if (mi < nI) {
    xt0 = nodeX[((size_t)t * nI + mi) * 3];
    xt1 = nodeX[((size_t)t * nI + mi) * 3 + 1];
    xt2 = nodeX[((size_t)t * nI + mi) * 3 + 2];
  }
  double2 a0 = make_double2(0, 0), a1 = a0, a2 = a0, a3 = a0;
  for (int k = fptr[t]; k < fptr[t + 1]; ++k) {
    int s = fsrc[k];
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nI; i += blockDim.x) sX[i] = nodeX[(size_t)s * nI * 3 + i];
    for (int i = threadIdx.x; i < 4 * nI; i += blockDim.x) sS[i] = src[(size_t)s * 4 * nI + i];
    __syncthreads();
    if (mi < nI) {
      for (int mj = 0; mj < nI; ++mj) {
        double dx = xt0 - sX[3 * mj], dy = xt1 - sX[3 * mj + 1], dz = xt2 - sX[3 * mj + 2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double sn, cs;
        sincos(kappa * r, &sn, &cs);
        double ir = 1.0 / r;
        double gr = cs * ir, gi = sn * ir;
        double2 v0 = sS[mj], v1 = sS[nI + mj], v2 = sS[2 * nI + mj], v3 = sS[3 * nI + mj];
        a0.x += gr * v0.x - gi * v0.y; a0.y += gr * v0.y + gi * v0.x;
        a1.x += gr * v1.x - gi * v1.y; a1.y += gr * v1.y + gi * v1.x;
        a2.x += gr * v2.x - gi * v2.y; a2.y += gr * v2.y + gi * v2.x;
        a3.x += gr * v3.x - gi * v3.y; a3.y += gr * v3.y + gi * v3.x;
      }
    }
  }
  if (mi < nI) {
    const double f = 0.25 / M_PI;
    double2 *o = acc + (size_t)t * 4 * nI;
    o[mi] = make_double2(f * a0.x, f * a0.y);
    o[nI + mi] = make_double2(f * a1.x, f * a1.y);
    o[2 * nI + mi] = make_double2(f * a2.x, f * a2.y);
    o[3 * nI + mi] = make_double2(f * a3.x, f * a3.y);
  }
}

// ------------------------------------------------------------------------ a6 M2L (FP32)
// Phase-split kernel: with centres c_t, c_s and r0 = |c_t - c_s|,
//   G = e^{i kappa r0} e^{i kappa (r - r0)} / (4 pi r),
// e^{i kappa r0} in FP64 once per pair; node offsets from the centres in FP32, and
// r - r0 = (2 d.delta + |delta|^2) / (r + r0) (d = c_t - c_s, delta = offset difference)
// without cancellation.  Each pair's FP32 sum is rotated by its FP64 phase and accumulated
// in FP64.
__global__ void k_m2l_f32(const int *__restrict__ targets, const int *__restrict__ fptr, const int *__restrict__ fsrc,
                          int nI, double kappa, const double *__restrict__ center, const float *__restrict__ nodeXf,
                          const float2 *__restrict__ src, double2 *__restrict__ acc) {
  int t = targets[blockIdx.x];
  extern __shared__ float smf[];
  float *sX = smf;                        // [nI][3]
  float2 *sS = (float2 *)(smf + 3 * nI + (3 * nI & 1));  // [4][nI]
  __shared__ double sPh[2];
  __shared__ float sD[4];
  int mi = threadIdx.x;
  float xt0 = 0, xt1 = 0, xt2 = 0;
  if (mi < nI) {
    xt0 = nodeXf[((size_t)t * nI + mi) * 3];
    xt1 = nodeXf[((size_t)t * nI + mi) * 3 + 1];
    xt2 = nodeXf[((size_t)t * nI + mi) * 3 + 2];
  }
  const double ct0 = center[4 * t], ct1 = center[4 * t + 1], ct2 = center[4 * t + 2];
  const float kf = (float)kappa;
  double2 a0 = make_double2(0, 0), a1 = a0, a2 = a0, a3 = a0;
  for (int k = fptr[t]; k < fptr[t + 1]; ++k) {
    int s = fsrc[k];
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nI; i += blockDim.x) sX[i] = nodeXf[(size_t)s * nI * 3 + i];
    for (int i = threadIdx.x; i < 4 * nI; i += blockDim.x) sS[i] = src[(size_t)s * 4 * nI + i];
    if (threadIdx.x == 0) {
      double d0 = ct0 - center[4 * s], d1 = ct1 - center[4 * s + 1], d2 = ct2 - center[4 * s + 2];
      double r0 = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      double sn, cs;
      sincos(kappa * r0, &sn, &cs);
      sPh[0] = cs * 0.25 / M_PI;
      sPh[1] = sn * 0.25 / M_PI;
      sD[0] = (float)d0;
      sD[1] = (float)d1;
      sD[2] = (float)d2;
      sD[3] = (float)r0;
    }
    __syncthreads();
    if (mi < nI) {
      const float d0 = sD[0], d1 = sD[1], d2 = sD[2], r0 = sD[3];
      float b0x = 0, b0y = 0, b1x = 0, b1y = 0, b2x = 0, b2y = 0, b3x = 0, b3y = 0;
      for (int mj = 0; mj < nI; ++mj) {
        float e0 = xt0 - sX[3 * mj], e1 = xt1 - sX[3 * mj + 1], e2 = xt2 - sX[3 * mj + 2];
        float v0 = d0 + e0, v1 = d1 + e1, v2 = d2 + e2;
        float r2 = v0 * v0 + v1 * v1 + v2 * v2;
        float r = sqrtf(r2);
        float dr = (2.f * (d0 * e0 + d1 * e1 + d2 * e2) + (e0 * e0 + e1 * e1 + e2 * e2)) / (r + r0);
        float sn, cs;
        sincosf(kf * dr, &sn, &cs);
        float ir = 1.f / r;
        float gr = cs * ir, gi = sn * ir;
        float2 w0 = sS[mj], w1 = sS[nI + mj], w2 = sS[2 * nI + mj], w3 = sS[3 * nI + mj];
        b0x += gr * w0.x - gi * w0.y; b0y += gr * w0.y + gi * w0.x;
        b1x += gr * w1.x - gi * w1.y; b1y += gr * w1.y + gi * w1.x;
        b2x += gr * w2.x - gi * w2.y; b2y += gr * w2.y + gi * w2.x;
        b3x += gr * w3.x - gi * w3.y; b3y += gr * w3.y + gi * w3.x;
      }
      const double pr = sPh[0], pi = sPh[1];
      a0.x += pr * b0x - pi * b0y; a0.y += pr * b0y + pi * b0x;
      a1.x += pr * b1x - pi * b1y; a1.y += pr * b1y + pi * b1x;
      a2.x += pr * b2x - pi * b2y; a2.y += pr * b2y + pi * b2x;
      a3.x += pr * b3x - pi * b3y; a3.y += pr * b3y + pi * b3x;
    }
  }
  if (mi < nI) {
    double2 *o = acc + (size_t)t * 4 * nI;
    o[mi] = a0;
    o[nI + mi] = a1;
    o[2 * nI + mi] = a2;
    o[3 * nI + mi] = a3;
  }
}

// ------------------------------------------------------------------------ a7 L2L
// child_c(f, m2', m1') += sum_{m2} E[c2][m2][m2'] sum_{m1} E[c1][m1][m1'] parent(f, m2, m1)
template <class R>
__global__ void k_l2l(int nparent, int par_off, int ch_off, int q1, const double *__restrict__ Et,
                      C2<R> *__restrict__ loc) {
  int pid = blockIdx.x;
  if (pid >= nparent) return;
  int nI = q1 * q1;
  extern __shared__ unsigned char smraw[];
  R *sE = (R *)smraw;
  C2<R> *par = (C2<R> *)(smraw + sizeof(double) * 2 * kMaxQ1 * kMaxQ1);  // [3][nI]
  C2<R> *T = par + 3 * nI;                                              // [2][3][q1 m2][q1 m1']
  for (int i = threadIdx.x; i < 2 * q1 * q1; i += blockDim.x) sE[i] = (R)Et[i];
  const C2<R> *pl = loc + (size_t)(par_off + pid) * 3 * nI;
  for (int i = threadIdx.x; i < 3 * nI; i += blockDim.x) par[i] = pl[i];
  __syncthreads();
  for (int i = threadIdx.x; i < 6 * nI; i += blockDim.x) {
    int c1 = i / (3 * nI), rem = i % (3 * nI), f = rem / nI, r2 = rem % nI, m2 = r2 / q1, m1p = r2 % q1;
    C2<R> s = mk<R>(0, 0);
    const C2<R> *pp = par + f * nI + m2 * q1;
    for (int m1 = 0; m1 < q1; ++m1) {
      R e = sE[(c1 * q1 + m1) * q1 + m1p];
      s.x += e * pp[m1].x;
      s.y += e * pp[m1].y;
    }
    T[i] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 12 * nI; i += blockDim.x) {
    int cidx = i / (3 * nI), rem = i % (3 * nI), f = rem / nI, r2 = rem % nI, m2p = r2 / q1, m1p = r2 % q1;
    int c1 = cidx & 1, c2 = cidx >> 1;
    const C2<R> *tt = T + (c1 * 3 + f) * nI;
    C2<R> s = mk<R>(0, 0);
    for (int m2 = 0; m2 < q1; ++m2) {
      R e = sE[(c2 * q1 + m2) * q1 + m2p];
      s.x += e * tt[m2 * q1 + m1p].x;
      s.y += e * tt[m2 * q1 + m1p].y;
    }
    C2<R> *cl = loc + (size_t)(ch_off + 4 * pid + cidx) * 3 * nI;
    C2<R> o = cl[f * nI + r2];
    o.x += s.x;
    o.y += s.y;
    cl[f * nI + r2] = o;
  }
}

// ------------------------------------------------------------------------ a8 leaf evaluation
// y*_{0,b,a} = h^2 sum_m M[m1][a] M[m2][b] l_0(m) + h sum_m Md[m1][a] M[m2][b] l_div(m)
// y*_{1,b,a} = h^2 sum_m M[m1][a] M[m2][b] l_1(m) + h sum_m M[m1][a] Md[m2][b] l_div(m)
template <class R>
__global__ void k_leaf_eval(int nE, int leaf_off, int p1, int q1, R h, const double *__restrict__ Mt,
                            const double *__restrict__ Mdt, const C2<R> *__restrict__ loc, double2 *__restrict__ ys) {
  int e = blockIdx.x;
  if (e >= nE) return;
  int nI = q1 * q1;
  __shared__ R sM[kMaxQ1 * kMaxP1], sMd[kMaxQ1 * kMaxP1];
  __shared__ C2<R> R0[kMaxQ1 * kMaxP1], R1[kMaxQ1 * kMaxP1], R2[kMaxQ1 * kMaxP1], Rd[kMaxQ1 * kMaxP1];
  for (int i = threadIdx.x; i < q1 * p1; i += blockDim.x) {
    sM[i] = (R)Mt[i];
    sMd[i] = (R)Mdt[i];
  }
  __syncthreads();
  const C2<R> *l = loc + (size_t)(leaf_off + e) * 3 * nI;
  for (int i = threadIdx.x; i < q1 * p1; i += blockDim.x) {
    int m2 = i / p1, a = i % p1;
    C2<R> s0 = mk<R>(0, 0), s1 = s0, s2 = s0, sd = s0;
    for (int m1 = 0; m1 < q1; ++m1) {
      R M = sM[m1 * p1 + a], Md = sMd[m1 * p1 + a];
      C2<R> v0 = l[m2 * q1 + m1], v1 = l[nI + m2 * q1 + m1], v2 = l[2 * nI + m2 * q1 + m1];
      s0.x += M * v0.x; s0.y += M * v0.y;
      s1.x += M * v1.x; s1.y += M * v1.y;
      s2.x += M * v2.x; s2.y += M * v2.y;
      sd.x += Md * v2.x; sd.y += Md * v2.y;
    }
    R0[i] = s0;
    R1[i] = s1;
    R2[i] = s2;
    Rd[i] = sd;
  }
  __syncthreads();
  R h2 = h * h;
  for (int i = threadIdx.x; i < 2 * p1 * p1; i += blockDim.x) {
    int al = i / (p1 * p1), b = (i / p1) % p1, a = i % p1;
    R ax = 0, ay = 0;
    for (int m2 = 0; m2 < q1; ++m2) {
      R M = sM[m2 * p1 + b], Md = sMd[m2 * p1 + b];
      if (al == 0) {
        C2<R> u = R0[m2 * p1 + a], d = Rd[m2 * p1 + a];
        ax += h2 * M * u.x + h * M * d.x;
        ay += h2 * M * u.y + h * M * d.y;
      } else {
        C2<R> u = R1[m2 * p1 + a], d = R2[m2 * p1 + a];
        ax += h2 * M * u.x + h * Md * d.x;
        ay += h2 * M * u.y + h * Md * d.y;
      }
    }
    ys[(size_t)e * 2 * p1 * p1 + i] = make_double2((double)ax, (double)ay);
  }
}

// ------------------------------------------------------------------------ drivers
static size_t m2m_smem(int q1, size_t csz) { return sizeof(double) * 2 * kMaxQ1 * kMaxQ1 + csz * 24 * q1 * q1; }
static size_t l2l_smem(int q1, size_t csz) { return sizeof(double) * 2 * kMaxQ1 * kMaxQ1 + csz * 9 * q1 * q1; }

template <class R>
static efie_status far_chain(Ctx *c, const double2 *xs, double2 *ys, C2<R> *mom, C2<R> *srcv, C2<R> *loc,
                             const double *M, const double *Md, const double *E) {
  const int nI = c->nI, q1 = c->q1, p1 = c->p1, m = c->m;
  const R h = (R)(1.0 / c->n);
  cudaStream_t st = c->stream;
  size_t csz = sizeof(C2<R>);
  k_leaf_moments<R><<<c->nE, 128, 0, st>>>(c->nE, c->lev_off[m], p1, q1, h, M, Md, xs, mom); ++c->launches;
  for (int l = m - 1; l >= 0; --l) {
    int npar = c->np << (2 * l);
    k_m2m<R><<<npar, 128, m2m_smem(q1, csz), st>>>(npar, c->lev_off[l], c->lev_off[l + 1], q1, E, mom); ++c->launches;
  }
  long long tot = (long long)c->ncl * nI;
  k_fold<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, nI, c->d_nodeD, mom, srcv); ++c->launches;
  cudaEventRecord(c->tm.ev[3], st);
  int thr = ((nI + 31) / 32) * 32;
  if (c->n_m2l_targets > 0) {
    if (sizeof(R) == 8) {
      size_t sm = sizeof(double) * (3 * nI + 1) + sizeof(double2) * 4 * nI;
      k_m2l_f64<<<c->n_m2l_targets, thr, sm, st>>>(c->d_m2l_targets, c->d_far_ptr, c->d_far_src, nI, c->kappa,
                                                   c->d_nodeX, (const double2 *)srcv, c->d_acc); ++c->launches;
    } else {
      size_t sm = sizeof(float) * (3 * nI + 1) + sizeof(float2) * 4 * nI;
      k_m2l_f32<<<c->n_m2l_targets, thr, sm, st>>>(c->d_m2l_targets, c->d_far_ptr, c->d_far_src, nI, c->kappa,
                                                   c->d_center, c->d_nodeXf, (const float2 *)srcv, c->d_acc); ++c->launches;
    }
  }
  cudaEventRecord(c->tm.ev[4], st);
  k_unfold<R, double2><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, nI, (R)(1.0 / (c->kappa * c->kappa)),
                                                                     c->d_nodeD, c->d_acc, loc); ++c->launches;
  for (int l = 0; l < m; ++l) {
    int npar = c->np << (2 * l);
    k_l2l<R><<<npar, 128, l2l_smem(q1, csz), st>>>(npar, c->lev_off[l], c->lev_off[l + 1], q1, E, loc); ++c->launches;
  }
  k_leaf_eval<R><<<c->nE, 128, 0, st>>>(c->nE, c->lev_off[m], p1, q1, h, M, Md, loc, ys); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

efie_status dev_set_kernel_attrs(Ctx *c) {
  size_t mx = 0;
  for (size_t csz : {sizeof(double2), sizeof(float2)}) mx = std::max(mx, m2m_smem(c->q1, csz));
  EFIE_CUDA(cudaFuncSetAttribute(k_m2m<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
  EFIE_CUDA(cudaFuncSetAttribute(k_m2m<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
  EFIE_CUDA(cudaFuncSetAttribute(k_l2l<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
  EFIE_CUDA(cudaFuncSetAttribute(k_l2l<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
  return EFIE_OK;
}

// ys = (N + F) xs; the near field runs on the second stream, concurrently with the far
// chain, into its own buffer; both are summed by the caller (scatter) or here.
static efie_status superspace_apply(Ctx *c, const double2 *xs, double2 *ys, double2 *ysn) {
  cudaStream_t st = c->stream;
  EFIE_CUDA(cudaEventRecord(c->fork, st));
  EFIE_CUDA(cudaStreamWaitEvent(c->stream2, c->fork, 0));
  EFIE_TRY(dev_near_apply(c, xs, ysn, c->stream2));
  EFIE_CUDA(cudaEventRecord(c->tm.ev[2], c->stream2));
  EFIE_CUDA(cudaEventRecord(c->join, c->stream2));
  if (c->opt.precision == EFIE_MIXED_FP32) {
    EFIE_TRY(far_chain<float>(c, xs, ys, c->d_momf, c->d_srcf, c->d_locf, c->d_M, c->d_Md, c->d_E));
  } else {
    EFIE_TRY(far_chain<double>(c, xs, ys, c->d_mom, c->d_src, c->d_loc, c->d_M, c->d_Md, c->d_E));
  }
  EFIE_CUDA(cudaEventRecord(c->tm.ev[5], st));
  EFIE_CUDA(cudaStreamWaitEvent(st, c->join, 0));
  return EFIE_OK;
}

efie_status dev_matvec_super(Ctx *c, const double2 *xs, double2 *ys) {
  cudaEventRecord(c->tm.ev[0], c->stream);
  cudaEventRecord(c->tm.ev[1], c->stream);
  EFIE_TRY(superspace_apply(c, xs, ys, c->d_ysn));
  k_add<<<(c->nsup + 255) / 256, 256, 0, c->stream>>>(c->nsup, ys, c->d_ysn); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  cudaEventRecord(c->tm.ev[6], c->stream);
  return EFIE_OK;
}

efie_status dev_matvec(Ctx *c, const double2 *x, double2 *y) {
  cudaStream_t st = c->stream;
  EFIE_CUDA(cudaEventRecord(c->tm.ev[0], st));
  k_gather<<<(c->nsup + 255) / 256, 256, 0, st>>>(c->nsup, c->d_tg_ptr, c->d_tg_col, c->d_tg_val, x, c->d_xs); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_CUDA(cudaEventRecord(c->tm.ev[1], st));
  EFIE_TRY(superspace_apply(c, c->d_xs, c->d_ys, c->d_ysn));
  k_scatter<<<(c->ndof + 255) / 256, 256, 0, st>>>(c->ndof, c->d_ts_ptr, c->d_ts_col, c->d_ts_val, c->d_ys, c->d_ysn,
                                                  y); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_CUDA(cudaEventRecord(c->tm.ev[6], st));
  return EFIE_OK;
}

efie_status dev_scatter(Ctx *c, const double2 *ys, double2 *y) {
  k_scatter<<<(c->ndof + 255) / 256, 256, 0, c->stream>>>(c->ndof, c->d_ts_ptr, c->d_ts_col, c->d_ts_val, ys, nullptr,
                                                         y); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

efie_status dev_gather(Ctx *c, const double2 *x, double2 *xs) {
  k_gather<<<(c->nsup + 255) / 256, 256, 0, c->stream>>>(c->nsup, c->d_tg_ptr, c->d_tg_col, c->d_tg_val, x, xs); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

efie_status dev_alloc_work(Ctx *c) {
  size_t ncl = c->ncl, nI = c->nI;
  EFIE_TRY(dalloc(c, &c->d_x, c->ndof));
  EFIE_TRY(dalloc(c, &c->d_y, c->ndof));
  EFIE_TRY(dalloc(c, &c->d_xs, c->nsup));
  EFIE_TRY(dalloc(c, &c->d_ys, c->nsup));
  EFIE_TRY(dalloc(c, &c->d_ysn, c->nsup));
  EFIE_TRY(dalloc(c, &c->d_acc, ncl * 4 * nI));
  EFIE_CUDA(cudaMemset(c->d_acc, 0, sizeof(double2) * ncl * 4 * nI));
  if (c->opt.precision == EFIE_MIXED_FP32) {
    EFIE_TRY(dalloc(c, &c->d_momf, ncl * 3 * nI));
    EFIE_TRY(dalloc(c, &c->d_srcf, ncl * 4 * nI));
    EFIE_TRY(dalloc(c, &c->d_locf, ncl * 3 * nI));
  } else {
    EFIE_TRY(dalloc(c, &c->d_mom, ncl * 3 * nI));
    EFIE_TRY(dalloc(c, &c->d_src, ncl * 4 * nI));
    EFIE_TRY(dalloc(c, &c->d_loc, ncl * 3 * nI));
  }
  EFIE_TRY(dalloc(c, &c->d_M, c->q1 * c->p1));
  EFIE_TRY(dalloc(c, &c->d_Md, c->q1 * c->p1));
  EFIE_TRY(dalloc(c, &c->d_E, 2 * c->q1 * c->q1));
  EFIE_CUDA(cudaMemcpy(c->d_M, c->tab.M.data(), 8 * c->tab.M.size(), cudaMemcpyHostToDevice));
  EFIE_CUDA(cudaMemcpy(c->d_Md, c->tab.Md.data(), 8 * c->tab.Md.size(), cudaMemcpyHostToDevice));
  EFIE_CUDA(cudaMemcpy(c->d_E, c->tab.E.data(), 8 * c->tab.E.size(), cudaMemcpyHostToDevice));
  EFIE_CUDA(cudaDeviceSynchronize());
  return dev_set_kernel_attrs(c);
}

}  // namespace efie
