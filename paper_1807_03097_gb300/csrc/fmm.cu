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
#include "fastmath.cuh"

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
                               const double *__restrict__ Mdt, const double2 *__restrict__ xs, C2<R> *__restrict__ mom,
                               size_t xstride = 0, size_t mstride = 0) {
  int e = blockIdx.x;
  if (e >= nE) return;
  xs += blockIdx.y * xstride;  // right-hand side blockIdx.y of a batch
  mom += blockIdx.y * mstride;
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
                      C2<R> *__restrict__ mom, size_t mstride = 0) {
  int pid = blockIdx.x;
  if (pid >= nparent) return;
  mom += blockIdx.y * mstride;
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

// ------------------------------------------------------------------------ a6 M2L (FP32, node-major)
// Folded source fields of the FP32 path, node-major: src[(id nI + m) 2] = (u_x, u_y),
// src[(id nI + m) 2 + 1] = (u_z, nu).
__global__ void k_fold_f32n(long long tot, int nI, const double *__restrict__ nodeD, const float2 *__restrict__ mom,
                            float4 *__restrict__ src) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  int id = (int)(t / nI), mi = (int)(t % nI);
  const double *D = nodeD + 6 * t;
  const float2 *mm = mom + (size_t)id * 3 * nI;
  float2 m0 = mm[mi], m1 = mm[nI + mi], nu = mm[2 * nI + mi];
  float u[6];
  for (int k = 0; k < 3; ++k) {
    float d1 = (float)D[k], d2 = (float)D[3 + k];
    u[2 * k] = d1 * m0.x + d2 * m1.x;
    u[2 * k + 1] = d1 * m0.y + d2 * m1.y;
  }
  src[2 * t] = make_float4(u[0], u[1], u[2], u[3]);
  src[2 * t + 1] = make_float4(u[4], u[5], nu.x, nu.y);
}

// Per far pair (CSR order): d = c_t - c_s and r0 = |d| in FP32, e^{i kappa r0} / (4 pi) from
// FP64.  Computed once at setup.
__global__ void k_pair_table(int ntarget, const int *__restrict__ targets, const int *__restrict__ fptr,
                             const int *__restrict__ fsrc, const double *__restrict__ center, double kappa,
                             float4 *__restrict__ pgeo, float2 *__restrict__ pph) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntarget) return;
  int t = targets[i];
  for (int k = fptr[t]; k < fptr[t + 1]; ++k) {
    int s = fsrc[k];
    double d0 = center[4 * t] - center[4 * s], d1 = center[4 * t + 1] - center[4 * s + 1],
           d2 = center[4 * t + 2] - center[4 * s + 2];
    double r0 = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    double sn, cs;
    sincos(kappa * r0, &sn, &cs);
    pgeo[k] = make_float4((float)d0, (float)d1, (float)d2, (float)r0);
    pph[k] = make_float2((float)(cs * 0.25 / M_PI), (float)(sn * 0.25 / M_PI));
  }
}

// s + e = a + b exactly (Knuth two-sum, branch-free); used for the compensated FP32
// accumulation of per-pair partial sums, which keeps the long sums over all source
// clusters close to FP64 accuracy
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b) {
  float s = hi + b;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (b - bp);
  hi = s;
  lo += err;
}

// d = a * b + c on two FP32 lanes at once (Blackwell packed FMA)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long A = *reinterpret_cast<unsigned long long *>(&a);
  unsigned long long B = *reinterpret_cast<unsigned long long *>(&b);
  unsigned long long C = *reinterpret_cast<unsigned long long *>(&c);
  unsigned long long D;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D) : "l"(A), "l"(B), "l"(C));
  return *reinterpret_cast<float2 *>(&D);
}

// FP32 M2L, one warp per target cluster; lane owns target nodes m = lane + j T (j < NT,
// T = ceil(nI / NT) <= 32) and sweeps the source nodes of every admissible source cluster two
// at a time, so that the kernel values of two entries (m, m'), (m, m'+1) are generated and
// applied with packed FP32 instructions (fma / add / mul .f32x2 on the pair).  With x_t, x_s
// the node offsets from the cluster centres, d = c_t - c_s and r0 = |d|:
//   MODE 0 (direct): r^2 = |u|^2 + |x_s|^2 - 2 u.x_s with u = d + x_t, phase = kappa r -
//     kappa r0; used when the host has checked that kappa * max r * 2^-24 < 5e-6 (a fixed
//     perturbation of the matrix of at most about 2e-5 rad per entry);
//   MODE 1 (split): num = r^2 - r0^2 = (|x_t|^2 + 2 d.x_t) + (|x_s|^2 - 2 d.x_s) - 2 x_t.x_s,
//     every term of the size of num (no cancellation against r0^2), r = sqrt(r0^2 + num),
//     phase = kappa (r - r0) = num / ((r + r0) / kappa); the host has checked that every phase
//     lies within +-100 pi;  MODE 2: MODE 1 plus a two-constant Cody-Waite reduction of the
//     phase to [-pi, pi] before the hardware sine / cosine.
// G = e^{i kappa r0}/(4 pi) * e^{i phase} / r.  The pair factor e^{i kappa r0}/(4 pi) is
// applied to the source fields while they are staged in shared memory.  Staging of a source
// pair k (nodes 2k, 2k+1; an odd last node is paired with a copy of itself with zero fields):
//   sC[2k]   = (-2x_e, -2x_o, -2y_e, -2y_o),  sC[2k+1] = (-2z_e, -2z_o, b_e, b_o)
//     (b = |x_s|^2 in MODE 0, |x_s|^2 - 2 d.x_s otherwise),
//   sF[6k..6k+5] = Re w (fields 0-1, 2-3), Im w (0-1, 2-3), -Im w (0-1, 2-3), each float4 holding
//     (field f even node, field f odd node, field f+1 even node, field f+1 odd node).
// Per pair the packed partial sums (even and odd source nodes separately) are folded and
// added to running sums over all source clusters with two-sum (compensated) addition; the
// running sums and their compensation terms live in shared memory ([NT][16][32 lanes] per warp,
// touched once per source cluster), which keeps the registers for the inner loop.
template <int NT, int MODE>
__global__ void __launch_bounds__(128, (NT <= 3 ? 4 : 2)) k_m2l_f32w(const int *__restrict__ targets, int ntarget,
                                                  const int *__restrict__ fptr, const int *__restrict__ fsrc,
                                                  const float4 *__restrict__ pgeo, const float2 *__restrict__ pph,
                                                  int nI, float kappa, const float4 *__restrict__ nodeX4,
                                                  const float4 *__restrict__ src, float4 *__restrict__ acc) {
  extern __shared__ float4 sm4[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (blockDim.x >> 5) + wib;
  if (wg >= ntarget) return;
  const int NSP = (nI + 1) >> 1;  // source node pairs
  float4 *sT = sm4 + (size_t)wib * (nI + 8 * NSP + 4 * 32 * NT);
  float4 *sC = sT + nI;   // [2 NSP]
  float4 *sF = sC + 2 * NSP;  // [6 NSP]
  float *sA = reinterpret_cast<float *>(sF + 6 * NSP);  // [NT][16][32]: running sums, compensation
  const int t = targets[wg];
  const int T = (nI + NT - 1) / NT;
  for (int i = lane; i < nI; i += 32) sT[i] = nodeX4[(size_t)t * nI + i];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int q = 0; q < 16; ++q) sA[(j * 16 + q) * 32 + lane] = 0.f;
  const float inv2pi = 0.15915494309189535f, c1 = 6.28318548202514648f, c2 = -1.7484555e-7f;
  const float kinv = 1.f / kappa;
  for (int k = fptr[t]; k < fptr[t + 1]; ++k) {
    const int s = fsrc[k];
    const float4 g = pgeo[k];
    const float2 ph = pph[k];
    __syncwarp();
    for (int i = lane; i < 2 * NSP; i += 32) {
      const int kp = i >> 1, e = i & 1;
      const int n = min(2 * kp + e, nI - 1);
      const bool real = 2 * kp + e < nI;
      const float4 x = nodeX4[(size_t)s * nI + n];
      float4 u = make_float4(0.f, 0.f, 0.f, 0.f), v = u;
      if (real) {
        u = src[2 * ((size_t)s * nI + n)];
        v = src[2 * ((size_t)s * nI + n) + 1];
      }
      const float bb = MODE == 0 ? x.x * x.x + x.y * x.y + x.z * x.z
                                 : x.x * x.x + x.y * x.y + x.z * x.z - 2.f * (g.x * x.x + g.y * x.y + g.z * x.z);
      // fields w_f = ph * (u.xy, u.zw, v.xy, v.zw)
      const float wr[4] = {ph.x * u.x - ph.y * u.y, ph.x * u.z - ph.y * u.w, ph.x * v.x - ph.y * v.y,
                           ph.x * v.z - ph.y * v.w};
      const float wi[4] = {ph.x * u.y + ph.y * u.x, ph.x * u.w + ph.y * u.z, ph.x * v.y + ph.y * v.x,
                           ph.x * v.w + ph.y * v.z};
      float *c = reinterpret_cast<float *>(sC + 2 * kp);
      c[e] = -2.f * x.x;
      c[2 + e] = -2.f * x.y;
      c[4 + e] = -2.f * x.z;
      c[6 + e] = bb;
      float *f = reinterpret_cast<float *>(sF + 6 * kp);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = (q >> 1) * 4 + (q & 1) * 2 + e;
        f[o] = wr[q];
        f[8 + o] = wi[q];
        f[16 + o] = -wi[q];
      }
    }
    __syncwarp();
    // per-lane constants of this pair for each target node
    float2 U[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int mi = lane + j * T;
      const float4 x = sT[(lane < T && mi < nI) ? mi : 0];
      float ax, ay, az, aa;
      if (MODE == 0) {
        ax = g.x + x.x;
        ay = g.y + x.y;
        az = g.z + x.z;
        aa = ax * ax + ay * ay + az * az;
      } else {
        ax = x.x;
        ay = x.y;
        az = x.z;
        aa = x.x * x.x + x.y * x.y + x.z * x.z + 2.f * (g.x * x.x + g.y * x.y + g.z * x.z);
      }
      U[j][0] = make_float2(ax, ax);
      U[j][1] = make_float2(ay, ay);
      U[j][2] = make_float2(az, az);
      U[j][3] = make_float2(aa, aa);
    }
    const float2 r0sq = make_float2(g.w * g.w, g.w * g.w), nkr0 = make_float2(-kappa * g.w, -kappa * g.w);
    const float2 kap2 = make_float2(kappa, kappa), kinv2 = make_float2(kinv, kinv);
    const float2 r0k = make_float2(g.w * kinv, g.w * kinv);
    float2 are[NT][4], aim[NT][4];  // this pair's packed partial sums (even, odd source nodes)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) are[j][q] = aim[j][q] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int kp = 0; kp < NSP; ++kp) {
      const float4 ca = sC[2 * kp], cb = sC[2 * kp + 1];
      const float2 sx = make_float2(ca.x, ca.y), sy = make_float2(ca.z, ca.w), sz = make_float2(cb.x, cb.y),
                   sb = make_float2(cb.z, cb.w);
      float2 gr[NT], gi[NT];
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        float2 v = __fadd2_rn(U[j][3], sb);
        v = __ffma2_rn(U[j][0], sx, v);
        v = __ffma2_rn(U[j][1], sy, v);
        v = __ffma2_rn(U[j][2], sz, v);
        float2 rinv, phs;
        if (MODE == 0) {
          rinv = make_float2(rsqrt_ftz(v.x), rsqrt_ftz(v.y));
          phs = __ffma2_rn(kap2, __fmul2_rn(v, rinv), nkr0);
        } else {
          const float2 r2 = __fadd2_rn(v, r0sq);
          rinv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
          const float2 den = __ffma2_rn(__fmul2_rn(r2, rinv), kinv2, r0k);
          phs = __fmul2_rn(v, make_float2(rcp_ftz(den.x), rcp_ftz(den.y)));
          if (MODE == 2) {
            const float2 qq = __fmul2_rn(phs, make_float2(inv2pi, inv2pi));
            const float2 qn = make_float2(-rintf(qq.x), -rintf(qq.y));
            phs = __ffma2_rn(qn, make_float2(c1, c1), phs);
            phs = __ffma2_rn(qn, make_float2(c2, c2), phs);
          }
        }
        const float2 sn = make_float2(sin_ftz(phs.x), sin_ftz(phs.y));
        const float2 cs = make_float2(cos_ftz(phs.x), cos_ftz(phs.y));
        gr[j] = __fmul2_rn(cs, rinv);
        gi[j] = __fmul2_rn(sn, rinv);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4 fr = sF[6 * kp + h], fi = sF[6 * kp + 2 + h], fn = sF[6 * kp + 4 + h];
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
          const int q = 2 * h + qq;
          const float2 wr = qq ? make_float2(fr.z, fr.w) : make_float2(fr.x, fr.y);
          const float2 wi = qq ? make_float2(fi.z, fi.w) : make_float2(fi.x, fi.y);
          const float2 wn = qq ? make_float2(fn.z, fn.w) : make_float2(fn.x, fn.y);
#pragma unroll
          for (int j = 0; j < NT; ++j) {
            are[j][q] = __ffma2_rn(gi[j], wn, __ffma2_rn(gr[j], wr, are[j][q]));
            aim[j][q] = __ffma2_rn(gi[j], wr, __ffma2_rn(gr[j], wi, aim[j][q]));
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float *h0 = sA + (j * 16 + 2 * q) * 32 + lane, *h1 = h0 + 32, *l0 = h0 + 8 * 32, *l1 = h1 + 8 * 32;
        float vh0 = *h0, vl0 = *l0, vh1 = *h1, vl1 = *l1;
        two_sum_acc(vh0, vl0, are[j][q].x + are[j][q].y);
        two_sum_acc(vh1, vl1, aim[j][q].x + aim[j][q].y);
        *h0 = vh0;
        *l0 = vl0;
        *h1 = vh1;
        *l1 = vl1;
      }
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    int mi = lane + j * T;
    if (lane < T && mi < nI) {
      float o[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) o[q] = sA[(j * 16 + q) * 32 + lane] + sA[(j * 16 + 8 + q) * 32 + lane];
      acc[2 * ((size_t)t * nI + mi)] = make_float4(o[0], o[1], o[2], o[3]);
      acc[2 * ((size_t)t * nI + mi) + 1] = make_float4(o[4], o[5], o[6], o[7]);
    }
  }
}

// FP32 M2L over unordered admissible pairs: every coupling tile K_ts (entries as in
// k_m2l_f32w) is evaluated once and applied in both directions, acc_t += K_ts w_s and
// acc_s += K_ts^T w_t (K is symmetric in the two clusters: it depends on |x_t - x_s| only).
// One warp per owner cluster t; lane l < T owns the target rows m = l + j T (j < NT).  The
// tile is swept along its diagonals: at step k lane l takes the source column c = (l + k) mod
// nI, so the row sums stay in the lane (forward) and the column sum of column c moves one lane
// down per step (shuffle) while it collects the rows of every lane (backward); lane 0 stores a
// column when its sum has passed all lanes, and the columns that started mid-way are completed
// after the sweep.  Column sums of a pair go to the pair's slot of `back`; a second kernel adds
// the slots of every non-owner cluster in a fixed order.  Row sums enter running sums over the
// pairs with two-sum compensation (shared memory, [NT][16][32] per warp).
template <int NT, int MODE>
__global__ void __launch_bounds__(128, (NT <= 3 ? 4 : 2)) k_m2l_sym(
    const int *__restrict__ targets, int ntarget, const int *__restrict__ optr, const int *__restrict__ osrc,
    const int *__restrict__ oslot, const float4 *__restrict__ pgeo, const float2 *__restrict__ pph, int nI,
    float kappa, const float4 *__restrict__ nodeX4, const float4 *__restrict__ src, float4 *__restrict__ acc,
    float4 *__restrict__ back) {
  extern __shared__ float4 sm4[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (blockDim.x >> 5) + wib;
  if (wg >= ntarget) return;
  float4 *sT = sm4 + (size_t)wib * (6 * nI + 4 * 32 * NT);
  float4 *sC = sT + nI;      // [nI] (-2x, -2y, -2z, b) of the source nodes
  float4 *sW = sC + nI;      // [nI][2] phase-rotated source fields
  float4 *sO = sW + 2 * nI;  // [nI][2] column sums of the pair
  float *sA = reinterpret_cast<float *>(sO + 2 * nI);
  const int t = targets[wg];
  const int T = (nI + NT - 1) / NT;
  const bool act = lane < T;
  for (int i = lane; i < nI; i += 32) sT[i] = nodeX4[(size_t)t * nI + i];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int q = 0; q < 16; ++q) sA[(j * 16 + q) * 32 + lane] = 0.f;
  const float inv2pi = 0.15915494309189535f, c1 = 6.28318548202514648f, c2 = -1.7484555e-7f;
  const float kinv = 1.f / kappa;
  for (int kp = optr[t]; kp < optr[t + 1]; ++kp) {
    const int s = osrc[kp], u = oslot[kp];
    const float4 g = pgeo[kp];
    const float2 ph = pph[kp];
    __syncwarp();
    for (int i = lane; i < nI; i += 32) {
      const float4 x = nodeX4[(size_t)s * nI + i];
      const float bb = MODE == 0 ? x.x * x.x + x.y * x.y + x.z * x.z
                                 : x.x * x.x + x.y * x.y + x.z * x.z - 2.f * (g.x * x.x + g.y * x.y + g.z * x.z);
      sC[i] = make_float4(-2.f * x.x, -2.f * x.y, -2.f * x.z, bb);
      const float4 a = src[2 * ((size_t)s * nI + i)], b = src[2 * ((size_t)s * nI + i) + 1];
      sW[2 * i] = make_float4(ph.x * a.x - ph.y * a.y, ph.x * a.y + ph.y * a.x, ph.x * a.z - ph.y * a.w,
                              ph.x * a.w + ph.y * a.z);
      sW[2 * i + 1] = make_float4(ph.x * b.x - ph.y * b.y, ph.x * b.y + ph.y * b.x, ph.x * b.z - ph.y * b.w,
                                  ph.x * b.w + ph.y * b.z);
    }
    __syncwarp();
    float U[NT][4], wt[NT][8], at[NT][8];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int m = lane + j * T;
      const bool ok = act && m < nI;
      const float4 x = sT[ok ? m : 0];
      if (MODE == 0) {
        U[j][0] = g.x + x.x;
        U[j][1] = g.y + x.y;
        U[j][2] = g.z + x.z;
        U[j][3] = U[j][0] * U[j][0] + U[j][1] * U[j][1] + U[j][2] * U[j][2];
      } else {
        U[j][0] = x.x;
        U[j][1] = x.y;
        U[j][2] = x.z;
        U[j][3] = x.x * x.x + x.y * x.y + x.z * x.z + 2.f * (g.x * x.x + g.y * x.y + g.z * x.z);
      }
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      if (ok) {
        a = src[2 * ((size_t)t * nI + m)];
        b = src[2 * ((size_t)t * nI + m) + 1];
      }
      wt[j][0] = ph.x * a.x - ph.y * a.y;
      wt[j][1] = ph.x * a.y + ph.y * a.x;
      wt[j][2] = ph.x * a.z - ph.y * a.w;
      wt[j][3] = ph.x * a.w + ph.y * a.z;
      wt[j][4] = ph.x * b.x - ph.y * b.y;
      wt[j][5] = ph.x * b.y + ph.y * b.x;
      wt[j][6] = ph.x * b.z - ph.y * b.w;
      wt[j][7] = ph.x * b.w + ph.y * b.z;
#pragma unroll
      for (int q = 0; q < 8; ++q) at[j][q] = 0.f;
    }
    const float r0 = g.w, r0sq = g.w * g.w, nkr0 = -kappa * g.w, r0k = g.w * kinv;
    float ac[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ac[q] = 0.f;
#pragma unroll 1
    for (int k = 0; k < nI; ++k) {
      int cix = lane + k;
      if (cix >= nI) cix -= nI;
      if (act) {
        const float4 c4 = sC[cix], w0 = sW[2 * cix], w1 = sW[2 * cix + 1];
        const float ws[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int j = 0; j < NT; ++j) {
          if (lane + j * T < nI) {
            const float v = fmaf(U[j][0], c4.x, fmaf(U[j][1], c4.y, fmaf(U[j][2], c4.z, U[j][3] + c4.w)));
            float rinv, phs;
            if (MODE == 0) {
              rinv = rsqrt_ftz(v);
              phs = fmaf(kappa, v * rinv, nkr0);
            } else {
              const float r2 = v + r0sq;
              rinv = rsqrt_ftz(r2);
              phs = v * rcp_ftz(fmaf(r2 * rinv, kinv, r0k));
              if (MODE == 2) {
                const float qn = -rintf(phs * inv2pi);
                phs = fmaf(qn, c1, phs);
                phs = fmaf(qn, c2, phs);
              }
            }
            const float gr = cos_ftz(phs) * rinv, gi = sin_ftz(phs) * rinv;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
              at[j][2 * f] = fmaf(gr, ws[2 * f], fmaf(-gi, ws[2 * f + 1], at[j][2 * f]));
              at[j][2 * f + 1] = fmaf(gr, ws[2 * f + 1], fmaf(gi, ws[2 * f], at[j][2 * f + 1]));
              ac[2 * f] = fmaf(gr, wt[j][2 * f], fmaf(-gi, wt[j][2 * f + 1], ac[2 * f]));
              ac[2 * f + 1] = fmaf(gr, wt[j][2 * f + 1], fmaf(gi, wt[j][2 * f], ac[2 * f + 1]));
            }
          }
        }
      }
      if (lane == 0) {
        sO[2 * k] = make_float4(ac[0], ac[1], ac[2], ac[3]);
        sO[2 * k + 1] = make_float4(ac[4], ac[5], ac[6], ac[7]);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) ac[q] = __shfl_down_sync(0xffffffffu, ac[q], 1);
    }
    __syncwarp();
    // columns 0 .. T-2 started mid-way: lane l now holds the rest of column l
    if (lane + 1 < T && lane < nI) {
      float4 o0 = sO[2 * lane], o1 = sO[2 * lane + 1];
      sO[2 * lane] = make_float4(o0.x + ac[0], o0.y + ac[1], o0.z + ac[2], o0.w + ac[3]);
      sO[2 * lane + 1] = make_float4(o1.x + ac[4], o1.y + ac[5], o1.z + ac[6], o1.w + ac[7]);
    }
    __syncwarp();
    for (int i = lane; i < 2 * nI; i += 32) back[(size_t)u * 2 * nI + i] = sO[i];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float *hp = sA + (j * 16 + q) * 32 + lane, *lp = hp + 8 * 32;
        float vh = *hp, vl = *lp;
        two_sum_acc(vh, vl, at[j][q]);
        *hp = vh;
        *lp = vl;
      }
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int m = lane + j * T;
    if (act && m < nI) {
      float o[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) o[q] = sA[(j * 16 + q) * 32 + lane] + sA[(j * 16 + 8 + q) * 32 + lane];
      acc[2 * ((size_t)t * nI + m)] = make_float4(o[0], o[1], o[2], o[3]);
      acc[2 * ((size_t)t * nI + m) + 1] = make_float4(o[4], o[5], o[6], o[7]);
    }
  }
}

// acc_c (node m) = [owner's row sums] + sum over the pairs where c is the other cluster of their
// column sums, added in list order with two-sum compensation.
__global__ void k_m2l_sym_reduce(int nred, const int *__restrict__ red, const int *__restrict__ optr,
                                 const int *__restrict__ pptr, const int *__restrict__ pslot, int nI,
                                 const float4 *__restrict__ back, float4 *__restrict__ acc) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)nred * nI) return;
  const int c = red[i / nI], m = (int)(i % nI);
  float h[8], l[8];
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
  if (optr[c + 1] > optr[c]) {
    a = acc[2 * ((size_t)c * nI + m)];
    b = acc[2 * ((size_t)c * nI + m) + 1];
  }
  h[0] = a.x; h[1] = a.y; h[2] = a.z; h[3] = a.w; h[4] = b.x; h[5] = b.y; h[6] = b.z; h[7] = b.w;
#pragma unroll
  for (int q = 0; q < 8; ++q) l[q] = 0.f;
  for (int j = pptr[c]; j < pptr[c + 1]; ++j) {
    const size_t o = ((size_t)pslot[j] * nI + m) * 2;
    const float4 x = back[o], y = back[o + 1];
    const float v[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) two_sum_acc(h[q], l[q], v[q]);
  }
  acc[2 * ((size_t)c * nI + m)] = make_float4(h[0] + l[0], h[1] + l[1], h[2] + l[2], h[3] + l[3]);
  acc[2 * ((size_t)c * nI + m) + 1] = make_float4(h[4] + l[4], h[5] + l[5], h[6] + l[6], h[7] + l[7]);
}

__global__ void k_unfold_f32n(long long tot, int nI, float ik2, const double *__restrict__ nodeD,
                              const float4 *__restrict__ acc, float2 *__restrict__ loc) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  int id = (int)(t / nI), mi = (int)(t % nI);
  const double *D = nodeD + 6 * t;
  float4 u = acc[2 * t], v = acc[2 * t + 1];
  float cr[3] = {u.x, u.z, v.x}, ci[3] = {u.y, u.w, v.y};
  float l0x = 0, l0y = 0, l1x = 0, l1y = 0;
  for (int k = 0; k < 3; ++k) {
    l0x += (float)D[k] * cr[k];
    l0y += (float)D[k] * ci[k];
    l1x += (float)D[3 + k] * cr[k];
    l1y += (float)D[3 + k] * ci[k];
  }
  float2 *l = loc + (size_t)id * 3 * nI;
  l[mi] = make_float2(l0x, l0y);
  l[nI + mi] = make_float2(l1x, l1y);
  l[2 * nI + mi] = make_float2(-ik2 * v.z, -ik2 * v.w);
}

// ------------------------------------------------------------------------ a6 M2L, stored matrices
// When they fit in device memory, the coupling matrices of all admissible blocks are
// evaluated once at setup, K[k][m'][m] = G(F_t(x_m) - F_s(x_m')) / (4 pi) (column m'
// contiguous over the target nodes m), and every product streams them from HBM.

__global__ void k_build_K_f64(long long total, int nI, const int *__restrict__ far_tgt, const int *__restrict__ fsrc,
                              double kappa, const double *__restrict__ nodeX, double2 *__restrict__ K) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const long long nI2 = (long long)nI * nI;
  const long long k = idx / nI2;
  const int rem = (int)(idx - k * nI2), mj = rem / nI, mi = rem % nI;
  const int t = far_tgt[k], s = fsrc[k];
  const double *xt = nodeX + ((size_t)t * nI + mi) * 3, *xs = nodeX + ((size_t)s * nI + mj) * 3;
  double dx = xt[0] - xs[0], dy = xt[1] - xs[1], dz = xt[2] - xs[2];
  double r = sqrt(dx * dx + dy * dy + dz * dz);
  double sn, cs;
  sincos(kappa * r, &sn, &cs);
  double f = 0.25 / (M_PI * r);
  K[idx] = make_double2(f * cs, f * sn);
}

// FP32 matrices from the phase-split form with correctly rounded sqrt / division and the
// full-range sine / cosine (evaluated once, so the accurate functions cost nothing per product).
__global__ void k_build_K_f32(long long total, int nI, const int *__restrict__ far_tgt, const int *__restrict__ fsrc,
                              const float4 *__restrict__ pgeo, const float2 *__restrict__ pph, float kappa,
                              const float4 *__restrict__ nodeX4, float2 *__restrict__ K) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const long long nI2 = (long long)nI * nI;
  const long long k = idx / nI2;
  const int rem = (int)(idx - k * nI2), mj = rem / nI, mi = rem % nI;
  const int t = far_tgt[k], s = fsrc[k];
  const float4 g = pgeo[k];
  const float2 ph = pph[k];
  const float4 xt = nodeX4[(size_t)t * nI + mi], xs = nodeX4[(size_t)s * nI + mj];
  float ex = xt.x - xs.x, ey = xt.y - xs.y, ez = xt.z - xs.z;
  float num = 2.f * (g.x * ex + g.y * ey + g.z * ez) + (ex * ex + ey * ey + ez * ez);
  float r = sqrtf(g.w * g.w + num);
  float phs = kappa * (num / (r + g.w));
  float sn, cs;
  sincosf(phs, &sn, &cs);
  float gr = cs / r, gi = sn / r;
  K[idx] = make_float2(ph.x * gr - ph.y * gi, ph.x * gi + ph.y * gr);
}

template <int NT>
__global__ void __launch_bounds__(128) k_m2l_f32_stored(const int *__restrict__ targets, int ntarget,
                                                        const int *__restrict__ fptr, const int *__restrict__ fsrc,
                                                        const float2 *__restrict__ K, int nI,
                                                        const float4 *__restrict__ src, float4 *__restrict__ acc) {
  extern __shared__ float4 sm4[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (blockDim.x >> 5) + wib;
  if (wg >= ntarget) return;
  float4 *sW = sm4 + (size_t)wib * 4 * nI;  // [nI][2] fields, then [nI][2] rotated copies
  float4 *sR = sW + 2 * nI;
  const int t = targets[wg];
  const int T = (nI + NT - 1) / NT;
  float ah[NT][8], al[NT][8];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int q = 0; q < 8; ++q) ah[j][q] = al[j][q] = 0.f;
  for (int k = fptr[t]; k < fptr[t + 1]; ++k) {
    const int s = fsrc[k];
    __syncwarp();
    for (int i = lane; i < nI; i += 32) {
      float4 u = src[2 * ((size_t)s * nI + i)], v = src[2 * ((size_t)s * nI + i) + 1];
      sW[2 * i] = u;
      sW[2 * i + 1] = v;
      sR[2 * i] = make_float4(-u.y, u.x, -u.w, u.z);
      sR[2 * i + 1] = make_float4(-v.y, v.x, -v.w, v.z);
    }
    __syncwarp();
    const float2 *Kk = K + (size_t)k * nI * nI;
    float2 a[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) a[j][q] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int mj = 0; mj < nI; ++mj) {
      const float4 wa = sW[2 * mj], wb = sW[2 * mj + 1], ra = sR[2 * mj], rb = sR[2 * mj + 1];
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int mi = lane + j * T;
        const float2 kv = (lane < T && mi < nI) ? __ldcs(Kk + (size_t)mj * nI + mi) : make_float2(0.f, 0.f);
        const float2 gr = make_float2(kv.x, kv.x), gi = make_float2(kv.y, kv.y);
        a[j][0] = ffma2(gi, make_float2(ra.x, ra.y), ffma2(gr, make_float2(wa.x, wa.y), a[j][0]));
        a[j][1] = ffma2(gi, make_float2(ra.z, ra.w), ffma2(gr, make_float2(wa.z, wa.w), a[j][1]));
        a[j][2] = ffma2(gi, make_float2(rb.x, rb.y), ffma2(gr, make_float2(wb.x, wb.y), a[j][2]));
        a[j][3] = ffma2(gi, make_float2(rb.z, rb.w), ffma2(gr, make_float2(wb.z, wb.w), a[j][3]));
      }
    }
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        two_sum_acc(ah[j][2 * q], al[j][2 * q], a[j][q].x);
        two_sum_acc(ah[j][2 * q + 1], al[j][2 * q + 1], a[j][q].y);
      }
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    int mi = lane + j * T;
    if (lane < T && mi < nI) {
      float o[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) o[q] = ah[j][q] + al[j][q];
      acc[2 * ((size_t)t * nI + mi)] = make_float4(o[0], o[1], o[2], o[3]);
      acc[2 * ((size_t)t * nI + mi) + 1] = make_float4(o[4], o[5], o[6], o[7]);
    }
  }
}

// FP64 form with stored matrices: warp per target cluster, fields [cluster][4][node].
template <int NT>
__global__ void __launch_bounds__(128) k_m2l_f64_stored(const int *__restrict__ targets, int ntarget,
                                                        const int *__restrict__ fptr, const int *__restrict__ fsrc,
                                                        const double2 *__restrict__ K, int nI,
                                                        const double2 *__restrict__ src, double2 *__restrict__ acc) {
  extern __shared__ double2 smd2[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (blockDim.x >> 5) + wib;
  if (wg >= ntarget) return;
  double2 *sS = smd2 + (size_t)wib * 4 * nI;
  const int t = targets[wg];
  const int T = (nI + NT - 1) / NT;
  double ar[NT][4], ai[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) ar[j][q] = ai[j][q] = 0.0;
  for (int k = fptr[t]; k < fptr[t + 1]; ++k) {
    const int s = fsrc[k];
    __syncwarp();
    for (int i = lane; i < 4 * nI; i += 32) sS[i] = src[(size_t)s * 4 * nI + i];
    __syncwarp();
    const double2 *Kk = K + (size_t)k * nI * nI;
#pragma unroll 2
    for (int mj = 0; mj < nI; ++mj) {
      double2 w[4] = {sS[mj], sS[nI + mj], sS[2 * nI + mj], sS[3 * nI + mj]};
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int mi = lane + j * T;
        const double2 kv = (lane < T && mi < nI) ? __ldcs(Kk + (size_t)mj * nI + mi) : make_double2(0.0, 0.0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ar[j][q] += kv.x * w[q].x - kv.y * w[q].y;
          ai[j][q] += kv.x * w[q].y + kv.y * w[q].x;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    int mi = lane + j * T;
    if (lane < T && mi < nI)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[(size_t)t * 4 * nI + q * nI + mi] = make_double2(ar[j][q], ai[j][q]);
  }
}

// ------------------------------------------------------------------------ a7 L2L
// child_c(f, m2', m1') += sum_{m2} E[c2][m2][m2'] sum_{m1} E[c1][m1][m1'] parent(f, m2, m1)
template <class R>
__global__ void k_l2l(int nparent, int par_off, int ch_off, int q1, const double *__restrict__ Et,
                      C2<R> *__restrict__ loc, size_t mstride = 0) {
  int pid = blockIdx.x;
  if (pid >= nparent) return;
  loc += blockIdx.y * mstride;
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
                            const double *__restrict__ Mdt, const C2<R> *__restrict__ loc, double2 *__restrict__ ys,
                            size_t mstride = 0, size_t ystride = 0) {
  int e = blockIdx.x;
  if (e >= nE) return;
  loc += blockIdx.y * mstride;  // right-hand side blockIdx.y of a batch
  ys += blockIdx.y * ystride;
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
constexpr int kM2LWarps = 4;

// per warp: target nodes, staged source pairs, running sums [NT][16][32] (NT = ceil(nI / 32))
static size_t m2l_f32_smem(int nI) {
  return sizeof(float4) * ((size_t)nI + 8 * (size_t)((nI + 1) / 2) + 4 * 32 * (size_t)((nI + 31) / 32)) * kM2LWarps;
}

static size_t m2l_sym_smem(int nI) {
  return sizeof(float4) * (6 * (size_t)nI + 4 * 32 * (size_t)((nI + 31) / 32)) * kM2LWarps;
}

template <int MODE>
static efie_status launch_m2l_sym_t(Ctx *c, cudaStream_t st) {
  const int nI = c->nI, NT = (nI + 31) / 32;
  const unsigned blocks = (unsigned)((c->n_own_targets + kM2LWarps - 1) / kM2LWarps);
  const size_t sm = m2l_sym_smem(nI);
  const float kf = (float)c->kappa;
  if (c->n_own_targets > 0) {
    switch (NT) {
#define EFIE_SYM_CASE(N)                                                                                     \
  case N:                                                                                                   \
    k_m2l_sym<N, MODE><<<blocks, 32 * kM2LWarps, sm, st>>>(c->d_own_targets, c->n_own_targets, c->d_own_ptr,   \
                                                          c->d_own_src, c->d_own_slot, c->d_own_pgeo,          \
                                                          c->d_own_pph, nI, kf, c->d_nodeX4, c->d_srcf,        \
                                                          c->d_accf, c->d_back);                               \
    ++c->launches;                                                                                          \
    break;
      EFIE_SYM_CASE(1)
      EFIE_SYM_CASE(2)
      EFIE_SYM_CASE(3)
      EFIE_SYM_CASE(4)
      EFIE_SYM_CASE(5)
      EFIE_SYM_CASE(6)
      EFIE_SYM_CASE(7)
      EFIE_SYM_CASE(8)
      EFIE_SYM_CASE(9)
      EFIE_SYM_CASE(10)
#undef EFIE_SYM_CASE
      default:
        c->err = "q too large for the FP32 M2L kernel";
        return EFIE_EINVAL;
    }
  }
  const long long tot = (long long)c->n_red * nI;
  if (tot > 0) {
    k_m2l_sym_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(c->n_red, c->d_red, c->d_own_ptr, c->d_par_ptr,
                                                                    c->d_par_slot, nI, c->d_back, c->d_accf);
    ++c->launches;
  }
  return EFIE_OK;
}

template <int MODE>
static efie_status launch_m2l_f32_t(Ctx *c, cudaStream_t st) {
  if (c->d_back) return launch_m2l_sym_t<MODE>(c, st);
  const int nI = c->nI, NT = (nI + 31) / 32;
  const unsigned blocks = (unsigned)((c->n_m2l_targets + kM2LWarps - 1) / kM2LWarps);
  const size_t sm = m2l_f32_smem(nI);
  const float kf = (float)c->kappa;
  switch (NT) {
#define EFIE_M2L_CASE(N)                                                                                      \
  case N:                                                                                                    \
    k_m2l_f32w<N, MODE><<<blocks, 32 * kM2LWarps, sm, st>>>(c->d_m2l_targets, c->n_m2l_targets, c->d_far_ptr,  \
                                                           c->d_far_src, c->d_pgeo, c->d_pph, nI, kf,          \
                                                           c->d_nodeX4, c->d_srcf, c->d_accf);                 \
    ++c->launches;                                                                                           \
    break;
    EFIE_M2L_CASE(1)
    EFIE_M2L_CASE(2)
    EFIE_M2L_CASE(3)
    EFIE_M2L_CASE(4)
    EFIE_M2L_CASE(5)
    EFIE_M2L_CASE(6)
    EFIE_M2L_CASE(7)
    EFIE_M2L_CASE(8)
    EFIE_M2L_CASE(9)
    EFIE_M2L_CASE(10)
#undef EFIE_M2L_CASE
    default:
      c->err = "q too large for the FP32 M2L kernel";
      return EFIE_EINVAL;
  }
  return EFIE_OK;
}

static efie_status launch_m2l_f32(Ctx *c, cudaStream_t st) {
  if (c->m2l_mode == 0) return launch_m2l_f32_t<0>(c, st);
  if (c->m2l_mode == 1) return launch_m2l_f32_t<1>(c, st);
  return launch_m2l_f32_t<2>(c, st);
}

static efie_status launch_m2l_stored(Ctx *c, cudaStream_t st, bool f32) {
  const int nI = c->nI, NT = (nI + 31) / 32;
  const unsigned blocks = (unsigned)((c->n_m2l_targets + kM2LWarps - 1) / kM2LWarps);
  const size_t sm = (f32 ? sizeof(float4) * 4 : sizeof(double2) * 4) * (size_t)nI * kM2LWarps;
  switch (NT) {
#define EFIE_M2LS_CASE(N)                                                                                      \
  case N:                                                                                                     \
    if (f32)                                                                                                  \
      k_m2l_f32_stored<N><<<blocks, 32 * kM2LWarps, sm, st>>>(c->d_m2l_targets, c->n_m2l_targets, c->d_far_ptr, \
                                                              c->d_far_src, (const float2 *)c->d_K, nI,        \
                                                              c->d_srcf, c->d_accf);                          \
    else                                                                                                      \
      k_m2l_f64_stored<N><<<blocks, 32 * kM2LWarps, sm, st>>>(c->d_m2l_targets, c->n_m2l_targets, c->d_far_ptr, \
                                                              c->d_far_src, (const double2 *)c->d_K, nI,       \
                                                              c->d_src, c->d_acc);                            \
    ++c->launches;                                                                                            \
    break;
    EFIE_M2LS_CASE(1)
    EFIE_M2LS_CASE(2)
    EFIE_M2LS_CASE(3)
    EFIE_M2LS_CASE(4)
    EFIE_M2LS_CASE(5)
    EFIE_M2LS_CASE(6)
    EFIE_M2LS_CASE(7)
    EFIE_M2LS_CASE(8)
    EFIE_M2LS_CASE(9)
    EFIE_M2LS_CASE(10)
#undef EFIE_M2LS_CASE
    default:
      c->err = "q too large for the stored-matrix M2L kernel";
      return EFIE_EINVAL;
  }
  return EFIE_OK;
}

// Decide whether the coupling matrices are kept (m2l_store option) and evaluate them.
static efie_status m2l_store_matrices(Ctx *c) {
  dfree(c, c->d_K);
  c->k_stored = false;
  if (c->nfar == 0 || c->opt.m2l_store == 1) return EFIE_OK;
  const bool f32 = c->opt.precision == EFIE_MIXED_FP32;
  const size_t nI2 = (size_t)c->nI * c->nI;
  const size_t bytes = (size_t)c->nfar * nI2 * (f32 ? sizeof(float2) : sizeof(double2));
  size_t freeb = 0, totb = 0;
  EFIE_CUDA(cudaMemGetInfo(&freeb, &totb));
  // auto: keep them for the FP64 form only (evaluating FP64 sine / cosine / sqrt is the
  // bottleneck of that form on this GPU, while the FP32 form evaluates faster than HBM can
  // stream the stored matrices)
  if (c->opt.m2l_store == 0 && (f32 || bytes > freeb / 2)) return EFIE_OK;
  if (pool_alloc(c, &c->d_K, bytes) != EFIE_OK) {
    c->d_K = nullptr;
    if (c->opt.m2l_store == 2) {
      c->err = "coupling matrices do not fit in device memory";
      return EFIE_ENOMEM;
    }
    return EFIE_OK;
  }
  const long long total = (long long)c->nfar * (long long)nI2;
  const unsigned grid = (unsigned)((total + 255) / 256);
  if (f32)
    k_build_K_f32<<<grid, 256, 0, c->stream>>>(total, c->nI, c->d_far_tgt, c->d_far_src, c->d_pgeo, c->d_pph,
                                               (float)c->kappa, c->d_nodeX4, (float2 *)c->d_K);
  else
    k_build_K_f64<<<grid, 256, 0, c->stream>>>(total, c->nI, c->d_far_tgt, c->d_far_src, c->kappa, c->d_nodeX,
                                               (double2 *)c->d_K);
  ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  const int smb = (int)(sizeof(double2) * 4 * kMaxQ1 * kMaxQ1 * kM2LWarps);
  for (auto f : {k_m2l_f32_stored<1>, k_m2l_f32_stored<2>, k_m2l_f32_stored<3>, k_m2l_f32_stored<4>,
                 k_m2l_f32_stored<5>, k_m2l_f32_stored<6>, k_m2l_f32_stored<7>, k_m2l_f32_stored<8>,
                 k_m2l_f32_stored<9>, k_m2l_f32_stored<10>})
    EFIE_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
  for (auto f : {k_m2l_f64_stored<1>, k_m2l_f64_stored<2>, k_m2l_f64_stored<3>, k_m2l_f64_stored<4>,
                 k_m2l_f64_stored<5>, k_m2l_f64_stored<6>, k_m2l_f64_stored<7>, k_m2l_f64_stored<8>,
                 k_m2l_f64_stored<9>, k_m2l_f64_stored<10>})
    EFIE_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smb));
  c->k_stored = true;
  return EFIE_OK;
}

template <int MODE>
static efie_status m2l_sym_attrs(int bytes) {
  cudaError_t e = cudaSuccess;
  for (auto f : {k_m2l_sym<1, MODE>, k_m2l_sym<2, MODE>, k_m2l_sym<3, MODE>, k_m2l_sym<4, MODE>,
                 k_m2l_sym<5, MODE>, k_m2l_sym<6, MODE>, k_m2l_sym<7, MODE>, k_m2l_sym<8, MODE>,
                 k_m2l_sym<9, MODE>, k_m2l_sym<10, MODE>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e == cudaSuccess ? EFIE_OK : EFIE_ECUDA;
}

template <int MODE>
static efie_status m2l_f32_attrs(int bytes) {
  cudaError_t e = cudaSuccess;
  for (auto f : {k_m2l_f32w<1, MODE>, k_m2l_f32w<2, MODE>, k_m2l_f32w<3, MODE>, k_m2l_f32w<4, MODE>,
                 k_m2l_f32w<5, MODE>, k_m2l_f32w<6, MODE>, k_m2l_f32w<7, MODE>, k_m2l_f32w<8, MODE>,
                 k_m2l_f32w<9, MODE>, k_m2l_f32w<10, MODE>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e == cudaSuccess ? EFIE_OK : EFIE_ECUDA;
}

static efie_status launch_m2l_f32(Ctx *c, cudaStream_t st);

// Best of 3 device times (CUDA events on the context stream) of the M2L as it is configured.
static efie_status time_m2l(Ctx *c, float *best) {
  EFIE_TRY(launch_m2l_f32(c, c->stream));  // warm-up
  *best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    EFIE_CUDA(cudaEventRecord(c->tm.ev[3], c->stream));
    EFIE_TRY(launch_m2l_f32(c, c->stream));
    EFIE_CUDA(cudaEventRecord(c->tm.ev[4], c->stream));
    EFIE_CUDA(cudaEventSynchronize(c->tm.ev[4]));
    float ms = 0.f;
    EFIE_CUDA(cudaEventElapsedTime(&ms, c->tm.ev[3], c->tm.ev[4]));
    *best = std::min(*best, ms);
  }
  return EFIE_OK;
}

// M2L autotuner (option m2l_pairs = 2): the ordered-pair kernel (one warp per target cluster,
// its whole far list) and the unordered-pair kernel (one warp per owner, each coupling tile
// applied both ways) are timed on this problem's blocks and the faster is kept; the other's
// buffers are returned.  Sources are zero during the timing (the work does not depend on them).
static efie_status m2l_autotune(Ctx *c) {
  if (c->n_m2l_targets == 0) return EFIE_OK;
  EFIE_CUDA(cudaMemsetAsync(c->d_srcf, 0, sizeof(float4) * (size_t)c->ncl * 2 * c->nI, c->stream));
  float t_sym = 0.f, t_ord = 0.f;
  EFIE_TRY(time_m2l(c, &t_sym));
  float4 *back = c->d_back;
  c->d_back = nullptr;
  efie_status s = time_m2l(c, &t_ord);
  c->d_back = back;
  EFIE_TRY(s);
  c->m2l_tune_ms[0] = t_ord;
  c->m2l_tune_ms[1] = t_sym;
  if (t_ord <= t_sym) {
    dfree(c, c->d_back);
    dfree(c, c->d_own_pgeo);
    dfree(c, c->d_own_pph);
  }
  EFIE_CUDA(cudaMemsetAsync(c->d_accf, 0, sizeof(float4) * (size_t)c->ncl * 2 * c->nI, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  return EFIE_OK;
}

// node offsets (float4) and the per-pair table of the FP32 M2L
static efie_status m2l_f32_tables(Ctx *c) {
  const size_t n = (size_t)c->ncl * c->nI;
  std::vector<float> xf(3 * n);
  EFIE_CUDA(cudaMemcpyAsync(xf.data(), c->d_nodeXf, 12 * n, cudaMemcpyDeviceToHost, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<float4> x4(n);
  for (size_t i = 0; i < n; ++i) x4[i] = make_float4(xf[3 * i], xf[3 * i + 1], xf[3 * i + 2], 0.f);
  EFIE_TRY(dalloc(c, &c->d_nodeX4, n));
  EFIE_CUDA(cudaMemcpyAsync(c->d_nodeX4, x4.data(), 16 * n, cudaMemcpyHostToDevice, c->stream));
  EFIE_TRY(dalloc(c, &c->d_pgeo, (size_t)std::max(c->nfar, 1)));
  EFIE_TRY(dalloc(c, &c->d_pph, (size_t)std::max(c->nfar, 1)));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  if (c->n_m2l_targets > 0) {
    k_pair_table<<<(c->n_m2l_targets + 127) / 128, 128, 0, c->stream>>>(c->n_m2l_targets, c->d_m2l_targets,
                                                                        c->d_far_ptr, c->d_far_src, c->d_center,
                                                                        c->kappa, c->d_pgeo, c->d_pph);
    ++c->launches;
    EFIE_CUDA(cudaGetLastError());
  }
  EFIE_TRY(m2l_f32_attrs<0>((int)m2l_f32_smem(kMaxQ1 * kMaxQ1)));
  EFIE_TRY(m2l_f32_attrs<1>((int)m2l_f32_smem(kMaxQ1 * kMaxQ1)));
  EFIE_TRY(m2l_f32_attrs<2>((int)m2l_f32_smem(kMaxQ1 * kMaxQ1)));
  // unordered-pair form (option m2l_pairs): the column sums of every pair take npairs x nI x 32
  // bytes; used when they fit in a quarter of the free memory, else the one-sided kernel runs
  dfree(c, c->d_back);
  if (c->opt.m2l_pairs >= 1 && c->npairs > 0) {
    size_t freeb = 0, totb = 0;
    EFIE_CUDA(cudaMemGetInfo(&freeb, &totb));
    const size_t bytes = (size_t)c->npairs * c->nI * 2 * sizeof(float4);
    if (bytes <= freeb / 4) {
      EFIE_TRY(dalloc(c, &c->d_own_pgeo, (size_t)c->npairs));
      EFIE_TRY(dalloc(c, &c->d_own_pph, (size_t)c->npairs));
      EFIE_TRY(dalloc(c, &c->d_back, (size_t)c->npairs * c->nI * 2));
      k_pair_table<<<(c->n_own_targets + 127) / 128, 128, 0, c->stream>>>(c->n_own_targets, c->d_own_targets,
                                                                          c->d_own_ptr, c->d_own_src, c->d_center,
                                                                          c->kappa, c->d_own_pgeo, c->d_own_pph);
      ++c->launches;
      EFIE_CUDA(cudaGetLastError());
      EFIE_TRY(m2l_sym_attrs<0>((int)m2l_sym_smem(kMaxQ1 * kMaxQ1)));
      EFIE_TRY(m2l_sym_attrs<1>((int)m2l_sym_smem(kMaxQ1 * kMaxQ1)));
      EFIE_TRY(m2l_sym_attrs<2>((int)m2l_sym_smem(kMaxQ1 * kMaxQ1)));
    }
  }
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  if (c->opt.m2l_pairs == 2 && c->d_back) EFIE_TRY(m2l_autotune(c));
  return EFIE_OK;
}
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
  const unsigned gtot = (unsigned)((tot + 255) / 256);
  if (sizeof(R) == 8) {
    k_fold<double><<<gtot, 256, 0, st>>>(tot, nI, c->d_nodeD, (const double2 *)mom, (double2 *)srcv); ++c->launches;
  } else {
    k_fold_f32n<<<gtot, 256, 0, st>>>(tot, nI, c->d_nodeD, (const float2 *)mom, c->d_srcf); ++c->launches;
  }
  cudaEventRecord(c->tm.ev[3], st);
  if (c->n_m2l_targets > 0 && c->k_stored) {
    EFIE_TRY(launch_m2l_stored(c, st, sizeof(R) == 4));
  } else if (c->n_m2l_targets > 0) {
    if (sizeof(R) == 8) {
      int thr = ((nI + 31) / 32) * 32;
      size_t sm = sizeof(double) * (3 * nI + 1) + sizeof(double2) * 4 * nI;
      k_m2l_f64<<<c->n_m2l_targets, thr, sm, st>>>(c->d_m2l_targets, c->d_far_ptr, c->d_far_src, nI, c->kappa,
                                                   c->d_nodeX, (const double2 *)srcv, c->d_acc); ++c->launches;
    } else {
      EFIE_TRY(launch_m2l_f32(c, st));
    }
  }
  cudaEventRecord(c->tm.ev[4], st);
  if (sizeof(R) == 8) {
    k_unfold<double, double2><<<gtot, 256, 0, st>>>(tot, nI, 1.0 / (c->kappa * c->kappa), c->d_nodeD, c->d_acc,
                                                    (double2 *)loc); ++c->launches;
  } else {
    k_unfold_f32n<<<gtot, 256, 0, st>>>(tot, nI, (float)(1.0 / (c->kappa * c->kappa)), c->d_nodeD, c->d_accf,
                                        (float2 *)loc); ++c->launches;
  }
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
    EFIE_TRY(far_chain<float>(c, xs, ys, c->d_momf, nullptr, c->d_locf, c->d_M, c->d_Md, c->d_E));
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
  EFIE_CUDA(cudaMemsetAsync(c->d_acc, 0, sizeof(double2) * ncl * 4 * nI, c->stream));
  if (c->opt.precision == EFIE_MIXED_FP32) {
    EFIE_TRY(dalloc(c, &c->d_momf, ncl * 3 * nI));
    EFIE_TRY(dalloc(c, &c->d_srcf, ncl * 2 * nI));
    EFIE_TRY(dalloc(c, &c->d_accf, ncl * 2 * nI));
    EFIE_CUDA(cudaMemsetAsync(c->d_accf, 0, sizeof(float4) * ncl * 2 * nI, c->stream));
    EFIE_TRY(dalloc(c, &c->d_locf, ncl * 3 * nI));
    EFIE_TRY(m2l_f32_tables(c));
  } else {
    EFIE_TRY(dalloc(c, &c->d_mom, ncl * 3 * nI));
    EFIE_TRY(dalloc(c, &c->d_src, ncl * 4 * nI));
    EFIE_TRY(dalloc(c, &c->d_loc, ncl * 3 * nI));
  }
  EFIE_TRY(dalloc(c, &c->d_M, c->q1 * c->p1));
  EFIE_TRY(dalloc(c, &c->d_Md, c->q1 * c->p1));
  EFIE_TRY(dalloc(c, &c->d_E, 2 * c->q1 * c->q1));
  EFIE_CUDA(cudaMemcpyAsync(c->d_M, c->tab.M.data(), 8 * c->tab.M.size(), cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(c->d_Md, c->tab.Md.data(), 8 * c->tab.Md.size(), cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(c->d_E, c->tab.E.data(), 8 * c->tab.E.size(), cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  EFIE_TRY(dev_set_kernel_attrs(c));
  return m2l_store_matrices(c);
}

}  // namespace efie

// ========================================================================================
// Several right-hand sides at once (mixed form).  The cheap stages run once per right-hand
// side; the M2L evaluates the coupling tile G(m, m') of every admissible block once into
// shared memory and applies it to the 4 fields of up to kRB right-hand sides.
namespace efie {

constexpr int kRB = 8;             // right-hand sides per M2L block
constexpr int kFB = 4 * kRB;       // fields per M2L block
constexpr int kMultiThreads = 256;
constexpr int kMultiMaxNI = 144;   // (q + 1)^2 limit of the shared-memory tile

// node-major folded sources of all right-hand sides: src[(id nI + m) ld + 4 r + {x, y, z, div}].
// The row stride ld = 4 x (allocated right-hand sides) does not change with R, so rows of
// clusters that receive no M2L stay zero whatever the number of right-hand sides of earlier
// products.
__global__ void k_fold_multi(long long tot, int nI, int R, int ld, size_t mstride, const double *__restrict__ nodeD,
                             const float2 *__restrict__ mom, float2 *__restrict__ src) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int id = (int)(t / nI), mi = (int)(t % nI);
  const double *D = nodeD + 6 * t;
  for (int r = 0; r < R; ++r) {
    const float2 *mm = mom + r * mstride + (size_t)id * 3 * nI;
    float2 m0 = mm[mi], m1 = mm[nI + mi], nu = mm[2 * nI + mi];
    float2 *o = src + (size_t)t * ld + 4 * r;
    for (int k = 0; k < 3; ++k) {
      float d1 = (float)D[k], d2 = (float)D[3 + k];
      o[k] = make_float2(d1 * m0.x + d2 * m1.x, d1 * m0.y + d2 * m1.y);
    }
    o[3] = nu;
  }
}

__global__ void k_unfold_multi(long long tot, int nI, int R, int ld, size_t lstride, float ik2,
                               const double *__restrict__ nodeD,
                               const float2 *__restrict__ acc, float2 *__restrict__ loc) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  const int id = (int)(t / nI), mi = (int)(t % nI);
  const double *D = nodeD + 6 * t;
  for (int r = 0; r < R; ++r) {
    const float2 *a = acc + (size_t)t * ld + 4 * r;
    float l0x = 0, l0y = 0, l1x = 0, l1y = 0;
    for (int k = 0; k < 3; ++k) {
      l0x += (float)D[k] * a[k].x;
      l0y += (float)D[k] * a[k].y;
      l1x += (float)D[3 + k] * a[k].x;
      l1y += (float)D[3 + k] * a[k].y;
    }
    float2 *l = loc + r * lstride + (size_t)id * 3 * nI;
    l[mi] = make_float2(l0x, l0y);
    l[nI + mi] = make_float2(l1x, l1y);
    l[2 * nI + mi] = make_float2(-ik2 * a[3].x, -ik2 * a[3].y);
  }
}

// One block per (target cluster, group of kRB right-hand sides).  Thread t owns field
// f = t % kFB of the group and the target nodes m = t / kFB + 8 k.  For every source cluster:
// stage its node offsets and the group's fields, evaluate the (q+1)^4 tile of
// e^{i kappa r0}/(4 pi) e^{i kappa (r - r0)}/r (same phase forms as the single-field kernel)
// into shared memory, multiply-accumulate, and add the pair's FP32 partial sums to the
// running sums with two-sum compensation.
template <int KM>
__global__ void __launch_bounds__(kMultiThreads) k_m2l_f32_multi(
    const int *__restrict__ targets, const int *__restrict__ fptr, const int *__restrict__ fsrc,
    const float4 *__restrict__ pgeo, const float2 *__restrict__ pph, int nI, float kappa, int mode,
    const float4 *__restrict__ nodeX4, int F, int ld, const float2 *__restrict__ src, float2 *__restrict__ acc) {
  extern __shared__ float4 smm[];
  float4 *sXt = smm;                              // [nI]
  float4 *sXs = sXt + nI;                         // [nI]
  float2 *sS = (float2 *)(sXs + nI);              // [nI][kFB]
  float2 *sG = sS + (size_t)nI * kFB;             // [nI][nI] (row: target node)
  const int t = targets[blockIdx.x];
  const int f0 = blockIdx.y * kFB;
  const int tid = threadIdx.x, f = tid % kFB, mg = tid / kFB;
  const bool fval = f0 + f < F;
  for (int i = tid; i < nI; i += blockDim.x) sXt[i] = nodeX4[(size_t)t * nI + i];
  float ah[KM][2], al[KM][2];
#pragma unroll
  for (int k = 0; k < KM; ++k) ah[k][0] = ah[k][1] = al[k][0] = al[k][1] = 0.f;
  const float inv2pi = 0.15915494309189535f, c1 = 6.28318548202514648f, c2 = -1.7484555e-7f;
  for (int kk = fptr[t]; kk < fptr[t + 1]; ++kk) {
    const int s = fsrc[kk];
    const float4 g = pgeo[kk];
    const float2 ph = pph[kk];
    __syncthreads();
    for (int i = tid; i < nI; i += blockDim.x) sXs[i] = nodeX4[(size_t)s * nI + i];
    for (int i = tid; i < nI * kFB; i += blockDim.x) {
      const int mj = i / kFB, ff = i % kFB;
      sS[i] = (f0 + ff < F) ? src[((size_t)s * nI + mj) * ld + f0 + ff] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float r0 = g.w, r0sq = g.w * g.w, kr0 = kappa * g.w;
    for (int e = tid; e < nI * nI; e += blockDim.x) {
      const int mi = e / nI, mj = e % nI;
      const float4 xt = sXt[mi], xs = sXs[mj];
      float ex = xt.x - xs.x, ey = xt.y - xs.y, ez = xt.z - xs.z, rinv, phs;
      if (mode == 0) {
        float vx = g.x + ex, vy = g.y + ey, vz = g.z + ez;
        float r2 = vx * vx + vy * vy + vz * vz;
        rinv = rsqrt_ftz(r2);
        phs = fmaf(kappa, r2 * rinv, -kr0);
      } else {
        float num = fmaf(2.f, g.x * ex + g.y * ey + g.z * ez, ex * ex + ey * ey + ez * ez);
        float r2 = r0sq + num;
        rinv = rsqrt_ftz(r2);
        phs = kappa * num * rcp_ftz(r2 * rinv + r0);
        if (mode == 2) {
          float q = rintf(phs * inv2pi);
          phs = fmaf(-q, c1, phs);
          phs = fmaf(-q, c2, phs);
        }
      }
      const float sn = sin_ftz(phs), cs = cos_ftz(phs);
      const float gr = cs * rinv, gi = sn * rinv;
      sG[e] = make_float2(ph.x * gr - ph.y * gi, ph.x * gi + ph.y * gr);
    }
    __syncthreads();
    float pr[KM], pim[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) pr[k] = pim[k] = 0.f;
    for (int mj = 0; mj < nI; ++mj) {
      const float2 sv = sS[mj * kFB + f];
#pragma unroll
      for (int k = 0; k < KM; ++k) {
        const int mi = mg + 8 * k;
        if (mi < nI) {
          const float2 gv = sG[mi * nI + mj];
          pr[k] = fmaf(gv.x, sv.x, fmaf(-gv.y, sv.y, pr[k]));
          pim[k] = fmaf(gv.x, sv.y, fmaf(gv.y, sv.x, pim[k]));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      two_sum_acc(ah[k][0], al[k][0], pr[k]);
      two_sum_acc(ah[k][1], al[k][1], pim[k]);
    }
  }
  if (fval) {
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      const int mi = mg + 8 * k;
      if (mi < nI) acc[((size_t)t * nI + mi) * ld + f0 + f] = make_float2(ah[k][0] + al[k][0], ah[k][1] + al[k][1]);
    }
  }
}

static size_t multi_smem(int nI) {
  return sizeof(float4) * 2 * nI + sizeof(float2) * ((size_t)nI * kFB + (size_t)nI * nI);
}

efie_status dev_batch_alloc(Ctx *c, int R) {
  if (R <= c->batch_cap) return EFIE_OK;
  const size_t ncl = c->ncl, nI = c->nI;
  EFIE_TRY(dalloc(c, &c->d_xB, (size_t)R * c->ndof));
  EFIE_TRY(dalloc(c, &c->d_yB, (size_t)R * c->ndof));
  EFIE_TRY(dalloc(c, &c->d_xsB, (size_t)R * c->nsup));
  EFIE_TRY(dalloc(c, &c->d_ysB, (size_t)R * c->nsup));
  EFIE_TRY(dalloc(c, &c->d_ysnB, (size_t)R * c->nsup));
  EFIE_TRY(dalloc(c, &c->d_momB, (size_t)R * ncl * 3 * nI));
  EFIE_TRY(dalloc(c, &c->d_srcB, (size_t)R * ncl * 4 * nI));
  EFIE_TRY(dalloc(c, &c->d_accB, (size_t)R * ncl * 4 * nI));
  EFIE_CUDA(cudaMemsetAsync(c->d_accB, 0, sizeof(float2) * (size_t)R * ncl * 4 * nI, c->stream));
  EFIE_TRY(dalloc(c, &c->d_locB, (size_t)R * ncl * 3 * nI));
  if (c->opt.precision == EFIE_MIXED_FP32 && m2l_tc_supported(c)) EFIE_TRY(m2l_tc_prepare(c));
  const int sm = (int)multi_smem(kMultiMaxNI);
  for (auto fn : {k_m2l_f32_multi<1>, k_m2l_f32_multi<2>, k_m2l_f32_multi<4>, k_m2l_f32_multi<8>,
                  k_m2l_f32_multi<12>, k_m2l_f32_multi<16>, k_m2l_f32_multi<18>})
    EFIE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  c->batch_cap = R;
  return EFIE_OK;
}

__global__ void k_sum2(size_t n, const double2 *__restrict__ a, const double2 *__restrict__ b, double2 *__restrict__ y) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = make_double2(a[i].x + b[i].x, a[i].y + b[i].y);
}

// Y[r] = A X[r], r < R (host arrays of device pointers).  superspace: X[r] and Y[r] are
// superspace vectors and the product is (N + F) X[r] (no T gather / scatter).
efie_status dev_matvec_batch(Ctx *c, int R, const double2 *const *X, double2 *const *Y, bool superspace) {
  if (c->opt.precision != EFIE_MIXED_FP32 || R == 1 || (c->nI > kMultiMaxNI && !m2l_tc_supported(c))) {
    for (int r = 0; r < R; ++r) EFIE_TRY(superspace ? dev_matvec_super(c, X[r], Y[r]) : dev_matvec(c, X[r], Y[r]));
    return EFIE_OK;
  }
  EFIE_TRY(dev_batch_alloc(c, R));
  cudaStream_t st = c->stream;
  // phase events as in the single-vector product: 0 start, 1 gathered, 2 near done (second
  // stream), 3 moments folded, 4 M2L done, 5 local expansions evaluated, 6 end
  EFIE_CUDA(cudaEventRecord(c->tm.ev[0], st));
  const int nI = c->nI, q1 = c->q1, p1 = c->p1, m = c->m;
  const float h = (float)(1.0 / c->n);
  const size_t mstride = (size_t)c->ncl * 3 * nI;
  for (int r = 0; r < R; ++r) {
    double2 *xs = c->d_xsB + (size_t)r * c->nsup;
    if (superspace) {
      EFIE_CUDA(cudaMemcpyAsync(xs, X[r], sizeof(double2) * c->nsup, cudaMemcpyDeviceToDevice, st));
    } else {
      k_gather<<<(c->nsup + 255) / 256, 256, 0, st>>>(c->nsup, c->d_tg_ptr, c->d_tg_col, c->d_tg_val,
                                                      X[r], xs); ++c->launches;
    }
  }
  EFIE_CUDA(cudaEventRecord(c->tm.ev[1], st));
  EFIE_CUDA(cudaEventRecord(c->fork, st));
  EFIE_CUDA(cudaStreamWaitEvent(c->stream2, c->fork, 0));
  EFIE_TRY(dev_near_apply_batch(c, R, c->d_xsB, c->d_ysnB, (size_t)c->nsup, c->stream2));
  EFIE_CUDA(cudaEventRecord(c->tm.ev[2], c->stream2));
  EFIE_CUDA(cudaEventRecord(c->join, c->stream2));
  // leaf moments and M2M of all right-hand sides: grid dimension y = right-hand side
  k_leaf_moments<float><<<dim3(c->nE, R), 128, 0, st>>>(c->nE, c->lev_off[m], p1, q1, h, c->d_M, c->d_Md, c->d_xsB,
                                                        c->d_momB, (size_t)c->nsup, mstride); ++c->launches;
  for (int l = m - 1; l >= 0; --l) {
    int npar = c->np << (2 * l);
    k_m2m<float><<<dim3(npar, R), 128, m2m_smem(q1, sizeof(float2)), st>>>(npar, c->lev_off[l], c->lev_off[l + 1], q1,
                                                                           c->d_E, c->d_momB, mstride); ++c->launches;
  }
  const long long tot = (long long)c->ncl * nI;
  const unsigned gtot = (unsigned)((tot + 255) / 256);
  const int ld = 4 * c->batch_cap;
  k_fold_multi<<<gtot, 256, 0, st>>>(tot, nI, R, ld, mstride, c->d_nodeD, c->d_momB, c->d_srcB); ++c->launches;
  EFIE_CUDA(cudaEventRecord(c->tm.ev[3], st));
  const bool use_tc = c->opt.m2l_batch != 1 && m2l_tc_supported(c);
  if (c->n_m2l_targets > 0 && use_tc) {
    EFIE_TRY(launch_m2l_tc(c, st, 4 * R, ld, c->d_srcB, c->d_accB));
  } else if (c->n_m2l_targets > 0) {
    const int F = 4 * R, KM = (nI + 7) / 8;
    dim3 grid(c->n_m2l_targets, (F + kFB - 1) / kFB);
    const size_t sm = multi_smem(nI);
    const float kf = (float)c->kappa;
#define EFIE_MULTI(K)                                                                                        \
  k_m2l_f32_multi<K><<<grid, kMultiThreads, sm, st>>>(c->d_m2l_targets, c->d_far_ptr, c->d_far_src, c->d_pgeo, \
                                                     c->d_pph, nI, kf, c->m2l_mode, c->d_nodeX4, F, ld, c->d_srcB, \
                                                     c->d_accB);
    if (KM <= 1) { EFIE_MULTI(1) }
    else if (KM <= 2) { EFIE_MULTI(2) }
    else if (KM <= 4) { EFIE_MULTI(4) }
    else if (KM <= 8) { EFIE_MULTI(8) }
    else if (KM <= 12) { EFIE_MULTI(12) }
    else if (KM <= 16) { EFIE_MULTI(16) }
    else { EFIE_MULTI(18) }
#undef EFIE_MULTI
    ++c->launches;
  }
  EFIE_CUDA(cudaEventRecord(c->tm.ev[4], st));
  k_unfold_multi<<<gtot, 256, 0, st>>>(tot, nI, R, ld, mstride, (float)(1.0 / (c->kappa * c->kappa)), c->d_nodeD,
                                       c->d_accB, c->d_locB); ++c->launches;
  for (int l = 0; l < m; ++l) {
    int npar = c->np << (2 * l);
    k_l2l<float><<<dim3(npar, R), 128, l2l_smem(q1, sizeof(float2)), st>>>(npar, c->lev_off[l], c->lev_off[l + 1], q1,
                                                                           c->d_E, c->d_locB, mstride); ++c->launches;
  }
  k_leaf_eval<float><<<dim3(c->nE, R), 128, 0, st>>>(c->nE, c->lev_off[m], p1, q1, h, c->d_M, c->d_Md, c->d_locB,
                                                     c->d_ysB, mstride, (size_t)c->nsup); ++c->launches;
  EFIE_CUDA(cudaEventRecord(c->tm.ev[5], st));
  EFIE_CUDA(cudaStreamWaitEvent(st, c->join, 0));
  for (int r = 0; r < R; ++r) {
    if (superspace) {
      k_sum2<<<(c->nsup + 255) / 256, 256, 0, st>>>((size_t)c->nsup, c->d_ysB + (size_t)r * c->nsup,
                                                    c->d_ysnB + (size_t)r * c->nsup, Y[r]); ++c->launches;
    } else {
      k_scatter<<<(c->ndof + 255) / 256, 256, 0, st>>>(c->ndof, c->d_ts_ptr, c->d_ts_col, c->d_ts_val,
                                                       c->d_ysB + (size_t)r * c->nsup,
                                                       c->d_ysnB + (size_t)r * c->nsup, Y[r]); ++c->launches;
    }
  }
  EFIE_CUDA(cudaEventRecord(c->tm.ev[6], st));
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

}  // namespace efie
