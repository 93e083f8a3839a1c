// Near field (a2, a9): element-pair blocks of eq. Vkh for the non-admissible leaf pairs of
// Algorithm 1, computed on the device in FP64 with tensor Gauss rules for separated pairs
// and the Sauter-Schwab singularity-removing substitutions [SS97] for touching pairs
// (identical: 8 Duffy parts, common edge: 6, common vertex: 4), and their application
// y*_e = sum_{e'} N_{e e'} x*_{e'} as an HBM-streaming block-sparse product.
#include <algorithm>
#include <cmath>

#include "geom.cuh"
#include "tc.cuh"

namespace efie {

// s + e = a + b exactly (Knuth's two-sum): running FP32 sums with a compensation term
__device__ __forceinline__ void two_sum(float &hi, float &lo, float b) {
  const float s = hi + b, bp = s - hi;
  lo += (hi - (s - bp)) + (b - bp);
  hi = s;
}

constexpr int kQC = 64;          // quadrature points staged per chunk
constexpr int kQuadThreads = 2 * kQC;  // one thread per (point, side) in the geometry phase

struct QuadArgs {
  const PatchDesc *patches;
  const double *knots;
  const double4 *cpw;
  const NearPair *pairs;
  const int *todo;   // indices of the pairs computed here (the others are mirrored)
  const int *slot;   // pair index -> position of its block in the CSR order of the apply
  int ntodo;
  int n, p, gr, gs;
  const double *rx, *rw, *sx, *sw;  // Gauss rules on [0,1]
  double kappa, h;
  double2 *blocks;   // [nnear][nb col][nb row]
};

__device__ inline void sym_apply(int code, double u0, double u1, double &a, double &b) {
  a = (code & 1) ? u1 : u0;
  b = (code & 1) ? u0 : u1;
  if (code & 2) a = 1.0 - a;
  if (code & 4) b = 1.0 - b;
}

// Canonical coordinates (s_hat, t_hat) and weight of quadrature point k of a pair.
__device__ inline void canonical_point(int kind, int g, const double *x, const double *w, int k, double sh[2],
                                       double th[2], double &W) {
  int g2 = g * g, g4 = g2 * g2;
  int part = k / g4, rem = k - part * g4;
  int i0 = rem / (g2 * g), i1 = (rem / g2) % g, i2 = (rem / g) % g, i3 = rem % g;
  W = w[i0] * w[i1] * w[i2] * w[i3];
  double a = x[i0], b = x[i1], c = x[i2], d = x[i3];
  if (kind == 0) {
    sh[0] = a; sh[1] = b; th[0] = c; th[1] = d;
  } else if (kind == 3) {
    // identical: relative coordinates in one of 4 quadrants, split into 2 triangles
    int sgn0 = (part & 1) ? -1 : 1, sgn1 = (part & 2) ? -1 : 1;
    double z0 = (part >> 2) == 0 ? a : a * b;
    double z1 = (part >> 2) == 0 ? a * b : a;
    sh[0] = (sgn0 < 0 ? z0 : 0.0) + (1.0 - z0) * c;
    sh[1] = (sgn1 < 0 ? z1 : 0.0) + (1.0 - z1) * d;
    th[0] = sh[0] + sgn0 * z0;
    th[1] = sh[1] + sgn1 * z1;
    W *= a * (1.0 - z0) * (1.0 - z1);
  } else if (kind == 2) {
    // common edge {x2 = 0}: singular coordinates (|z1|, s2, t2), 3 pyramids x 2 signs
    int sgn = (part & 1) ? -1 : 1, pyr = part >> 1;
    double z, s2, t2;
    if (pyr == 0) { z = a; s2 = a * b; t2 = a * c; }
    else if (pyr == 1) { s2 = a; z = a * b; t2 = a * c; }
    else { t2 = a; z = a * b; s2 = a * c; }
    sh[0] = (sgn < 0 ? z : 0.0) + (1.0 - z) * d;
    th[0] = sh[0] + sgn * z;
    sh[1] = s2;
    th[1] = t2;
    W *= a * a * (1.0 - z);
  } else {
    // common vertex at the origin: 4 pyramids by the largest coordinate
    double v[4];
    double e[3] = {b, c, d};
    int t = 0;
    for (int q = 0; q < 4; ++q) v[q] = (q == part) ? a : a * e[t++];
    sh[0] = v[0]; sh[1] = v[1]; th[0] = v[2]; th[1] = v[3];
    W *= a * a * a;
  }
}

// Points staged per chunk: 64 for p <= 3, 32 for p = 4 (shared memory).
template <int P> struct QuadChunk { static constexpr int n = P <= 3 ? 64 : 32; };

// Shared memory of one block of k_near_quad<P> (doubles).
template <int P>
__host__ __device__ constexpr size_t quad_smem_doubles() {
  constexpr int Q = QuadChunk<P>::n, NS = (P + 1) * (P + 1), NB = 2 * NS;
  return (size_t)Q * (NS + 2 * NS)       // psi, d psi at the target points
         + (size_t)Q * (NS + 2 * NS)     // psi, d psi at the source points
         + (size_t)Q * 2 * NB * 2        // SA
         + (size_t)Q * NB * 2            // SC
         + (size_t)2 * Q * 10            // X, d1F, d2F (+ weight) of both sides
         + (size_t)Q * 10;               // cA[alpha][beta], cB
}

// One block per element pair.  The block entry of eq. Vkh for target row r = (alpha, a, b)
// and source column c = (beta, c1, c2) is, at a quadrature point with weight W and points
// s, t in the two elements (h = 1/n the element size, psi_ab = B_a B_b the Bernstein products,
// d_alpha psi their derivatives in the element coordinates, G = e^{i kappa |x-y|}/(4 pi |x-y|)):
//   W G [ h^4 <d_alpha F(s), d_beta F'(t)> psi_ab(s) psi'_c(t) - kappa^-2 h^2 d_alpha psi_ab(s) d_beta psi'_c(t) ].
// Per chunk of Q points: (1) one thread per (point, side) evaluates the NURBS map and the
// Bernstein values; (2) one thread per point forms the kernel value and the five complex
// coefficients cA_ab = W G h^4 <d_a F, d_b F'> and cB = -W G kappa^-2 h^2; (3) the products of
// the source-side values with the coefficients, SA[alpha][c] = cA_{alpha beta(c)} psi'_c and
// SC[c] = cB d_beta psi'_c; (4) every thread adds to its entries
//   B[r][c] += psi_ab SA[alpha][c] + d_alpha psi_ab SC[c]    (4 FP64 FMAs per entry and point).
// GD bounds the NURBS degrees at compile time.
template <int P, int GD>
__global__ void __launch_bounds__(kQuadThreads) k_near_quad(QuadArgs A) {
  constexpr int Q = QuadChunk<P>::n;
  constexpr int P1 = P + 1, NS = P1 * P1, NB = 2 * NS, NB2 = NB * NB;
  constexpr int EPT = (NB2 + kQuadThreads - 1) / kQuadThreads;
  extern __shared__ double sm[];
  double *Pt = sm;                    // [Q][NS]
  double *Dt = Pt + Q * NS;           // [Q][2][NS]
  double *Ps = Dt + Q * 2 * NS;       // [Q][NS]
  double *Ds = Ps + Q * NS;           // [Q][2][NS]
  double2 *SA = reinterpret_cast<double2 *>(Ds + Q * 2 * NS);  // [Q][2][NB]
  double2 *SC = SA + Q * 2 * NB;      // [Q][NB]
  double *Gm = reinterpret_cast<double *>(SC + Q * NB);  // [2][Q][10]: X, d1F, d2F, weight
  double *Cf = Gm + 2 * Q * 10;       // [Q][10]: cA_00, cA_01, cA_10, cA_11, cB (re, im)
  int pi = blockIdx.x;
  if (pi >= A.ntodo) return;
  const NearPair pr = A.pairs[A.todo[pi]];
  const int n = A.n, n2 = n * n;
  const int g = pr.kind == 0 ? A.gr : A.gs;
  const double *gx = pr.kind == 0 ? A.rx : A.sx;
  const double *gw = pr.kind == 0 ? A.rw : A.sw;
  const int parts = pr.kind == 0 ? 1 : (pr.kind == 3 ? 8 : (pr.kind == 2 ? 6 : 4));
  const int nq = parts * g * g * g * g;
  const double h = A.h, h2 = h * h, h4 = h2 * h2, ik2 = 1.0 / (A.kappa * A.kappa);

  // element placement
  int ej = pr.e / n2, eK = pr.e % n2, fj = pr.e2 / n2, fK = pr.e2 % n2;
  int ea = 0, eb = 0, fa = 0, fb = 0;
  for (int bt = 0; bt < 15; ++bt) {
    ea |= ((eK >> (2 * bt)) & 1) << bt;
    eb |= ((eK >> (2 * bt + 1)) & 1) << bt;
    fa |= ((fK >> (2 * bt)) & 1) << bt;
    fb |= ((fK >> (2 * bt + 1)) & 1) << bt;
  }

  double2 acc[EPT];
#pragma unroll
  for (int t = 0; t < EPT; ++t) acc[t] = make_double2(0.0, 0.0);
  const int tid = threadIdx.x;

  for (int q0 = 0; q0 < nq; q0 += Q) {
    // (1) geometry and Bernstein values, one thread per (point, side)
    for (int it = tid; it < 2 * Q; it += kQuadThreads) {
      const int side = it / Q, ql = it % Q, k = q0 + ql;
      double *G = Gm + (side * Q + ql) * 10;
      double *Pv = (side == 0 ? Pt : Ps) + ql * NS, *Dv = (side == 0 ? Dt : Ds) + ql * 2 * NS;
      if (k < nq) {
        double sh[2], th[2], W;
        canonical_point(pr.kind, g, gx, gw, k, sh, th, W);
        double sg0, sg1;
        const int code = side == 0 ? pr.r1 : pr.r2;
        sym_apply(code, side == 0 ? sh[0] : th[0], side == 0 ? sh[1] : th[1], sg0, sg1);
        const int pj = side == 0 ? ej : fj;
        const int ia = side == 0 ? ea : fa, ib = side == 0 ? eb : fb;
        double X[3], D1[3], D2[3];
        dev_patch_eval<GD>(A.patches[pj], A.knots, A.cpw, (ia + sg0) * h, (ib + sg1) * h, X, D1, D2);
        double B0[kMaxP1], dB0[kMaxP1], B1[kMaxP1], dB1[kMaxP1];
        dev_bernstein(P, sg0, B0, dB0);
        dev_bernstein(P, sg1, B1, dB1);
#pragma unroll
        for (int b = 0; b < P1; ++b)
#pragma unroll
          for (int a = 0; a < P1; ++a) {
            Pv[b * P1 + a] = B0[a] * B1[b];
            Dv[b * P1 + a] = dB0[a] * B1[b];
            Dv[NS + b * P1 + a] = B0[a] * dB1[b];
          }
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
          G[kk] = X[kk];
          G[3 + kk] = D1[kk];
          G[6 + kk] = D2[kk];
        }
        G[9] = W;
      } else {
        for (int r = 0; r < NS; ++r) {
          Pv[r] = 0.0;
          Dv[r] = 0.0;
          Dv[NS + r] = 0.0;
        }
        for (int kk = 0; kk < 9; ++kk) G[kk] = 0.0;
        G[2] = (double)side;  // dummy pair at distance 1; weight 0
        G[9] = 0.0;
      }
    }
    __syncthreads();
    // (2) kernel value and coefficients, one thread per point
    for (int ql = tid; ql < Q; ql += kQuadThreads) {
      const double *Gs = Gm + ql * 10, *Gt = Gm + (Q + ql) * 10;
      const double dx = Gs[0] - Gt[0], dy = Gs[1] - Gt[1], dz = Gs[2] - Gt[2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      double sn, cs;
      sincos(A.kappa * r, &sn, &cs);
      const double f = Gs[9] / (4.0 * M_PI * r);
      const double gre = f * cs, gim = f * sn;
      double *C = Cf + ql * 10;
#pragma unroll
      for (int al = 0; al < 2; ++al)
#pragma unroll
        for (int be = 0; be < 2; ++be) {
          const double *Da = Gs + 3 + 3 * al, *Db = Gt + 3 + 3 * be;
          const double gg = h4 * (Da[0] * Db[0] + Da[1] * Db[1] + Da[2] * Db[2]);
          C[2 * (2 * al + be)] = gre * gg;
          C[2 * (2 * al + be) + 1] = gim * gg;
        }
      C[8] = -ik2 * h2 * gre;
      C[9] = -ik2 * h2 * gim;
    }
    __syncthreads();
    // (3) source-side products SA, SC
    for (int it = tid; it < Q * NB; it += kQuadThreads) {
      const int ql = it / NB, cc = it % NB, be = cc / NS, cd = cc % NS;
      const double *C = Cf + ql * 10;
      const double ps = Ps[ql * NS + cd], ds = Ds[ql * 2 * NS + be * NS + cd];
#pragma unroll
      for (int al = 0; al < 2; ++al)
        SA[(ql * 2 + al) * NB + cc] = make_double2(C[2 * (2 * al + be)] * ps, C[2 * (2 * al + be) + 1] * ps);
      SC[ql * NB + cc] = make_double2(C[8] * ds, C[9] * ds);
    }
    __syncthreads();
    // (4) accumulation of this thread's entries (column-major index cc NB + rr)
#pragma unroll
    for (int t = 0; t < EPT; ++t) {
      const int idx = tid + t * kQuadThreads;
      if (idx < NB2) {
        const int cc = idx / NB, rr = idx % NB, al = rr / NS, ab = rr % NS;
        double re = 0.0, im = 0.0;
#pragma unroll 4
        for (int ql = 0; ql < Q; ++ql) {
          const double pt = Pt[ql * NS + ab], dt = Dt[ql * 2 * NS + al * NS + ab];
          const double2 sa = SA[(ql * 2 + al) * NB + cc], sc = SC[ql * NB + cc];
          re = fma(pt, sa.x, fma(dt, sc.x, re));
          im = fma(pt, sa.y, fma(dt, sc.y, im));
        }
        acc[t].x += re;
        acc[t].y += im;
      }
    }
    __syncthreads();
  }
  double2 *out = A.blocks + (size_t)A.slot[A.todo[pi]] * NB2;
#pragma unroll
  for (int t = 0; t < EPT; ++t) {
    int idx = threadIdx.x + t * kQuadThreads;
    if (idx < NB2) out[idx] = acc[t];
  }
}

// ------------------------------------------------------------------ separated pairs
// A separated pair (no common point) is integrated with the tensor Gauss rule of g points per
// direction on each element, so every point of the rule on an element is the same for all of
// that element's separated pairs.  Element tables hold, per element and Gauss point
// p = i0 g + i1 (s1 = x_i0, s2 = x_i1): F, d1F, d2F and the weight w_i0 w_i1.
__global__ void k_elem_table(const PatchDesc *patches, const double *knots, const double4 *cpw, int n, int nE, int g,
                             const double *gx, const double *gw, double *tab) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int G2 = g * g;
  if (t >= (long long)nE * G2) return;
  const int e = (int)(t / G2), p = (int)(t % G2), i0 = p / g, i1 = p % g;
  const int n2 = n * n, j = e / n2, K = e % n2;
  int ia = 0, ib = 0;
  for (int b = 0; b < 15; ++b) {
    ia |= ((K >> (2 * b)) & 1) << b;
    ib |= ((K >> (2 * b + 1)) & 1) << b;
  }
  const double h = 1.0 / n;
  double X[3], D1[3], D2[3];
  dev_patch_eval(patches[j], knots, cpw, (ia + gx[i0]) * h, (ib + gx[i1]) * h, X, D1, D2);
  double *o = tab + (size_t)t * 10;
  for (int k = 0; k < 3; ++k) {
    o[k] = X[k];
    o[3 + k] = D1[k];
    o[6 + k] = D2[k];
  }
  o[9] = gw[i0] * gw[i1];
}

constexpr int kSepMaxG = 8;  // largest rule of the separated-pair kernel (shared memory)

struct SepArgs {
  const NearPair *pairs;
  const int *list;  // pairs integrated here
  const int *slot;
  int nlist, g;
  const double *tab;  // element tables [nE][g^2][10]
  const double *gx;   // Gauss points on [0, 1]
  double kappa, h;
  double2 *blocks;
};

// Shared memory (bytes) of k_near_sep<P> for a rule of g points.
template <int P>
__host__ __device__ constexpr size_t sep_smem(int g) {
  return (size_t)g * g * g * g * 16 + (size_t)g * g * (P + 1) * (P + 1) * (8 + 16 + 16) + (size_t)2 * g * g * 10 * 8 +
         (size_t)2 * g * (P + 1) * 8;
}

// Separated pair (e, e'), rule of g points per direction: with the weighted kernel matrix
// Km[i][j] = W_i W_j e^{i kappa r_ij} / (4 pi r_ij) between the Gauss points of the two elements,
// the block entry of eq. Vkh is
//   B[(alpha, ab)][(beta, cd)] = sum_{k = 0..3} sum_i T_{alpha k}[i][ab] (Km S_{beta k})[i][cd],
//   T_{alpha k} = h^2 d_alpha F_k psi_ab (k < 3), h d_alpha psi_ab (k = 3)   (target points),
//   S_{beta k}  = h^2 d_beta F'_k psi'_cd (k < 3), -kappa^-2 h d_beta psi'_cd (k = 3)   (source).
// The sum over the source points is done once per (beta, k) for all target points (a g^2 x g^2
// by g^2 x (p+1)^2 complex-by-real product), which costs g^2 (p+1)^2 of the g^4 (2 (p+1)^2)^2
// per-point products of the direct form.
template <int P>
__global__ void __launch_bounds__(128) k_near_sep(SepArgs A) {
  constexpr int P1 = P + 1, NS = P1 * P1, NB = 2 * NS, NB2 = NB * NB;
  constexpr int EPT = (NB2 + 127) / 128;
  const int g = A.g, G2 = g * g;
  extern __shared__ double sm[];
  double2 *Km = reinterpret_cast<double2 *>(sm);  // [G2][G2]
  double2 *KS = Km + G2 * G2;                     // [G2][NS]
  double *S = reinterpret_cast<double *>(KS + G2 * NS);  // [G2][NS]
  double *T = S + G2 * NS;                        // [2 alpha][G2][NS]
  double *Et = T + 2 * G2 * NS;                   // [G2][10]
  double *Es = Et + G2 * 10;                      // [G2][10]
  double *Bx = Es + G2 * 10;                      // [g][P1] Bernstein values at the Gauss points
  double *dBx = Bx + g * P1;                      // [g][P1] derivatives
  const int pi = blockIdx.x;
  if (pi >= A.nlist) return;
  const int k = A.list[pi];
  const NearPair pr = A.pairs[k];
  const int tid = threadIdx.x;
  for (int i = tid; i < G2 * 10; i += 128) {
    Et[i] = A.tab[(size_t)pr.e * G2 * 10 + i];
    Es[i] = A.tab[(size_t)pr.e2 * G2 * 10 + i];
  }
  for (int i = tid; i < g; i += 128) {
    double B[kMaxP1], dB[kMaxP1];
    dev_bernstein(P, A.gx[i], B, dB);
    for (int a = 0; a < P1; ++a) {
      Bx[i * P1 + a] = B[a];
      dBx[i * P1 + a] = dB[a];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < G2 * G2; idx += 128) {
    const int i = idx / G2, j = idx % G2;
    const double *xt = Et + i * 10, *xs = Es + j * 10;
    const double dx = xt[0] - xs[0], dy = xt[1] - xs[1], dz = xt[2] - xs[2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    double sn, cs;
    sincos(A.kappa * r, &sn, &cs);
    const double f = xt[9] * xs[9] / (4.0 * M_PI * r);
    Km[idx] = make_double2(f * cs, f * sn);
  }
  const double h = A.h, h2 = h * h, ik2 = 1.0 / (A.kappa * A.kappa);
  double2 acc[EPT];
#pragma unroll
  for (int t = 0; t < EPT; ++t) acc[t] = make_double2(0.0, 0.0);
  for (int be = 0; be < 2; ++be) {
    for (int kk = 0; kk < 4; ++kk) {
      __syncthreads();
      // S_{beta k} at the source points, T_{alpha k} (alpha = 0, 1) at the target points
      for (int idx = tid; idx < G2 * NS; idx += 128) {
        const int pt = idx / NS, cd = idx % NS, c0 = cd % P1, c1 = cd / P1, i0 = pt / g, i1 = pt % g;
        const double psi = Bx[i0 * P1 + c0] * Bx[i1 * P1 + c1];
        const double dps[2] = {dBx[i0 * P1 + c0] * Bx[i1 * P1 + c1], Bx[i0 * P1 + c0] * dBx[i1 * P1 + c1]};
        const double *xs = Es + pt * 10, *xt = Et + pt * 10;
        S[idx] = kk < 3 ? h2 * xs[3 + 3 * be + kk] * psi : -ik2 * h * dps[be];
        T[idx] = kk < 3 ? h2 * xt[3 + kk] * psi : h * dps[0];
        T[G2 * NS + idx] = kk < 3 ? h2 * xt[6 + kk] * psi : h * dps[1];
      }
      __syncthreads();
      for (int idx = tid; idx < G2 * NS; idx += 128) {
        const int i = idx / NS, cd = idx % NS;
        double re = 0.0, im = 0.0;
        for (int j = 0; j < G2; ++j) {
          const double2 kv = Km[i * G2 + j];
          const double sv = S[j * NS + cd];
          re = fma(kv.x, sv, re);
          im = fma(kv.y, sv, im);
        }
        KS[idx] = make_double2(re, im);
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < EPT; ++t) {
        const int idx = tid + t * 128;
        if (idx < NB2) {
          const int cc = idx / NB, rr = idx % NB;
          if (cc / NS == be) {
            const int al = rr / NS, ab = rr % NS, cd = cc % NS;
            const double *Ta = T + al * G2 * NS;
            double re = 0.0, im = 0.0;
            for (int i = 0; i < G2; ++i) {
              const double tv = Ta[i * NS + ab];
              const double2 kv = KS[i * NS + cd];
              re = fma(tv, kv.x, re);
              im = fma(tv, kv.y, im);
            }
            acc[t].x += re;
            acc[t].y += im;
          }
        }
      }
    }
  }
  double2 *out = A.blocks + (size_t)A.slot[k] * NB2;
#pragma unroll
  for (int t = 0; t < EPT; ++t) {
    const int idx = tid + t * 128;
    if (idx < NB2) out[idx] = acc[t];
  }
}

// B(e2, e) = B(e, e2)^T for the pairs that were not integrated directly.
__global__ void k_near_mirror(int nb, const int *todo_m, const int *src_of, const int *slot, int nm,
                              double2 *blocks) {
  int nb2 = nb * nb;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nm * nb2) return;
  int k = (int)(t / nb2), idx = (int)(t % nb2);
  int cc = idx / nb, rr = idx % nb;
  int dst = slot[todo_m[k]], src = slot[src_of[k]];
  blocks[(size_t)dst * nb2 + cc * nb + rr] = blocks[(size_t)src * nb2 + rr * nb + cc];
}

efie_status dev_near_quadrature(Ctx *c, const std::vector<NearPair> &pairs, const std::vector<int> &mirror) {
  if (c->nnear == 0) return EFIE_OK;
  const int nb = c->nb;
  // pairs integrated here (the others are mirrored): touching pairs by the Duffy kernel,
  // separated pairs by the element-table kernel when its rule fits in shared memory
  const bool sep_fast = c->gr <= kSepMaxG;
  std::vector<int> todo, todo_sep, todo_m, src_of;
  for (int k = 0; k < c->nnear; ++k) {
    if (pairs[k].e <= pairs[k].e2) {
      if (sep_fast && pairs[k].kind == 0) todo_sep.push_back(k);
      else todo.push_back(k);
    } else {
      todo_m.push_back(k);
      src_of.push_back(mirror[k]);
    }
  }
  NearPair *d_pairs = nullptr;
  int *d_todo = nullptr, *d_todo_m = nullptr, *d_src_of = nullptr, *d_slot = nullptr, *d_sep = nullptr;
  double *d_tab = nullptr;
  std::vector<int> slot(c->nnear);
  for (int at = 0; at < c->nnear; ++at) slot[c->near_perm[at]] = at;
  double *d_rule = nullptr;
  EFIE_TRY(dalloc(c, &d_pairs, pairs.size()));
  EFIE_TRY(dalloc(c, &d_todo, todo.size()));
  EFIE_TRY(dalloc(c, &d_sep, todo_sep.size()));
  EFIE_TRY(dalloc(c, &d_todo_m, todo_m.size()));
  EFIE_TRY(dalloc(c, &d_src_of, src_of.size()));
  EFIE_TRY(dalloc(c, &d_rule, 2 * (size_t)(c->gr + c->gs)));
  EFIE_TRY(dalloc(c, &d_slot, slot.size()));
  cudaStream_t s0 = c->stream;
  EFIE_CUDA(cudaMemcpyAsync(d_slot, slot.data(), 4 * slot.size(), cudaMemcpyHostToDevice, s0));
  EFIE_CUDA(cudaMemcpyAsync(d_pairs, pairs.data(), sizeof(NearPair) * pairs.size(), cudaMemcpyHostToDevice, s0));
  if (!todo.empty()) EFIE_CUDA(cudaMemcpyAsync(d_todo, todo.data(), 4 * todo.size(), cudaMemcpyHostToDevice, s0));
  if (!todo_sep.empty())
    EFIE_CUDA(cudaMemcpyAsync(d_sep, todo_sep.data(), 4 * todo_sep.size(), cudaMemcpyHostToDevice, s0));
  if (!todo_m.empty()) {
    EFIE_CUDA(cudaMemcpyAsync(d_todo_m, todo_m.data(), 4 * todo_m.size(), cudaMemcpyHostToDevice, s0));
    EFIE_CUDA(cudaMemcpyAsync(d_src_of, src_of.data(), 4 * src_of.size(), cudaMemcpyHostToDevice, s0));
  }
  std::vector<double> rule;
  rule.insert(rule.end(), c->tab.gx.begin(), c->tab.gx.end());
  rule.insert(rule.end(), c->tab.gw.begin(), c->tab.gw.end());
  rule.insert(rule.end(), c->tab.sx.begin(), c->tab.sx.end());
  rule.insert(rule.end(), c->tab.sw.begin(), c->tab.sw.end());
  EFIE_CUDA(cudaMemcpyAsync(d_rule, rule.data(), 8 * rule.size(), cudaMemcpyHostToDevice, s0));
  EFIE_TRY(dalloc(c, &c->d_nblk, (size_t)c->nnear * nb * nb));

  QuadArgs A;
  A.patches = c->d_patches;
  A.knots = c->d_knots;
  A.cpw = c->d_cpw;
  A.pairs = d_pairs;
  A.todo = d_todo;
  A.slot = d_slot;
  A.ntodo = (int)todo.size();
  A.n = c->n;
  A.p = c->p;
  A.gr = c->gr;
  A.gs = c->gs;
  A.rx = d_rule;
  A.rw = d_rule + c->gr;
  A.sx = d_rule + 2 * c->gr;
  A.sw = d_rule + 2 * c->gr + c->gs;
  A.kappa = c->kappa;
  A.h = 1.0 / c->n;
  A.blocks = c->d_nblk;
  c->near_quad_pairs = (int)todo.size();
  c->near_sep_pairs = (int)todo_sep.size();
  c->near_quad_points = 0;
  for (int k : todo) {
    const int kind = pairs[k].kind, g = kind == 0 ? c->gr : c->gs;
    const int parts = kind == 0 ? 1 : (kind == 3 ? 8 : (kind == 2 ? 6 : 4));
    c->near_quad_points += (long long)parts * g * g * g * g;
  }
  // compile-time bound of the NURBS degrees of this geometry
  int gdeg = 1;
  for (const PatchDesc &pd : c->patches) gdeg = std::max(gdeg, std::max(pd.deg[0], pd.deg[1]));
  const int GDsel = gdeg <= 2 ? 2 : (gdeg <= 4 ? 4 : 8);
  EFIE_CUDA(cudaEventRecord(c->tm.ev[7], c->stream));
  bool launched = A.ntodo == 0;
#define EFIE_QUAD(PP, GG)                                                                                 \
  if (!launched && c->p == PP && GDsel == GG) {                                                           \
    const size_t smem = sizeof(double) * quad_smem_doubles<PP>();                                         \
    EFIE_CUDA(cudaFuncSetAttribute(k_near_quad<PP, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                   (int)smem));                                                          \
    k_near_quad<PP, GG><<<A.ntodo, kQuadThreads, smem, c->stream>>>(A);                                   \
    ++c->launches;                                                                                        \
    launched = true;                                                                                      \
  }
  EFIE_QUAD(1, 2) EFIE_QUAD(1, 4) EFIE_QUAD(1, 8)
  EFIE_QUAD(2, 2) EFIE_QUAD(2, 4) EFIE_QUAD(2, 8)
  EFIE_QUAD(3, 2) EFIE_QUAD(3, 4) EFIE_QUAD(3, 8)
  EFIE_QUAD(4, 2) EFIE_QUAD(4, 4) EFIE_QUAD(4, 8)
#undef EFIE_QUAD
  if (!launched) {
    c->err = "device near-field quadrature supports 1 <= p <= 4";
    return EFIE_EINVAL;
  }
  EFIE_CUDA(cudaGetLastError());
  EFIE_CUDA(cudaEventRecord(c->tm.ev[6], c->stream));
  c->near_sep_ms = 0.f;
  if (!todo_sep.empty()) {
    // element tables at the g_reg x g_reg Gauss points, then one block per separated pair
    const int g = c->gr;
    EFIE_TRY(dalloc(c, &d_tab, (size_t)c->nE * g * g * 10));
    const long long tot = (long long)c->nE * g * g;
    k_elem_table<<<(unsigned)((tot + 127) / 128), 128, 0, s0>>>(c->d_patches, c->d_knots, c->d_cpw, c->n, c->nE, g,
                                                              d_rule, d_rule + g, d_tab); ++c->launches;
    SepArgs S;
    S.pairs = d_pairs;
    S.list = d_sep;
    S.slot = d_slot;
    S.nlist = (int)todo_sep.size();
    S.g = g;
    S.tab = d_tab;
    S.gx = d_rule;
    S.kappa = c->kappa;
    S.h = 1.0 / c->n;
    S.blocks = c->d_nblk;
    switch (c->p) {
#define EFIE_SEP(PP)                                                                                   \
  case PP: {                                                                                           \
    const size_t smem = sep_smem<PP>(g);                                                               \
    EFIE_CUDA(cudaFuncSetAttribute(k_near_sep<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_near_sep<PP><<<S.nlist, 128, smem, s0>>>(S);                                                     \
    ++c->launches;                                                                                     \
    break;                                                                                             \
  }
      EFIE_SEP(1)
      EFIE_SEP(2)
      EFIE_SEP(3)
      EFIE_SEP(4)
#undef EFIE_SEP
      default:
        c->err = "device near-field quadrature supports 1 <= p <= 4";
        return EFIE_EINVAL;
    }
    EFIE_CUDA(cudaGetLastError());
  }
  EFIE_CUDA(cudaEventRecord(c->tm.ev[5], c->stream));
  if (!todo_m.empty()) {
    long long tot = (long long)todo_m.size() * nb * nb;
    k_near_mirror<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(nb, d_todo_m, d_src_of, d_slot,
                                                                       (int)todo_m.size(), c->d_nblk); ++c->launches;
    EFIE_CUDA(cudaGetLastError());
  }
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  cudaEventElapsedTime(&c->near_quad_ms, c->tm.ev[7], c->tm.ev[6]);
  if (!todo_sep.empty()) cudaEventElapsedTime(&c->near_sep_ms, c->tm.ev[6], c->tm.ev[5]);
  dfree(c, d_pairs);
  dfree(c, d_todo);
  dfree(c, d_todo_m);
  dfree(c, d_src_of);
  dfree(c, d_rule);
  dfree(c, d_slot);
  dfree(c, d_sep);
  dfree(c, d_tab);
  return EFIE_OK;
}

// y*_e = sum over near sources e' of N_{e e'} x*_{e'} (a9).  One block of 4 warps per target
// element; the element's source blocks are dealt round-robin to lane groups of GS lanes
// (GS = 8, 16 or 32 >= nb rows, 32/GS groups per warp); lane r of a group owns rows r and
// r + 32.  Blocks are column-major, so a group reads each column as one contiguous run.
// The partial rows of the groups and warps are summed in shared memory in a fixed order.
template <class T> struct CT;
template <> struct CT<double> { using V = double2; };
template <> struct CT<float> { using V = float2; };

constexpr int kApplyWarps = 4;

template <class T, int NB>
__global__ void __launch_bounds__(32 * kApplyWarps) k_near_apply(int nE, const int *__restrict__ ptr,
                                                                 const int *__restrict__ src,
                                                                 const typename CT<T>::V *__restrict__ blocks,
                                                                 const double2 *__restrict__ xs,
                                                                 double2 *__restrict__ ysn) {
  using V = typename CT<T>::V;
  constexpr int GS = NB <= 8 ? 8 : (NB <= 16 ? 16 : 32);
  constexpr int NG = 32 / GS;                 // groups per warp
  constexpr int RPL = (NB + GS - 1) / GS;     // rows per lane
  constexpr int XPL = (NB + GS - 1) / GS;     // x entries per lane
  __shared__ T red[kApplyWarps * NG][NB][2];
  const int e = blockIdx.x;
  if (e >= nE) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / GS, r0 = lane % GS;
  const int gid = warp * NG + g, ngroups = kApplyWarps * NG;
  T ar[RPL], ai[RPL], cr[RPL], ci[RPL];  // running sums and (FP32) compensation terms
#pragma unroll
  for (int t = 0; t < RPL; ++t) ar[t] = ai[t] = cr[t] = ci[t] = T(0);
  const int k0 = ptr[e], k1 = ptr[e + 1];
  // every group walks the same number of iterations so that the shuffles stay uniform
  for (int kb = k0; kb < k1; kb += ngroups) {
    const int k = kb + gid;
    const bool act = k < k1;
    const V *B = blocks + (size_t)(act ? k : k0) * NB * NB;
    const double2 *x = xs + (size_t)src[act ? k : k0] * NB;
    T xr[XPL], xi[XPL];
#pragma unroll
    for (int t = 0; t < XPL; ++t) {
      int cidx = r0 + GS * t;
      double2 v = (act && cidx < NB) ? x[cidx] : make_double2(0.0, 0.0);
      xr[t] = (T)v.x;
      xi[t] = (T)v.y;
    }
    T pr[RPL], pim[RPL];  // this source block's contribution
#pragma unroll
    for (int t = 0; t < RPL; ++t) pr[t] = pim[t] = T(0);
#pragma unroll
    for (int tc = 0; tc < XPL; ++tc) {
      const int ncol = (NB - GS * tc) < GS ? (NB - GS * tc) : GS;
#pragma unroll 6
      for (int c0 = 0; c0 < ncol; ++c0) {
        const int cc = GS * tc + c0;
        T vr = __shfl_sync(0xffffffffu, xr[tc], g * GS + c0);
        T vi = __shfl_sync(0xffffffffu, xi[tc], g * GS + c0);
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          int rr = r0 + GS * t;
          if (act && rr < NB) {
            V b = B[cc * NB + rr];
            pr[t] += b.x * vr - b.y * vi;
            pim[t] += b.x * vi + b.y * vr;
          }
        }
      }
    }
    // per-source partial sums enter the running sums with two-sum compensation (FP32)
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      T sr = ar[t] + pr[t], si = ai[t] + pim[t];
      if (sizeof(T) == 4) {
        T br = sr - ar[t], bi = si - ai[t];
        cr[t] += (ar[t] - (sr - br)) + (pr[t] - br);
        ci[t] += (ai[t] - (si - bi)) + (pim[t] - bi);
      }
      ar[t] = sr;
      ai[t] = si;
    }
  }
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    int rr = r0 + GS * t;
    if (rr < NB) {
      red[gid][rr][0] = ar[t] + cr[t];
      red[gid][rr][1] = ai[t] + ci[t];
    }
  }
  __syncthreads();
  for (int rr = threadIdx.x; rr < NB; rr += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int q = 0; q < ngroups; ++q) {
      sr += (double)red[q][rr][0];
      si += (double)red[q][rr][1];
    }
    ysn[(size_t)e * NB + rr] = make_double2(sr, si);
  }
}

// x* in FP32 for the FP32 block product (converted once per product, not once per lane)
__global__ void k_vec_to_f32(int n, const double2 *__restrict__ x, float2 *__restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

// FP32 blocks, one right-hand side, streamed with 16-byte loads.  A block column of NB rows is
// read by LPC = NB / 2 lanes, each loading two consecutive rows (one float4), so a warp
// instruction reads CPR = 32 / LPC consecutive columns (contiguous in the column-major block) and
// a block takes NB / CPR rounds.  Lane l keeps the rows 2 (l % LPC), 2 (l % LPC) + 1 and the
// columns l / LPC + CPR k; its x* entries (FP32 copy) come through the cache.
template <int NB>
__device__ __forceinline__ void near_block16(const float4 *__restrict__ B, const float2 *__restrict__ x, int rp,
                                              int cg, bool act, float4 *b, float2 *xv) {
  constexpr int LPC = NB / 2, CPR = 32 / LPC, ROUNDS = (NB + CPR - 1) / CPR;
#pragma unroll
  for (int t = 0; t < ROUNDS; ++t) {
    const int col = cg + CPR * t;
    const bool ok = act && col < NB;
    b[t] = ok ? __ldcs(B + col * LPC + rp) : make_float4(0.f, 0.f, 0.f, 0.f);
    xv[t] = ok ? x[col] : make_float2(0.f, 0.f);
  }
}

// One warp per target element (a contiguous range of elements per warp, the same count for
// every warp): the warp reads the element's source blocks BIF at a time (their loads in flight
// together), adds each block's FP32 partial sums to running sums by two-sum (compensated), and
// combines its column groups with shuffles in a fixed order (FP64 sum).  No shared memory and no block barrier, so a
// warp goes on to its next element as soon as it has written the last.
template <int NB, int BIF>
__global__ void __launch_bounds__(128) k_near_apply_w(int nE, int per, const int *__restrict__ ptr,
                                                      const int *__restrict__ src, const float4 *__restrict__ blocks,
                                                      const float2 *__restrict__ xs, double2 *__restrict__ ysn) {
  constexpr int LPC = NB / 2, CPR = 32 / LPC, ROUNDS = (NB + CPR - 1) / CPR;
  constexpr int F4 = NB * NB / 2;
  const int lane = threadIdx.x & 31;
  const int rp = lane % LPC, cg = lane / LPC;
  const bool act = cg < CPR;
  const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int e0 = wid * per, e1 = min(e0 + per, nE);
  for (int e = e0; e < e1; ++e) {
    float h[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
    const int k0 = ptr[e], k1 = ptr[e + 1];
    for (int k = k0; k < k1; k += BIF) {
      float4 b[BIF][ROUNDS];
      float2 xv[BIF][ROUNDS];
#pragma unroll
      for (int i = 0; i < BIF; ++i) {
        const bool have = k + i < k1;
        const int kk = have ? k + i : k;
        near_block16<NB>(blocks + (size_t)kk * F4, xs + (size_t)src[kk] * NB, rp, cg, act && have, b[i], xv[i]);
      }
#pragma unroll
      for (int i = 0; i < BIF; ++i) {
        float p[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < ROUNDS; ++t) {
          p[0] = fmaf(b[i][t].x, xv[i][t].x, fmaf(-b[i][t].y, xv[i][t].y, p[0]));
          p[1] = fmaf(b[i][t].x, xv[i][t].y, fmaf(b[i][t].y, xv[i][t].x, p[1]));
          p[2] = fmaf(b[i][t].z, xv[i][t].x, fmaf(-b[i][t].w, xv[i][t].y, p[2]));
          p[3] = fmaf(b[i][t].z, xv[i][t].y, fmaf(b[i][t].w, xv[i][t].x, p[3]));
        }
        if (k + i < k1)
#pragma unroll
          for (int q = 0; q < 4; ++q) two_sum(h[q], cmp[q], p[q]);
      }
    }
    double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int g = 0; g < CPR; ++g)
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] += (double)__shfl_sync(0xffffffffu, h[q] + cmp[q], g * LPC + rp);
    if (lane < LPC) {
      ysn[(size_t)e * NB + 2 * lane] = make_double2(s[0], s[1]);
      ysn[(size_t)e * NB + 2 * lane + 1] = make_double2(s[2], s[3]);
    }
  }
}

// The same product for several right-hand sides (FP32 blocks, mixed form): each block is read
// once for a group of up to RB right-hand sides (grid dimension y), which divides the HBM
// traffic of the near field by RB.  Vectors of right-hand side r start at r * vstride.
template <int NB, int RB>
__global__ void __launch_bounds__(32 * kApplyWarps) k_near_apply_multi(int nE, int R, size_t vstride,
                                                                       const int *__restrict__ ptr,
                                                                       const int *__restrict__ src,
                                                                       const float2 *__restrict__ blocks,
                                                                       const double2 *__restrict__ xs,
                                                                       double2 *__restrict__ ysn) {
  constexpr int GS = NB <= 8 ? 8 : (NB <= 16 ? 16 : 32);
  constexpr int NG = 32 / GS;
  constexpr int RPL = (NB + GS - 1) / GS;
  constexpr int XPL = (NB + GS - 1) / GS;
  __shared__ float red[kApplyWarps * NG][NB][RB][2];
  const int e = blockIdx.x;
  if (e >= nE) return;
  const int r0 = blockIdx.y * RB, nr = min(RB, R - r0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / GS, rl = lane % GS;
  const int gid = warp * NG + g, ngroups = kApplyWarps * NG;
  float ar[RPL][RB], ai[RPL][RB], cr[RPL][RB], ci[RPL][RB];
#pragma unroll
  for (int t = 0; t < RPL; ++t)
#pragma unroll
    for (int j = 0; j < RB; ++j) ar[t][j] = ai[t][j] = cr[t][j] = ci[t][j] = 0.f;
  const int k0 = ptr[e], k1 = ptr[e + 1];
  for (int kb = k0; kb < k1; kb += ngroups) {
    const int k = kb + gid;
    const bool act = k < k1;
    const float2 *B = blocks + (size_t)(act ? k : k0) * NB * NB;
    const size_t xo = (size_t)src[act ? k : k0] * NB;
    float xr[RB][XPL], xi[RB][XPL];
#pragma unroll
    for (int j = 0; j < RB; ++j)
#pragma unroll
      for (int t = 0; t < XPL; ++t) {
        const int cidx = rl + GS * t;
        double2 v = (act && cidx < NB && j < nr) ? xs[(size_t)(r0 + j) * vstride + xo + cidx] : make_double2(0.0, 0.0);
        xr[j][t] = (float)v.x;
        xi[j][t] = (float)v.y;
      }
    float pr[RPL][RB], pim[RPL][RB];
#pragma unroll
    for (int t = 0; t < RPL; ++t)
#pragma unroll
      for (int j = 0; j < RB; ++j) pr[t][j] = pim[t][j] = 0.f;
#pragma unroll
    for (int tc = 0; tc < XPL; ++tc) {
      const int ncol = (NB - GS * tc) < GS ? (NB - GS * tc) : GS;
#pragma unroll 2
      for (int c0 = 0; c0 < ncol; ++c0) {
        const int cc = GS * tc + c0;
        float2 b[RPL];
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
          const int rr = rl + GS * t;
          b[t] = (act && rr < NB) ? B[cc * NB + rr] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < RB; ++j) {
          const float vr = __shfl_sync(0xffffffffu, xr[j][tc], g * GS + c0);
          const float vi = __shfl_sync(0xffffffffu, xi[j][tc], g * GS + c0);
#pragma unroll
          for (int t = 0; t < RPL; ++t) {
            pr[t][j] += b[t].x * vr - b[t].y * vi;
            pim[t][j] += b[t].x * vi + b[t].y * vr;
          }
        }
      }
    }
    // per-source partial sums enter the running sums with two-sum compensation
#pragma unroll
    for (int t = 0; t < RPL; ++t)
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        const float sr = ar[t][j] + pr[t][j], si = ai[t][j] + pim[t][j];
        const float br = sr - ar[t][j], bi = si - ai[t][j];
        cr[t][j] += (ar[t][j] - (sr - br)) + (pr[t][j] - br);
        ci[t][j] += (ai[t][j] - (si - bi)) + (pim[t][j] - bi);
        ar[t][j] = sr;
        ai[t][j] = si;
      }
  }
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int rr = rl + GS * t;
    if (rr < NB)
#pragma unroll
      for (int j = 0; j < RB; ++j) {
        red[gid][rr][j][0] = ar[t][j] + cr[t][j];
        red[gid][rr][j][1] = ai[t][j] + ci[t][j];
      }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NB * nr; i += blockDim.x) {
    const int rr = i % NB, j = i / NB;
    double sr = 0.0, si = 0.0;
    for (int q = 0; q < ngroups; ++q) {
      sr += (double)red[q][rr][j][0];
      si += (double)red[q][rr][j][1];
    }
    ysn[(size_t)(r0 + j) * vstride + (size_t)e * NB + rr] = make_double2(sr, si);
  }
}

__global__ void k_blocks_to_f32(size_t n, const double2 *__restrict__ in, float2 *__restrict__ out) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

efie_status dev_near_blocks_f32(Ctx *c) {
  size_t n = (size_t)c->nnear * c->nb * c->nb;
  EFIE_TRY(dalloc(c, &c->d_nblkf, n));
  k_blocks_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, c->d_nblk, c->d_nblkf); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

efie_status dev_near_apply(Ctx *c, const double2 *xs, double2 *ysn, cudaStream_t st);

// R right-hand sides, vector r at xs + r vstride (FP32 blocks of the mixed form)
efie_status dev_near_apply_batch(Ctx *c, int R, const double2 *xs, double2 *ysn, size_t vstride, cudaStream_t st) {
  constexpr int RB = 8;
  if (!c->d_nblkf) {
    for (int r = 0; r < R; ++r) EFIE_TRY(dev_near_apply(c, xs + r * vstride, ysn + r * vstride, st));
    return EFIE_OK;
  }
  const dim3 grid(c->nE, (R + RB - 1) / RB);
  const int threads = 32 * kApplyWarps;
  switch (c->nb) {
#define EFIE_APPLYB_CASE(NBV)                                                                                \
  case NBV:                                                                                                  \
    k_near_apply_multi<NBV, RB><<<grid, threads, 0, st>>>(c->nE, R, vstride, c->d_near_ptr, c->d_near_src,   \
                                                          c->d_nblkf, xs, ysn);                              \
    break;
    EFIE_APPLYB_CASE(8)
    EFIE_APPLYB_CASE(18)
    EFIE_APPLYB_CASE(32)
    EFIE_APPLYB_CASE(50)
#undef EFIE_APPLYB_CASE
    default:
      c->err = "unsupported block size";
      return EFIE_EINVAL;
  }
  ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

efie_status dev_near_apply(Ctx *c, const double2 *xs, double2 *ysn, cudaStream_t st) {
  const bool f32 = c->opt.precision == EFIE_MIXED_FP32 && c->d_nblkf;
  const int threads = 32 * kApplyWarps;
  if (f32) {
    const unsigned grid = (unsigned)c->nE;
    const float4 *B = reinterpret_cast<const float4 *>(c->d_nblkf);
    bool done = c->nb == 8 || c->nb == 18 || c->nb == 32;
    if (done) {
      if (!c->d_xsf) EFIE_TRY(dalloc(c, &c->d_xsf, (size_t)c->nsup));
      k_vec_to_f32<<<(c->nsup + 255) / 256, 256, 0, st>>>(c->nsup, xs, c->d_xsf);
      ++c->launches;
      const float2 *xf = c->d_xsf;
      // one warp per element, the same number of elements per warp: about 20 warps per SM
      const int per = (c->nE + c->nsm * 20 - 1) / (c->nsm * 20);
      const int nw = (c->nE + per - 1) / per;
      const unsigned gw = (unsigned)((nw + 3) / 4);
      if (c->nb == 8) k_near_apply_w<8, 2><<<gw, 128, 0, st>>>(c->nE, per, c->d_near_ptr, c->d_near_src, B, xf, ysn);
      else if (c->nb == 18) k_near_apply_w<18, 2><<<gw, 128, 0, st>>>(c->nE, per, c->d_near_ptr, c->d_near_src, B, xf, ysn);
      else k_near_apply_w<32, 2><<<gw, 128, 0, st>>>(c->nE, per, c->d_near_ptr, c->d_near_src, B, xf, ysn);
      ++c->launches;
      EFIE_CUDA(cudaGetLastError());
      return EFIE_OK;
    }
  }
  switch (c->nb) {
#define EFIE_APPLY_CASE(NBV)                                                                                   \
  case NBV:                                                                                                   \
    if (f32)                                                                                                  \
      k_near_apply<float, NBV><<<c->nE, threads, 0, st>>>(c->nE, c->d_near_ptr, c->d_near_src, c->d_nblkf, xs, \
                                                          ysn);                                              \
    else                                                                                                      \
      k_near_apply<double, NBV><<<c->nE, threads, 0, st>>>(c->nE, c->d_near_ptr, c->d_near_src, c->d_nblk, xs, \
                                                           ysn);                                             \
    break;
    EFIE_APPLY_CASE(8)
    EFIE_APPLY_CASE(18)
    EFIE_APPLY_CASE(32)
    EFIE_APPLY_CASE(50)
#undef EFIE_APPLY_CASE
    default:
      c->err = "unsupported block size";
      return EFIE_EINVAL;
  }
  ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

}  // namespace efie
