// Device steps of the restarted GMRES (a11) shared by the single-system solver, the lockstep
// batch of one context and the lockstep group of independent problems, so that all three take
// the same arithmetic in the same order.
#pragma once

#include <cuda_runtime.h>

namespace efie {

constexpr int kDotThreads = 256;
constexpr int kRowsPerThread = 8;
constexpr int kChunk = kDotThreads * kRowsPerThread;  // vector entries per partial dot product
constexpr int kVecPerBlock = 8;
static_assert(kVecPerBlock == kDotThreads / 32, "one warp reduces one vector of a dot-product block");

// Partial dot products of one chunk: part[i * nchunk + chunk] = sum_{t in chunk} conj(V_i[t]) w[t]
// for i = i0 .. i0 + 7 (i < nvec).  Each thread sums its kRowsPerThread entries for the 8
// vectors; warp v then adds the 256 thread sums of vector v (8 per lane, then a shuffle tree), in
// a fixed order.  Called by all kDotThreads threads of a block.
__device__ __forceinline__ void dot_partial_chunk(int N, int nvec, int i0, int chunk, const double2 *__restrict__ V,
                                                  size_t ldv, const double2 *__restrict__ w,
                                                  double2 *__restrict__ part, int nchunk) {
  double2 acc[kVecPerBlock];
#pragma unroll
  for (int v = 0; v < kVecPerBlock; ++v) acc[v] = make_double2(0.0, 0.0);
  for (int rr = 0; rr < kRowsPerThread; ++rr) {
    int t = chunk * kChunk + rr * kDotThreads + threadIdx.x;
    if (t < N) {
      double2 wt = w[t];
#pragma unroll
      for (int v = 0; v < kVecPerBlock; ++v) {
        int i = i0 + v;
        if (i < nvec) {
          // conj(a) w as four FMAs into the running sums (FP64 is GB300's scarcest pipe)
          double2 a = V[(size_t)i * ldv + t];
          acc[v].x = fma(a.x, wt.x, acc[v].x);
          acc[v].x = fma(a.y, wt.y, acc[v].x);
          acc[v].y = fma(a.x, wt.y, acc[v].y);
          acc[v].y = fma(-a.y, wt.x, acc[v].y);
        }
      }
    }
  }
  __shared__ double2 red[kVecPerBlock][kDotThreads + 1];
#pragma unroll
  for (int v = 0; v < kVecPerBlock; ++v) red[v][threadIdx.x] = acc[v];
  __syncthreads();
  {
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double x = 0.0, y = 0.0;
#pragma unroll
    for (int k = 0; k < kDotThreads / 32; ++k) {
      x += red[v][lane + 32 * k].x;
      y += red[v][lane + 32 * k].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
    }
    if (lane == 0 && i0 + v < nvec) part[(size_t)(i0 + v) * nchunk + chunk] = make_double2(x, y);
  }
  __syncthreads();  // red is reused by the next call of the block
}

// h[i] = sum over the chunks of part[i][.], one warp, fixed order.
__device__ __forceinline__ void dot_final_warp(int i, int nchunk, const double2 *__restrict__ part,
                                               double2 *__restrict__ h) {
  int lane = threadIdx.x & 31;
  double x = 0.0, y = 0.0;
  for (int k = lane; k < nchunk; k += 32) {
    x += part[(size_t)i * nchunk + k].x;
    y += part[(size_t)i * nchunk + k].y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
  }
  if (lane == 0) h[i] = make_double2(x, y);
}

// w[t] += sgn * sum_i c_i V_i[t] for the kCombRows entries t0 .. t0 + 31 of one block of
// kCombThreads threads: warp k sums the vectors i = k, k + 8, k + 16, ... for its lane's entry
// (each load a 512-byte row segment), and the 8 partial sums are added in the order k = 0..7.
constexpr int kCombRows = 32;
constexpr int kCombThreads = 256;
__device__ __forceinline__ void combine_tile(int N, int t0, int nvec, const double2 *__restrict__ V, size_t ldv,
                                             const double2 *__restrict__ c, double sgn, double2 *__restrict__ w) {
  __shared__ double2 part[kCombThreads / 32][kCombRows];
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5, t = t0 + lane;
  double x = 0.0, y = 0.0;
  if (t < N) {
    for (int i = k; i < nvec; i += kCombThreads / 32) {
      double2 a = V[(size_t)i * ldv + t], ci = c[i];
      x = fma(ci.x, a.x, x);
      x = fma(-ci.y, a.y, x);
      y = fma(ci.x, a.y, y);
      y = fma(ci.y, a.x, y);
    }
  }
  part[k][lane] = make_double2(x, y);
  __syncthreads();
  if (k == 0 && t < N) {
    double sx = 0.0, sy = 0.0;
    for (int kk = 0; kk < kCombThreads / 32; ++kk) {
      sx += part[kk][lane].x;
      sy += part[kk][lane].y;
    }
    w[t].x += sgn * sx;
    w[t].y += sgn * sy;
  }
  __syncthreads();
}

__device__ __forceinline__ double2 scaled_entry(double2 w, double beta) {
  double f = beta > 0.0 ? 1.0 / beta : 0.0;
  return make_double2(w.x * f, w.y * f);
}

// Givens state layout in st: [0] beta of the new vector, [1] residual estimate,
// [2 .. 2+kr) cs, then sn (complex) [kr][2], then g (complex) [kr+1][2].
__device__ __forceinline__ void givens_init_dev(double *st, int kr, const double2 *h) {
  // g = (||r||, 0, ...); h[0] holds ||r||^2
  double beta = sqrt(h[0].x);
  double *g = st + 2 + kr + 2 * kr;
  for (int i = 0; i <= kr; ++i) {
    g[2 * i] = 0.0;
    g[2 * i + 1] = 0.0;
  }
  g[0] = beta;
  st[0] = beta;
  st[1] = beta;
}

// Column j of the Hessenberg matrix from the CGS2 coefficients h1 + h2 and the norm of the
// orthogonalised vector; previous rotations, new rotation, residual estimate |g_{j+1}|.
__device__ __forceinline__ void givens_step_dev(int j, int kr, const double2 *h1, const double2 *h2,
                                                const double2 *nrm2, double2 *H, double *st) {
  double *cs = st + 2;
  double *sn = st + 2 + kr;       // complex [kr]
  double *g = st + 2 + 3 * kr;    // complex [kr+1]
  double beta = sqrt(fmax(nrm2[0].x, 0.0));
  // the new column h1 + h2, rotated by the previous rotations; the entry that rotation i passes
  // on to row i + 1 stays in a register (the column of H is strided in memory)
  double2 a = make_double2(h1[0].x + h2[0].x, h1[0].y + h2[0].y);
  for (int i = 0; i < j; ++i) {
    const double2 b = make_double2(h1[i + 1].x + h2[i + 1].x, h1[i + 1].y + h2[i + 1].y);
    const double c = cs[i], sr = sn[2 * i], si = sn[2 * i + 1];
    // [a; b] <- [c a + s b; -conj(s) a + c b]
    const double2 na = make_double2(c * a.x + sr * b.x - si * b.y, c * a.y + sr * b.y + si * b.x);
    const double2 nb = make_double2(-(sr * a.x + si * a.y) + c * b.x, -(sr * a.y - si * a.x) + c * b.y);
    H[(size_t)i * kr + j] = na;
    a = nb;
  }
  double aa = hypot(a.x, a.y), tt = hypot(aa, beta);
  double c, sr, si;
  if (aa == 0.0) {
    c = 0.0; sr = 1.0; si = 0.0;
  } else {
    c = aa / tt;
    sr = (a.x / aa) * beta / tt;
    si = (a.y / aa) * beta / tt;
  }
  cs[j] = c;
  sn[2 * j] = sr;
  sn[2 * j + 1] = si;
  H[(size_t)j * kr + j] = make_double2(c * a.x + sr * beta, c * a.y + si * beta);
  double gr = g[2 * j], gi = g[2 * j + 1];
  g[2 * (j + 1)] = -(sr * gr + si * gi);
  g[2 * (j + 1) + 1] = -(sr * gi - si * gr);
  g[2 * j] = c * gr;
  g[2 * j + 1] = c * gi;
  st[0] = beta;
  st[1] = hypot(g[2 * (j + 1)], g[2 * (j + 1) + 1]);
}

// y = H(0:jd, 0:jd)^{-1} g(0:jd), one warp: row sums in parallel, rows in sequence.
__device__ __forceinline__ void backsolve_warp(int jd, int kr, const double2 *H, const double *st, double2 *y) {
  const double *g = st + 2 + 3 * kr;
  int lane = threadIdx.x & 31;
  for (int i = jd - 1; i >= 0; --i) {
    double x = 0.0, z = 0.0;
    for (int t = i + 1 + lane; t < jd; t += 32) {
      double2 hh = H[(size_t)i * kr + t], yy = y[t];
      x += hh.x * yy.x - hh.y * yy.y;
      z += hh.x * yy.y + hh.y * yy.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      z += __shfl_down_sync(0xffffffffu, z, o);
    }
    if (lane == 0) {
      double sr = g[2 * i] - x, si = g[2 * i + 1] - z;
      double2 d = H[(size_t)i * kr + i];
      double den = d.x * d.x + d.y * d.y;
      y[i] = make_double2((sr * d.x + si * d.y) / den, (si * d.x - sr * d.y) / den);
    }
    __syncwarp();
  }
}

}  // namespace efie
