// Device-resident restarted GMRES (a11) for the complex symmetric EFIE system (Sec. 5: complex
// GMRES without preconditioner, restarted every 1500 iterations).  Arnoldi by classical
// Gram-Schmidt applied twice (CGS2) with deterministic two-stage reductions (fixed order,
// independent of launch timing), Givens rotations and back substitution on the device.
// Only the residual estimate (8 bytes) crosses to the host per iteration.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "efie_internal.h"
#include "gmres_ops.cuh"

namespace efie {

// part[i * nchunk + chunk] = sum_{t in chunk} conj(V_i[t]) w[t], i = i0 .. i0+7
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(int N, int nvec, const double2 *__restrict__ V, size_t ldv,
                                                             const double2 *__restrict__ w, double2 *__restrict__ part,
                                                             int nchunk) {
  dot_partial_chunk(N, nvec, blockIdx.y * kVecPerBlock, blockIdx.x, V, ldv, w, part, nchunk);
}

// h[i] = sum over chunks (one warp per vector, fixed order)
__global__ void k_dot_final(int nvec, int nchunk, const double2 *__restrict__ part, double2 *__restrict__ h) {
  int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i >= nvec) return;
  dot_final_warp(i, nchunk, part, h);
}

// w[t] += sgn * sum_i h[i] V_i[t], kCombRows entries per block
__global__ void __launch_bounds__(kCombThreads) k_combine(int N, int nvec, const double2 *__restrict__ V, size_t ldv,
                                                          const double2 *__restrict__ h, double sgn,
                                                          double2 *__restrict__ w) {
  combine_tile(N, blockIdx.x * kCombRows, nvec, V, ldv, h, sgn, w);
}

__global__ void k_scale_copy(int N, const double2 *__restrict__ w, const double *__restrict__ st, int idx,
                             double2 *__restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  out[t] = scaled_entry(w[t], st[idx]);
}

__global__ void k_residual(int N, const double2 *__restrict__ b, double2 *__restrict__ r) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  r[t] = make_double2(b[t].x - r[t].x, b[t].y - r[t].y);
}

__global__ void k_givens_init(double *st, int kr, const double2 *h) { givens_init_dev(st, kr, h); }

__global__ void k_givens_step(int j, int kr, const double2 *h1, const double2 *h2, const double2 *nrm2, double2 *H,
                              double *st) {
  givens_step_dev(j, kr, h1, h2, nrm2, H, st);
}

__global__ void k_backsolve(int jd, int kr, const double2 *H, const double *st, double2 *y) {
  backsolve_warp(jd, kr, H, st, y);
}

static efie_status ensure_part(Ctx *c, int N, int nvec) {
  int nchunk = (N + kChunk - 1) / kChunk;
  int need = nchunk * (nvec + kVecPerBlock);
  if (need > c->part_cap) {
    EFIE_TRY(dalloc(c, &c->d_part, (size_t)need));
    c->part_cap = need;
  }
  return EFIE_OK;
}

// h[0..nvec) = V^H w (V columns of stride ldv)
static efie_status dots(Ctx *c, int N, int nvec, const double2 *V, size_t ldv, const double2 *w, double2 *h) {
  EFIE_TRY(ensure_part(c, N, nvec));
  int nchunk = (N + kChunk - 1) / kChunk;
  dim3 grid(nchunk, (nvec + kVecPerBlock - 1) / kVecPerBlock);
  k_dot_partial<<<grid, kDotThreads, 0, c->stream>>>(N, nvec, V, ldv, w, c->d_part, nchunk); ++c->launches;
  k_dot_final<<<(nvec + 7) / 8, 256, 0, c->stream>>>(nvec, nchunk, c->d_part, h); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

void drop_product_graph(Ctx *c) {
  if (c->g_mv) cudaGraphExecDestroy(c->g_mv);
  c->g_mv = nullptr;
  dfree(c, c->d_mvin);
}

// out = A in for the single-system solver as one CUDA-graph launch: the product chain (about
// 20 small kernels around the M2L, near field on the second stream) is captured once per setup
// with input d_mvin and output d_w, and replayed, without the launch gaps between its kernels.
static efie_status gmres_product(Ctx *c, const double2 *in, double2 *out) {
  cudaStream_t st = c->stream;
  const size_t bytes = sizeof(double2) * (size_t)c->ndof;
  if (!c->g_mv) {
    EFIE_TRY(dalloc(c, &c->d_mvin, (size_t)c->ndof));
    EFIE_CUDA(cudaMemsetAsync(c->d_mvin, 0, bytes, st));
    EFIE_TRY(dev_matvec(c, c->d_mvin, c->d_w));  // buffers created on first use exist before the capture
    EFIE_CUDA(cudaStreamSynchronize(st));
    const long long l0 = c->launches;
    EFIE_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const efie_status s = dev_matvec(c, c->d_mvin, c->d_w);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    c->mv_kernels = c->launches - l0;
    c->launches = l0;
    if (s != EFIE_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    EFIE_CUDA(e);
    const cudaError_t ei = cudaGraphInstantiate(&c->g_mv, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) c->g_mv = nullptr;
    EFIE_CUDA(ei);
  }
  EFIE_CUDA(cudaMemcpyAsync(c->d_mvin, in, bytes, cudaMemcpyDeviceToDevice, st));
  EFIE_CUDA(cudaGraphLaunch(c->g_mv, st));
  if (out != c->d_w) EFIE_CUDA(cudaMemcpyAsync(out, c->d_w, bytes, cudaMemcpyDeviceToDevice, st));
  c->launches += c->mv_kernels;
  return EFIE_OK;
}

efie_status dev_gmres(Ctx *c, const double2 *b, double2 *x, int *its_out, double *res_out, int *conv_out) {
  const int N = c->ndof;
  const int kr = std::max(1, std::min(c->opt.gmres_restart, c->opt.gmres_maxit));
  cudaStream_t st = c->stream;
  if (kr != c->kr) {
    EFIE_TRY(dalloc(c, &c->d_V, (size_t)(kr + 1) * N));
    EFIE_TRY(dalloc(c, &c->d_H, (size_t)(kr + 1) * kr));
    EFIE_TRY(dalloc(c, &c->d_h, (size_t)kr + 1));
    EFIE_TRY(dalloc(c, &c->d_h2, (size_t)kr + 1));
    EFIE_TRY(dalloc(c, &c->d_gs, (size_t)2 + 5 * kr + 2));
    c->kr = kr;
  }
  if (!c->d_w) {
    EFIE_TRY(dalloc(c, &c->d_w, N));
    EFIE_TRY(dalloc(c, &c->d_r, N));
    EFIE_TRY(dalloc(c, &c->d_sol, (size_t)kr + 1));
  }
  if (!c->h_res) c->h_res = static_cast<double *>(pinned_get(4 * sizeof(double)));
  if (!c->h_res) {
    c->err = "pinned host buffer: cudaMallocHost failed";
    return EFIE_ENOMEM;
  }
  double2 *V = c->d_V;
  const int blk = 256, grid = (N + blk - 1) / blk;
  // ||b||
  EFIE_TRY(dots(c, N, 1, b, N, b, c->d_h));
  EFIE_CUDA(cudaMemcpyAsync(c->h_res, c->d_h, sizeof(double2), cudaMemcpyDeviceToHost, st));
  EFIE_CUDA(cudaStreamSynchronize(st));
  const double bn = std::sqrt(std::max(c->h_res[0], 0.0));
  const double target = c->opt.tol_is_relative ? c->opt.gmres_tol * bn : c->opt.gmres_tol;
  EFIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * N, st));
  int its = 0, conv = 0;
  double res = bn;
  if (bn == 0.0) conv = 1;
  bool first = true;
  while (!conv && its < c->opt.gmres_maxit) {
    // r = b - A x
    if (first) {
      EFIE_CUDA(cudaMemcpyAsync(c->d_r, b, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
    } else {
      EFIE_TRY(gmres_product(c, x, c->d_r));
      k_residual<<<grid, blk, 0, st>>>(N, b, c->d_r); ++c->launches;
    }
    first = false;
    EFIE_TRY(dots(c, N, 1, c->d_r, N, c->d_r, c->d_h));
    k_givens_init<<<1, 1, 0, st>>>(c->d_gs, kr, c->d_h); ++c->launches;
    k_scale_copy<<<grid, blk, 0, st>>>(N, c->d_r, c->d_gs, 0, V); ++c->launches;
    EFIE_CUDA(cudaMemcpyAsync(c->h_res, c->d_gs, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    EFIE_CUDA(cudaStreamSynchronize(st));
    res = c->h_res[1];
    if (res <= target) {
      conv = 1;
      break;
    }
    int jd = 0;
    for (int j = 0; j < kr && its < c->opt.gmres_maxit; ++j) {
      double2 *vj = V + (size_t)j * N;
      EFIE_TRY(gmres_product(c, vj, c->d_w));
      ++its;
      // CGS2
      EFIE_TRY(dots(c, N, j + 1, V, N, c->d_w, c->d_h));
      k_combine<<<(N + kCombRows - 1) / kCombRows, kCombThreads, 0, st>>>(N, j + 1, V, N, c->d_h, -1.0, c->d_w); ++c->launches;
      EFIE_TRY(dots(c, N, j + 1, V, N, c->d_w, c->d_h2));
      k_combine<<<(N + kCombRows - 1) / kCombRows, kCombThreads, 0, st>>>(N, j + 1, V, N, c->d_h2, -1.0, c->d_w); ++c->launches;
      EFIE_TRY(dots(c, N, 1, c->d_w, N, c->d_w, c->d_h2 + kr));
      k_givens_step<<<1, 1, 0, st>>>(j, kr, c->d_h, c->d_h2, c->d_h2 + kr, c->d_H, c->d_gs); ++c->launches;
      k_scale_copy<<<grid, blk, 0, st>>>(N, c->d_w, c->d_gs, 0, V + (size_t)(j + 1) * N); ++c->launches;
      EFIE_CUDA(cudaGetLastError());
      EFIE_CUDA(cudaMemcpyAsync(c->h_res, c->d_gs, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      EFIE_CUDA(cudaStreamSynchronize(st));
      res = c->h_res[1];
      jd = j + 1;
      if (res <= target || !(res == res)) break;
    }
    if (jd > 0) {
      k_backsolve<<<1, 32, 0, st>>>(jd, kr, c->d_H, c->d_gs, c->d_sol); ++c->launches;
      k_combine<<<(N + kCombRows - 1) / kCombRows, kCombThreads, 0, st>>>(N, jd, V, N, c->d_sol, 1.0, x); ++c->launches;
      EFIE_CUDA(cudaGetLastError());
    }
    if (res <= target) {
      // confirm with the true residual
      EFIE_TRY(gmres_product(c, x, c->d_r));
      k_residual<<<grid, blk, 0, st>>>(N, b, c->d_r); ++c->launches;
      EFIE_TRY(dots(c, N, 1, c->d_r, N, c->d_r, c->d_h));
      EFIE_CUDA(cudaMemcpyAsync(c->h_res, c->d_h, sizeof(double2), cudaMemcpyDeviceToHost, st));
      EFIE_CUDA(cudaStreamSynchronize(st));
      res = std::sqrt(std::max(c->h_res[0], 0.0));
      if (res <= target * 1.05) conv = 1;
      first = false;
    }
    if (!(res == res)) break;
  }
  *its_out = its;
  *res_out = c->opt.tol_is_relative ? (bn > 0 ? res / bn : 0.0) : res;
  *conv_out = conv;
  return EFIE_OK;
}

efie_status dev_norms(Ctx *c, int N, const double2 *v, double *out) {
  EFIE_TRY(dots(c, N, 1, v, N, v, c->d_h));
  EFIE_CUDA(cudaMemcpyAsync(c->h_res, c->d_h, sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  *out = std::sqrt(std::max(c->h_res[0], 0.0));
  return EFIE_OK;
}

}  // namespace efie

// ========================================================================================
// R independent systems advanced in lockstep: every step collects the one matvec each
// unfinished system needs (A v_j during Arnoldi, A x for a restart or the final residual
// check), applies them in one batched pass, then runs each system's Gram-Schmidt, Givens and
// back-substitution exactly as the single-system solver does.  One host synchronisation per
// step reads all residual estimates.
namespace efie {

namespace {
enum Phase { kStart, kArnoldi, kConfirm, kDone };

struct GSys {
  const double2 *b = nullptr;
  double2 *x = nullptr;
  double2 *V = nullptr, *H = nullptr, *h = nullptr, *h2 = nullptr, *w = nullptr, *r = nullptr, *sol = nullptr;
  double *gs = nullptr;
  double bn = 0, target = 0, res = 0;
  int its = 0, conv = 0, j = 0, phase = kStart;
  bool r_ready = false;  // r holds b (first cycle) or b - A x (after a failed check)
};

}  // namespace

size_t gmres_batch_bytes_per_system(const Ctx *c) {
  const size_t N = c->ndof, kr = std::max(1, std::min(c->opt.gmres_restart, c->opt.gmres_maxit));
  return 16 * ((kr + 1) * N + (kr + 1) * kr + 3 * (kr + 1) + 2 * N) + 8 * (5 * kr + 4);
}

efie_status dev_gmres_batch(Ctx *c, int R, const double2 *const *b, double2 *const *x, int *its_out,
                            double *res_out, int *conv_out) {
  const int N = c->ndof;
  const int kr = std::max(1, std::min(c->opt.gmres_restart, c->opt.gmres_maxit));
  const int maxit = c->opt.gmres_maxit;
  cudaStream_t st = c->stream;
  const int blk = 256, grid = (N + blk - 1) / blk;
  DevTemp mem;
  std::vector<GSys> S(R);
  for (int i = 0; i < R; ++i) {
    GSys &s = S[i];
    s.b = b[i];
    s.x = x[i];
    EFIE_TRY(mem.get(c, &s.V, (size_t)(kr + 1) * N));
    EFIE_TRY(mem.get(c, &s.H, (size_t)(kr + 1) * kr));
    EFIE_TRY(mem.get(c, &s.h, (size_t)kr + 1));
    EFIE_TRY(mem.get(c, &s.h2, (size_t)kr + 1));
    EFIE_TRY(mem.get(c, &s.sol, (size_t)kr + 1));
    EFIE_TRY(mem.get(c, &s.w, (size_t)N));
    EFIE_TRY(mem.get(c, &s.r, (size_t)N));
    EFIE_TRY(mem.get(c, &s.gs, (size_t)2 + 5 * kr + 2));
  }
  if (c->h_resB_cap < 4 * R) {
    pinned_put(c->h_resB);
    c->h_resB_cap = 0;
    c->h_resB = static_cast<double *>(pinned_get(4 * R * sizeof(double)));
    if (!c->h_resB) {
      c->err = "pinned host buffer: cudaMallocHost failed";
      return EFIE_ENOMEM;
    }
    c->h_resB_cap = 4 * R;
  }
  double *hr = c->h_resB;
  // ||b|| of every system
  for (int i = 0; i < R; ++i) {
    EFIE_TRY(dots(c, N, 1, S[i].b, N, S[i].b, S[i].h));
    EFIE_CUDA(cudaMemcpyAsync(hr + 4 * i, S[i].h, sizeof(double2), cudaMemcpyDeviceToHost, st));
    EFIE_CUDA(cudaMemsetAsync(S[i].x, 0, sizeof(double2) * N, st));
  }
  EFIE_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < R; ++i) {
    GSys &s = S[i];
    s.bn = std::sqrt(std::max(hr[4 * i], 0.0));
    s.target = c->opt.tol_is_relative ? c->opt.gmres_tol * s.bn : c->opt.gmres_tol;
    s.res = s.bn;
    if (s.bn == 0.0) {
      s.conv = 1;
      s.phase = kDone;
    } else {
      EFIE_CUDA(cudaMemcpyAsync(s.r, s.b, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
      s.r_ready = true;
    }
  }
  std::vector<const double2 *> in;
  std::vector<double2 *> out;
  std::vector<int> who;
  for (;;) {
    in.clear();
    out.clear();
    who.clear();
    for (int i = 0; i < R; ++i) {
      GSys &s = S[i];
      if (s.phase == kArnoldi) {
        in.push_back(s.V + (size_t)s.j * N);
        out.push_back(s.w);
        who.push_back(i);
      } else if ((s.phase == kStart && !s.r_ready) || s.phase == kConfirm) {
        in.push_back(s.x);
        out.push_back(s.r);
        who.push_back(i);
      }
    }
    bool any = false;
    for (const GSys &s : S) any |= s.phase != kDone;
    if (!any) break;
    if (!in.empty()) EFIE_TRY(dev_matvec_batch(c, (int)in.size(), in.data(), out.data()));
    for (int i : who)
      if (S[i].phase != kArnoldi) {
        k_residual<<<grid, blk, 0, st>>>(N, S[i].b, S[i].r); ++c->launches;
      }
    for (int i = 0; i < R; ++i) {
      GSys &s = S[i];
      if (s.phase == kStart) {
        EFIE_TRY(dots(c, N, 1, s.r, N, s.r, s.h));
        k_givens_init<<<1, 1, 0, st>>>(s.gs, kr, s.h); ++c->launches;
        k_scale_copy<<<grid, blk, 0, st>>>(N, s.r, s.gs, 0, s.V); ++c->launches;
        EFIE_CUDA(cudaMemcpyAsync(hr + 4 * i, s.gs, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      } else if (s.phase == kArnoldi) {
        const int j = s.j;
        EFIE_TRY(dots(c, N, j + 1, s.V, N, s.w, s.h));
        k_combine<<<(N + kCombRows - 1) / kCombRows, kCombThreads, 0, st>>>(N, j + 1, s.V, N, s.h, -1.0, s.w); ++c->launches;
        EFIE_TRY(dots(c, N, j + 1, s.V, N, s.w, s.h2));
        k_combine<<<(N + kCombRows - 1) / kCombRows, kCombThreads, 0, st>>>(N, j + 1, s.V, N, s.h2, -1.0, s.w); ++c->launches;
        EFIE_TRY(dots(c, N, 1, s.w, N, s.w, s.h2 + kr));
        k_givens_step<<<1, 1, 0, st>>>(j, kr, s.h, s.h2, s.h2 + kr, s.H, s.gs); ++c->launches;
        k_scale_copy<<<grid, blk, 0, st>>>(N, s.w, s.gs, 0, s.V + (size_t)(j + 1) * N); ++c->launches;
        EFIE_CUDA(cudaMemcpyAsync(hr + 4 * i, s.gs, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
      } else if (s.phase == kConfirm) {
        EFIE_TRY(dots(c, N, 1, s.r, N, s.r, s.h));
        EFIE_CUDA(cudaMemcpyAsync(hr + 4 * i, s.h, sizeof(double2), cudaMemcpyDeviceToHost, st));
      }
    }
    EFIE_CUDA(cudaGetLastError());
    EFIE_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < R; ++i) {
      GSys &s = S[i];
      if (s.phase == kStart) {
        s.r_ready = false;
        s.res = hr[4 * i + 1];
        if (s.res <= s.target) {
          s.conv = 1;
          s.phase = kDone;
        } else if (s.its >= maxit) {
          s.phase = kDone;
        } else {
          s.phase = kArnoldi;
          s.j = 0;
        }
      } else if (s.phase == kArnoldi) {
        ++s.its;
        s.res = hr[4 * i + 1];
        const int jd = s.j + 1;
        const bool nan = !(s.res == s.res);
        if (s.res <= s.target || nan || jd == kr || s.its >= maxit) {
          k_backsolve<<<1, 32, 0, st>>>(jd, kr, s.H, s.gs, s.sol); ++c->launches;
          k_combine<<<(N + kCombRows - 1) / kCombRows, kCombThreads, 0, st>>>(N, jd, s.V, N, s.sol, 1.0, s.x); ++c->launches;
          if (s.res <= s.target) s.phase = kConfirm;
          else if (nan || s.its >= maxit) s.phase = kDone;
          else s.phase = kStart;
        } else {
          s.j = jd;
        }
      } else if (s.phase == kConfirm) {
        s.res = std::sqrt(std::max(hr[4 * i], 0.0));
        if (s.res <= s.target * 1.05) {
          s.conv = 1;
          s.phase = kDone;
        } else if (!(s.res == s.res) || s.its >= maxit) {
          s.phase = kDone;
        } else {
          s.phase = kStart;
          s.r_ready = true;
        }
      }
    }
  }
  EFIE_CUDA(cudaStreamSynchronize(st));
  EFIE_TRY(m2l_tc_check(c));
  for (int i = 0; i < R; ++i) {
    its_out[i] = S[i].its;
    res_out[i] = c->opt.tol_is_relative ? (S[i].bn > 0 ? S[i].res / S[i].bn : 0.0) : S[i].res;
    conv_out[i] = S[i].conv;
  }
  return EFIE_OK;
}

}  // namespace efie
