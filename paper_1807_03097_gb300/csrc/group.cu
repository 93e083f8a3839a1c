// Lockstep GMRES over independent problems (a11 across problems): several contexts, each set up
// for its own geometry, wavenumber, degree and refinement, solve their systems together.  Every
// step of the lockstep is one CUDA-graph launch on the group's stream, whatever the number of
// problems; the graph has three parts:
//   pre:      upload of the step table, end-of-cycle back substitution and update of x,
//             packing of each system's product input into its context;
//   products: the operator products of all unfinished systems, one branch per context (each
//             branch the context's own product chain: T gather, moments, M2M, M2L, L2L,
//             evaluation, near field on a second stream, T^T scatter); the graph is captured
//             again only when a tenth of its product branches belong to finished systems;
//   post:     residuals, CGS2 (two passes), norms, Givens rotations, the next Krylov vector and
//             the residual estimates of all systems, then one device-to-host copy of them.
// The per-system work of pre and post runs in one launch per operation over a table of chunks
// of 2048 vector entries (system, chunk), with the same arithmetic in the same order as the
// single-context solver (gmres_ops.cuh), so that a system solved in a group follows the same
// iterates as alone up to the rounding of its products.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "efie_internal.h"
#include "gmres_ops.cuh"

namespace efie {

namespace {

enum : int {
  G_INIT = 1,      // x = 0, r = b
  G_NORMB = 2,     // ||b||^2
  G_PRE = 4,       // y = H^-1 g (jd columns), x += V y
  G_PROD_V = 8,    // product of V_j into w
  G_PROD_X = 16,   // product of x, r = b - A x
  G_ARN = 32,      // Arnoldi step j: CGS2, norm, Givens, V_{j+1}
  G_START = 64,    // ||r||, Givens start, V_0 = r / ||r||
  G_CONFIRM = 128  // ||r||^2 of the true residual
};

struct GSysD {
  int N, kr, mode, j, jd, nchunk;
  double2 *V, *H, *h, *h2, *sol, *w, *r, *x, *b, *px, *py, *part;
  double *gs;
};

__global__ void k_g_backsolve(const GSysD *__restrict__ T) {
  const GSysD &s = T[blockIdx.x];
  if (!(s.mode & G_PRE)) return;
  backsolve_warp(s.jd, s.kr, s.H, s.gs, s.sol);
}

// grid (chunks, kChunk / kCombRows): the block's kCombRows entries of its chunk
__global__ void __launch_bounds__(kCombThreads) k_g_update_pack(const GSysD *__restrict__ T, const int *__restrict__ csys,
                                                                 const int *__restrict__ cidx) {
  const GSysD s = T[csys[blockIdx.x]];
  const int t0 = cidx[blockIdx.x] * kChunk + blockIdx.y * kCombRows;
  if (t0 >= s.N) return;
  if (s.mode & G_PRE) combine_tile(s.N, t0, s.jd, s.V, (size_t)s.N, s.sol, 1.0, s.x);
  const int t = t0 + (int)threadIdx.x;
  if (threadIdx.x >= kCombRows || t >= s.N) return;
  if (s.mode & G_INIT) {
    s.x[t] = make_double2(0.0, 0.0);
    s.r[t] = s.b[t];
  }
  if (s.mode & G_PROD_V) s.px[t] = s.V[(size_t)s.j * s.N + t];
  else if (s.mode & G_PROD_X) s.px[t] = s.x[t];
}

__global__ void __launch_bounds__(kDotThreads) k_g_unpack(const GSysD *__restrict__ T, const int *__restrict__ csys,
                                                           const int *__restrict__ cidx) {
  const GSysD s = T[csys[blockIdx.x]];
  const int ch = cidx[blockIdx.x];
  for (int rr = 0; rr < kRowsPerThread; ++rr) {
    int t = ch * kChunk + rr * kDotThreads + threadIdx.x;
    if (t >= s.N) continue;
    if (s.mode & G_PROD_V) {
      s.w[t] = s.py[t];
    } else if (s.mode & G_PROD_X) {
      double2 y = s.py[t], b = s.b[t];
      s.r[t] = make_double2(b.x - y.x, b.y - y.y);
    }
  }
}

// vectors of the dot products of pass 0 (first CGS pass, or a norm), 1 (second CGS pass),
// 2 (norm of the orthogonalised vector)
__device__ __forceinline__ int dot_operands(const GSysD &s, int pass, const double2 *&V, const double2 *&w,
                                            double2 *&dst) {
  V = w = nullptr;
  dst = nullptr;
  if (pass == 0) {
    if (s.mode & G_NORMB) {
      V = w = s.b;
      dst = s.h;
      return 1;
    }
    if (s.mode & (G_START | G_CONFIRM)) {
      V = w = s.r;
      dst = s.h;
      return 1;
    }
    if (s.mode & G_ARN) {
      V = s.V;
      w = s.w;
      dst = s.h;
      return s.j + 1;
    }
    return 0;
  }
  if (!(s.mode & G_ARN)) return 0;
  if (pass == 1) {
    V = s.V;
    w = s.w;
    dst = s.h2;
    return s.j + 1;
  }
  V = w = s.w;
  dst = s.h2 + s.kr;
  return 1;
}

__global__ void __launch_bounds__(kDotThreads) k_g_dot_partial(const GSysD *__restrict__ T, const int *__restrict__ csys,
                                                                const int *__restrict__ cidx, int pass) {
  const GSysD s = T[csys[blockIdx.x]];
  const double2 *V, *w;
  double2 *dst;
  const int nvec = dot_operands(s, pass, V, w, dst);
  // grid (chunks, G): block y takes the vector groups y, y + G, ...
  for (int i0 = kVecPerBlock * blockIdx.y; i0 < nvec; i0 += kVecPerBlock * gridDim.y)
    dot_partial_chunk(s.N, nvec, i0, cidx[blockIdx.x], V, (size_t)s.N, w, s.part, s.nchunk);
}

__global__ void k_g_dot_final(const GSysD *__restrict__ T, int pass) {
  const GSysD s = T[blockIdx.x];
  const double2 *V, *w;
  double2 *dst;
  const int nvec = dot_operands(s, pass, V, w, dst);
  for (int i = threadIdx.x >> 5; i < nvec; i += blockDim.x >> 5) dot_final_warp(i, s.nchunk, s.part, dst);
}

__global__ void __launch_bounds__(kCombThreads) k_g_combine(const GSysD *__restrict__ T, const int *__restrict__ csys,
                                                             const int *__restrict__ cidx, int pass) {
  const GSysD s = T[csys[blockIdx.x]];
  if (!(s.mode & G_ARN)) return;
  const int t0 = cidx[blockIdx.x] * kChunk + blockIdx.y * kCombRows;
  if (t0 >= s.N) return;
  combine_tile(s.N, t0, s.j + 1, s.V, (size_t)s.N, pass == 0 ? s.h : s.h2, -1.0, s.w);
}

// one thread per system: Givens step or start, then the values the host reads
__global__ void k_g_givens(const GSysD *__restrict__ T, int nsys, double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsys) return;
  const GSysD &s = T[i];
  if (s.mode & G_ARN) givens_step_dev(s.j, s.kr, s.h, s.h2, s.h2 + s.kr, s.H, s.gs);
  else if (s.mode & G_START) givens_init_dev(s.gs, s.kr, s.h);
  if (s.mode & (G_ARN | G_START)) {
    out[2 * i] = s.gs[0];
    out[2 * i + 1] = s.gs[1];
  } else if (s.mode & (G_CONFIRM | G_NORMB)) {
    out[2 * i] = s.h[0].x;
    out[2 * i + 1] = 0.0;
  }
}

__global__ void __launch_bounds__(kDotThreads) k_g_scale(const GSysD *__restrict__ T, const int *__restrict__ csys,
                                                          const int *__restrict__ cidx) {
  const GSysD s = T[csys[blockIdx.x]];
  if (!(s.mode & (G_ARN | G_START))) return;
  const int ch = cidx[blockIdx.x];
  const double beta = s.gs[0];
  const double2 *src = (s.mode & G_ARN) ? s.w : s.r;
  double2 *dst = s.V + ((s.mode & G_ARN) ? (size_t)(s.j + 1) * s.N : 0);
  for (int rr = 0; rr < kRowsPerThread; ++rr) {
    int t = ch * kChunk + rr * kDotThreads + threadIdx.x;
    if (t < s.N) dst[t] = scaled_entry(src[t], beta);
  }
}

enum Phase { kStart, kArnoldi, kConfirm, kDone };

struct HostSys {
  int N = 0, kr = 1, maxit = 1;
  double tol = 0.0;
  bool rel = true;
  Phase phase = kStart;
  int j = 0, its = 0, conv = 0;
  bool r_ready = false, pre = false;
  int jd = 0;
  double bn = 0.0, target = 0.0, res = 0.0;
};

}  // namespace

struct Group {
  Ctx gc;  // device, stream and device memory of the group itself
  std::vector<Ctx *> ctx;
  std::vector<int> ndof;  // DOFs of each context when the group was made (the chunk table's sizes)
  int nsys = 0, kr_max = 1, nchunks = 0;
  GSysD *h_tab = nullptr, *d_tab = nullptr;
  double *h_out = nullptr, *d_out = nullptr;
  int *d_csys = nullptr, *d_cidx = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};  // around the three graphs of a step
  double graph_ms[3] = {0.0, 0.0, 0.0};                       // pre, products, post (last solve)
  std::vector<cudaEvent_t> joins;
  // one graph per step: g_step = pre + products + post, g_noprod = pre + post (steps in which
  // no system needs a product)
  cudaGraphExec_t g_step = nullptr, g_noprod = nullptr;
  std::vector<int> members;  // systems with a product branch in g_step
  long long prod_kernels = 0;  // kernel nodes of the product branches
  // statistics of the last solve
  long long steps = 0, captures = 0, kernels = 0;
  double solve_ms = 0.0;
};

namespace {

constexpr int kPreKernels = 2, kPostKernels = 11;

efie_status capture_graph(Group *g, cudaGraphExec_t *out, efie_status (*body)(Group *)) {
  Ctx *c = &g->gc;
  cudaStream_t st = c->stream;
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  EFIE_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  efie_status s = body(g);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (s != EFIE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  EFIE_CUDA(e);
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  EFIE_CUDA(e);
  return EFIE_OK;
}

efie_status body_pre(Group *g) {
  Ctx *c = &g->gc;
  cudaStream_t st = c->stream;
  EFIE_CUDA(cudaMemcpyAsync(g->d_tab, g->h_tab, sizeof(GSysD) * g->nsys, cudaMemcpyHostToDevice, st));
  k_g_backsolve<<<g->nsys, 32, 0, st>>>(g->d_tab);
  k_g_update_pack<<<dim3(g->nchunks, kChunk / kCombRows), kCombThreads, 0, st>>>(g->d_tab, g->d_csys, g->d_cidx);
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

efie_status body_post(Group *g) {
  Ctx *c = &g->gc;
  cudaStream_t st = c->stream;
  k_g_unpack<<<g->nchunks, kDotThreads, 0, st>>>(g->d_tab, g->d_csys, g->d_cidx);
  for (int pass = 0; pass < 3; ++pass) {
    const int groups = pass == 2 ? 1 : std::min(32, (g->kr_max + 1 + kVecPerBlock - 1) / kVecPerBlock);
    k_g_dot_partial<<<dim3(g->nchunks, groups), kDotThreads, 0, st>>>(g->d_tab, g->d_csys, g->d_cidx, pass);
    k_g_dot_final<<<g->nsys, 256, 0, st>>>(g->d_tab, pass);
    if (pass < 2)
      k_g_combine<<<dim3(g->nchunks, kChunk / kCombRows), kCombThreads, 0, st>>>(g->d_tab, g->d_csys, g->d_cidx, pass);
  }
  k_g_givens<<<(g->nsys + 127) / 128, 128, 0, st>>>(g->d_tab, g->nsys, g->d_out);
  k_g_scale<<<g->nchunks, kDotThreads, 0, st>>>(g->d_tab, g->d_csys, g->d_cidx);
  EFIE_CUDA(cudaMemcpyAsync(g->h_out, g->d_out, sizeof(double) * 2 * g->nsys, cudaMemcpyDeviceToHost, st));
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

efie_status body_prod(Group *g) {
  Ctx *c = &g->gc;
  cudaStream_t st = c->stream;
  EFIE_CUDA(cudaEventRecord(g->fork, st));
  long long k0 = 0;
  for (Ctx *m : g->ctx) k0 += m->launches;
  for (int i : g->members) {
    Ctx *m = g->ctx[i];
    EFIE_CUDA(cudaStreamWaitEvent(m->stream, g->fork, 0));
    efie_status s = dev_matvec(m, m->d_x, m->d_y);
    if (s != EFIE_OK) {
      c->err = "product of problem " + std::to_string(i) + ": " + m->err;
      return s;
    }
    EFIE_CUDA(cudaEventRecord(g->joins[i], m->stream));
    EFIE_CUDA(cudaStreamWaitEvent(st, g->joins[i], 0));
  }
  long long k1 = 0;
  for (Ctx *m : g->ctx) k1 += m->launches;
  g->prod_kernels = k1 - k0;
  return EFIE_OK;
}

// The whole step as one graph; external event-record nodes around its three parts give their
// device times.
efie_status body_step_t(Group *g, bool products) {
  cudaStream_t st = g->gc.stream;
  Ctx *c = &g->gc;
  EFIE_CUDA(cudaEventRecordWithFlags(g->tev[0], st, cudaEventRecordExternal));
  EFIE_TRY(body_pre(g));
  EFIE_CUDA(cudaEventRecordWithFlags(g->tev[1], st, cudaEventRecordExternal));
  if (products) EFIE_TRY(body_prod(g));
  EFIE_CUDA(cudaEventRecordWithFlags(g->tev[2], st, cudaEventRecordExternal));
  EFIE_TRY(body_post(g));
  EFIE_CUDA(cudaEventRecordWithFlags(g->tev[3], st, cudaEventRecordExternal));
  return EFIE_OK;
}
efie_status body_step(Group *g) { return body_step_t(g, true); }
efie_status body_noprod(Group *g) { return body_step_t(g, false); }

void release(Group *g) {
  Ctx *c = &g->gc;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (g->g_step) cudaGraphExecDestroy(g->g_step);
  if (g->g_noprod) cudaGraphExecDestroy(g->g_noprod);
  g->g_step = g->g_noprod = nullptr;
  dfree(c, g->d_tab);
  dfree(c, g->d_out);
  dfree(c, g->d_csys);
  dfree(c, g->d_cidx);
  if (c->stream) cudaStreamSynchronize(c->stream);
  pinned_put(g->h_tab);
  pinned_put(g->h_out);
  g->h_tab = nullptr;
  g->h_out = nullptr;
  if (g->fork) cudaEventDestroy(g->fork);
  for (cudaEvent_t &e : g->tev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : g->joins) cudaEventDestroy(e);
  g->joins.clear();
  if (c->stream) cudaStreamDestroy(c->stream);
  c->stream = nullptr;
  if (c->pool_held) pool_unref(c->device);
  c->pool_held = false;
}

}  // namespace

}  // namespace efie

using efie::Ctx;
using efie::Group;

extern "C" {

efie_status efie_group_create(efie_group **out, efie_ctx *const *ctxs, int nctx) {
  using namespace efie;
  if (!out) return EFIE_EINVAL;
  *out = nullptr;
  if (!ctxs || nctx < 1) return EFIE_EINVAL;
  int dev = -1;
  for (int i = 0; i < nctx; ++i) {
    Ctx *m = reinterpret_cast<Ctx *>(ctxs[i]);
    if (!m) return EFIE_EINVAL;
    if (!m->setup_done) return EFIE_ESTATE;
    if (dev < 0) dev = m->device;
    if (m->device != dev) return EFIE_EINVAL;
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return EFIE_EINVAL;
  }
  Group *g = new (std::nothrow) Group();
  if (!g) return EFIE_ENOMEM;
  Ctx *c = &g->gc;
  c->device = dev;
  cudaSetDevice(dev);
  auto fail = [&](efie_status s) {
    release(g);
    delete g;
    return s;
  };
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(EFIE_ECUDA);
  if (pool_ref(dev) != EFIE_OK) return fail(EFIE_ECUDA);
  c->pool_held = true;
  if (cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) != cudaSuccess) return fail(EFIE_ECUDA);
  for (cudaEvent_t &e : g->tev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(EFIE_ECUDA);
  g->nsys = nctx;
  for (int i = 0; i < nctx; ++i) {
    Ctx *m = reinterpret_cast<Ctx *>(ctxs[i]);
    g->ctx.push_back(m);
    g->ndof.push_back(m->ndof);
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(EFIE_ECUDA);
    g->joins.push_back(e);
  }
  // chunk table: (system, chunk) for every kChunk entries of every system
  std::vector<int> csys, cidx;
  for (int i = 0; i < nctx; ++i) {
    const int nch = (g->ctx[i]->ndof + kChunk - 1) / kChunk;
    for (int k = 0; k < nch; ++k) {
      csys.push_back(i);
      cidx.push_back(k);
    }
  }
  g->nchunks = (int)csys.size();
  g->h_tab = static_cast<GSysD *>(pinned_get(sizeof(GSysD) * nctx));
  g->h_out = static_cast<double *>(pinned_get(sizeof(double) * 2 * nctx));
  if (!g->h_tab || !g->h_out) return fail(EFIE_ENOMEM);
  std::fill(g->h_tab, g->h_tab + nctx, GSysD{});
  efie_status s;
  if ((s = dalloc(c, &g->d_tab, (size_t)nctx)) != EFIE_OK || (s = dalloc(c, &g->d_out, (size_t)2 * nctx)) != EFIE_OK ||
      (s = dalloc(c, &g->d_csys, csys.size())) != EFIE_OK || (s = dalloc(c, &g->d_cidx, cidx.size())) != EFIE_OK)
    return fail(s);
  if (cudaMemcpyAsync(g->d_csys, csys.data(), sizeof(int) * csys.size(), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(g->d_cidx, cidx.data(), sizeof(int) * cidx.size(), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return fail(EFIE_ECUDA);
  *out = reinterpret_cast<efie_group *>(g);
  return EFIE_OK;
}

efie_status efie_group_destroy(efie_group *grp) {
  if (!grp) return EFIE_OK;
  Group *g = reinterpret_cast<Group *>(grp);
  cudaSetDevice(g->gc.device);
  efie::release(g);
  delete g;
  return EFIE_OK;
}

const char *efie_group_last_error(const efie_group *grp) {
  if (!grp) return "null group";
  return reinterpret_cast<const Group *>(grp)->gc.err.c_str();
}

int efie_group_stats(const efie_group *grp, double *out, int n) {
  if (!grp || !out || n < 1) return 0;
  const Group *g = reinterpret_cast<const Group *>(grp);
  const double v[9] = {(double)g->steps, (double)g->captures, (double)g->kernels, g->solve_ms,
                       (double)g->prod_kernels, (double)g->nchunks, g->graph_ms[0], g->graph_ms[1], g->graph_ms[2]};
  const int k = std::min(n, 9);
  for (int i = 0; i < k; ++i) out[i] = v[i];
  return k;
}

efie_status efie_group_solve(efie_group *grp, const double *const *b, double *const *x, int ptr_kind, int *iterations,
                             double *residuals, int *converged) {
  using namespace efie;
  if (!grp || !b || !x) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  Group *g = reinterpret_cast<Group *>(grp);
  Ctx *c = &g->gc;
  cudaSetDevice(c->device);
  const int K = g->nsys;
  for (int i = 0; i < K; ++i)
    if (!b[i] || !x[i]) return EFIE_EINVAL;
  for (int i = 0; i < K; ++i)
    if (!g->ctx[i]->setup_done || g->ctx[i]->ndof != g->ndof[i]) {
      c->err = "problem " + std::to_string(i) + " was set up again with other sizes since the group was made";
      return EFIE_ESTATE;
    }
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<HostSys> S(K);
  DevTemp mem;
  int kr_max = 1;
  for (int i = 0; i < K; ++i) {
    Ctx *m = g->ctx[i];
    HostSys &s = S[i];
    s.N = m->ndof;
    s.kr = std::max(1, std::min(m->opt.gmres_restart, m->opt.gmres_maxit));
    s.maxit = m->opt.gmres_maxit;
    s.tol = m->opt.gmres_tol;
    s.rel = m->opt.tol_is_relative != 0;
    kr_max = std::max(kr_max, s.kr);
    GSysD &d = g->h_tab[i];
    d = GSysD{};
    d.N = s.N;
    d.kr = s.kr;
    d.nchunk = (s.N + kChunk - 1) / kChunk;
    const size_t N = s.N, kr = s.kr;
    EFIE_TRY(mem.get(c, &d.V, (kr + 1) * N));
    EFIE_TRY(mem.get(c, &d.H, (kr + 1) * kr));
    EFIE_TRY(mem.get(c, &d.h, kr + 1));
    EFIE_TRY(mem.get(c, &d.h2, kr + 1));
    EFIE_TRY(mem.get(c, &d.sol, kr + 1));
    EFIE_TRY(mem.get(c, &d.w, N));
    EFIE_TRY(mem.get(c, &d.r, N));
    EFIE_TRY(mem.get(c, &d.gs, 2 + 5 * kr + 2));
    EFIE_TRY(mem.get(c, &d.part, (size_t)d.nchunk * (kr + 1 + kVecPerBlock)));
    if (ptr_kind == EFIE_PTR_DEVICE) {
      d.b = reinterpret_cast<double2 *>(const_cast<double *>(b[i]));
      d.x = reinterpret_cast<double2 *>(x[i]);
    } else {
      EFIE_TRY(mem.get(c, &d.b, N));
      EFIE_TRY(mem.get(c, &d.x, N));
      EFIE_CUDA(cudaMemcpyAsync(d.b, b[i], 16 * N, cudaMemcpyHostToDevice, c->stream));
    }
    d.px = m->d_x;
    d.py = m->d_y;
  }
  g->kr_max = kr_max;
  // every context finishes what it has queued, then its product runs once outside a graph
  // (buffers created on first use exist before the capture)
  for (Ctx *m : g->ctx) {
    EFIE_CUDA(cudaMemsetAsync(m->d_x, 0, 16 * (size_t)m->ndof, m->stream));
    EFIE_TRY(dev_matvec(m, m->d_x, m->d_y));
  }
  for (Ctx *m : g->ctx) EFIE_CUDA(cudaStreamSynchronize(m->stream));
  g->members.clear();
  for (int i = 0; i < K; ++i) g->members.push_back(i);
  EFIE_TRY(capture_graph(g, &g->g_noprod, body_noprod));
  EFIE_TRY(capture_graph(g, &g->g_step, body_step));
  g->steps = 0;
  g->captures = 1;
  g->kernels = 0;

  g->graph_ms[0] = g->graph_ms[1] = g->graph_ms[2] = 0.0;
  auto run_step = [&](bool any_product) -> efie_status {
    EFIE_CUDA(cudaGraphLaunch(any_product ? g->g_step : g->g_noprod, c->stream));
    EFIE_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 3; ++k) {
      float ms = 0.f;
      EFIE_CUDA(cudaEventElapsedTime(&ms, g->tev[k], g->tev[k + 1]));
      g->graph_ms[k] += ms;
    }
    ++g->steps;
    g->kernels += kPreKernels + kPostKernels + 1 + (any_product ? g->prod_kernels : 0);
    return EFIE_OK;
  };

  // step 0: x = 0, r = b, ||b||
  for (int i = 0; i < K; ++i) g->h_tab[i].mode = G_INIT | G_NORMB;
  EFIE_TRY(run_step(false));
  for (int i = 0; i < K; ++i) {
    HostSys &s = S[i];
    s.bn = std::sqrt(std::max(g->h_out[2 * i], 0.0));
    s.target = s.rel ? s.tol * s.bn : s.tol;
    s.res = s.bn;
    if (s.bn == 0.0) {
      s.conv = 1;
      s.phase = kDone;
    } else {
      s.r_ready = true;
    }
  }
  for (;;) {
    bool any = false, any_pre = false, any_prod = false;
    int done = 0;
    for (int i = 0; i < K; ++i) {
      HostSys &s = S[i];
      GSysD &d = g->h_tab[i];
      int mode = 0;
      if (s.pre) {
        mode |= G_PRE;
        d.jd = s.jd;
        any_pre = true;
      }
      if (s.phase == kStart) {
        if (!s.r_ready) mode |= G_PROD_X;
        mode |= G_START;
      } else if (s.phase == kArnoldi) {
        mode |= G_PROD_V | G_ARN;
        d.j = s.j;
      } else if (s.phase == kConfirm) {
        mode |= G_PROD_X | G_CONFIRM;
      } else {
        ++done;
      }
      any |= s.phase != kDone;
      any_prod |= (mode & (G_PROD_V | G_PROD_X)) != 0;
      d.mode = mode;
      s.pre = false;
    }
    if (!any) {
      if (any_pre) EFIE_TRY(run_step(false));  // the last updates of x
      break;
    }
    // products of finished systems are wasted work: capture again once they are a tenth of
    // the graph's branches
    int stale = 0;
    for (int i : g->members) stale += S[i].phase == kDone;
    if (stale > 0 && 10 * stale >= (int)g->members.size()) {
      g->members.clear();
      for (int i = 0; i < K; ++i)
        if (S[i].phase != kDone) g->members.push_back(i);
      EFIE_TRY(capture_graph(g, &g->g_step, body_step));
      ++g->captures;
    }
    EFIE_TRY(run_step(any_prod));
    for (int i = 0; i < K; ++i) {
      HostSys &s = S[i];
      const double *o = g->h_out + 2 * i;
      if (s.phase == kStart) {
        s.r_ready = false;
        s.res = o[1];
        if (s.res <= s.target) {
          s.conv = 1;
          s.phase = kDone;
        } else if (s.its >= s.maxit) {
          s.phase = kDone;
        } else {
          s.phase = kArnoldi;
          s.j = 0;
        }
      } else if (s.phase == kArnoldi) {
        ++s.its;
        s.res = o[1];
        const int jd = s.j + 1;
        const bool nan = !(s.res == s.res);
        if (s.res <= s.target || nan || jd == s.kr || s.its >= s.maxit) {
          s.pre = true;
          s.jd = jd;
          if (s.res <= s.target) s.phase = kConfirm;
          else if (nan || s.its >= s.maxit) s.phase = kDone;
          else s.phase = kStart;
        } else {
          s.j = jd;
        }
      } else if (s.phase == kConfirm) {
        s.res = std::sqrt(std::max(o[0], 0.0));
        if (s.res <= s.target * 1.05) {
          s.conv = 1;
          s.phase = kDone;
        } else if (!(s.res == s.res) || s.its >= s.maxit) {
          s.phase = kDone;
        } else {
          s.phase = kStart;
          s.r_ready = true;
        }
      }
    }
  }
  for (int i = 0; i < K; ++i) {
    const GSysD &d = g->h_tab[i];
    if (ptr_kind == EFIE_PTR_HOST)
      EFIE_CUDA(cudaMemcpyAsync(x[i], d.x, 16 * (size_t)S[i].N, cudaMemcpyDeviceToHost, c->stream));
    if (iterations) iterations[i] = S[i].its;
    if (residuals) residuals[i] = S[i].rel ? (S[i].bn > 0 ? S[i].res / S[i].bn : 0.0) : S[i].res;
    if (converged) converged[i] = S[i].conv;
  }
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  g->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  bool all = true;
  for (const HostSys &s : S) all &= s.conv != 0;
  return all ? EFIE_OK : EFIE_NOT_CONVERGED;
}

efie_status efie_setup_many(efie_ctx *const *ctxs, int nctx, int nthreads, efie_status *status) {
  if (!ctxs || nctx < 0 || nthreads < 1) return EFIE_EINVAL;
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<efie_status> st(nctx, EFIE_OK);
  std::atomic<int> next{0};
  auto work = [&]() {
    cudaSetDevice(dev);
    for (int i = next++; i < nctx; i = next++) st[i] = ctxs[i] ? efie_setup(ctxs[i]) : EFIE_EINVAL;
  };
  std::vector<std::thread> th;
  const int nt = std::min(nthreads, std::max(nctx, 1));
  for (int t = 0; t < nt; ++t) th.emplace_back(work);
  for (std::thread &t : th) t.join();
  efie_status worst = EFIE_OK;
  for (int i = 0; i < nctx; ++i) {
    if (status) status[i] = st[i];
    if (st[i] < 0 && worst == EFIE_OK) worst = st[i];
  }
  return worst;
}

}  // extern "C"
