// extern "C" entry points of the library (include/efie.h).  Argument checking, host/device
// copies and the order of the setup phases; every numerical step is a CUDA kernel in the
// other translation units.
#include <chrono>
#include <cmath>
#include <vector>
#include <cstring>
#include <new>

#include "efie_internal.h"

using namespace efie;

namespace efie {
efie_status dev_batch_alloc(Ctx *c, int R);
efie_status dev_scatter(Ctx *c, const double2 *ys, double2 *y);
efie_status dev_gather(Ctx *c, const double2 *x, double2 *xs);
efie_status dev_norms(Ctx *c, int N, const double2 *v, double *out);
efie_status dev_near_apply(Ctx *c, const double2 *xs, double2 *ysn, cudaStream_t st);
}  // namespace efie

namespace {

// Returns every device buffer of the context to the pool (in stream order on c->stream;
// callers make sure that no work on the second stream still reads them).
void release_device(Ctx *c) {
  drop_product_graph(c);
  dfree(c, c->d_patches); dfree(c, c->d_knots); dfree(c, c->d_cpw);
  dfree(c, c->d_tg_ptr); dfree(c, c->d_tg_col); dfree(c, c->d_tg_val);
  dfree(c, c->d_ts_ptr); dfree(c, c->d_ts_col); dfree(c, c->d_ts_val);
  dfree(c, c->d_nodeX); dfree(c, c->d_nodeD); dfree(c, c->d_nodeXf); dfree(c, c->d_center);
  dfree(c, c->d_far_ptr); dfree(c, c->d_far_src); dfree(c, c->d_m2l_targets);
  dfree(c, c->d_near_ptr); dfree(c, c->d_near_src); dfree(c, c->d_nblk); dfree(c, c->d_nblkf); dfree(c, c->d_xsf);
  dfree(c, c->d_M); dfree(c, c->d_Md); dfree(c, c->d_E); dfree(c, c->d_Mf); dfree(c, c->d_Mdf); dfree(c, c->d_Ef);
  dfree(c, c->d_x); dfree(c, c->d_y); dfree(c, c->d_xs); dfree(c, c->d_ys); dfree(c, c->d_ysn);
  dfree(c, c->d_mom); dfree(c, c->d_src); dfree(c, c->d_acc); dfree(c, c->d_loc);
  dfree(c, c->d_momf); dfree(c, c->d_srcf); dfree(c, c->d_locf); dfree(c, c->d_accm); dfree(c, c->d_accf);
  dfree(c, c->d_nodeX4); dfree(c, c->d_pgeo); dfree(c, c->d_pph); dfree(c, c->d_far_tgt);
  dfree(c, c->d_own_ptr); dfree(c, c->d_own_src); dfree(c, c->d_own_slot); dfree(c, c->d_own_targets);
  dfree(c, c->d_par_ptr); dfree(c, c->d_par_slot); dfree(c, c->d_red); dfree(c, c->d_own_pgeo);
  dfree(c, c->d_own_pph); dfree(c, c->d_back);
  dfree(c, c->d_K);
  c->k_stored = false;
  dfree(c, c->d_V); dfree(c, c->d_H); dfree(c, c->d_h); dfree(c, c->d_h2); dfree(c, c->d_part); dfree(c, c->d_gs);
  dfree(c, c->d_w); dfree(c, c->d_r); dfree(c, c->d_b); dfree(c, c->d_sol);
  dfree(c, c->d_xB); dfree(c, c->d_yB); dfree(c, c->d_xsB); dfree(c, c->d_ysB); dfree(c, c->d_ysnB);
  dfree(c, c->d_momB); dfree(c, c->d_srcB); dfree(c, c->d_accB); dfree(c, c->d_locB); dfree(c, c->d_tc_err);
  c->batch_cap = 0;
  c->kr = 0;
  c->part_cap = 0;
}

efie_status check_options(const efie_options *o) {
  if (!o) return EFIE_EINVAL;
  if (o->p < 1 || o->p > 4) return EFIE_EINVAL;
  if (o->level_m < 0 || o->level_m > 10) return EFIE_EINVAL;
  if (!(o->kappa > 0.0) || !std::isfinite(o->kappa)) return EFIE_EINVAL;
  if (o->q < 1 || o->q + 1 > kMaxQ1) return EFIE_EINVAL;
  if (!(o->eta > 0.0)) return EFIE_EINVAL;
  if (o->precision != EFIE_FP64 && o->precision != EFIE_MIXED_FP32) return EFIE_EINVAL;
  if (o->quad_regular < 0 || o->quad_regular > 16 || o->quad_singular < 0 || o->quad_singular > 16) return EFIE_EINVAL;
  if (o->gmres_restart < 1 || o->gmres_maxit < 1 || !(o->gmres_tol > 0.0)) return EFIE_EINVAL;
  if (o->m2l_store < 0 || o->m2l_store > 2) return EFIE_EINVAL;
  if (o->m2l_batch < 0 || o->m2l_batch > 2) return EFIE_EINVAL;
  if (o->m2l_batch == 2 && (o->q + 1) * (o->q + 1) > 128) return EFIE_EINVAL;
  if (o->leaf_dense < 0 || o->leaf_dense > 1) return EFIE_EINVAL;
  if (o->m2l_pairs < 0 || o->m2l_pairs > 2) return EFIE_EINVAL;
  return EFIE_OK;
}

}  // namespace

extern "C" {

efie_status efie_check_device_waits(efie_ctx *ctx, long long cycles) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || cycles < 1 || cycles > (1ll << 32)) return EFIE_EINVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) return EFIE_ECUDA;
  return dev_wait_selftest(c, cycles);
}

const char *efie_last_error(const efie_ctx *ctx) {
  const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
  return c ? c->err.c_str() : "";
}

const char *efie_status_string(efie_status s) {
  switch (s) {
    case EFIE_OK: return "ok";
    case EFIE_NOT_CONVERGED: return "GMRES did not reach the tolerance within gmres_maxit iterations";
    case EFIE_EINVAL: return "invalid argument";
    case EFIE_ENOMEM: return "out of memory";
    case EFIE_EGEOMETRY: return "invalid geometry (open, non-manifold, mismatched or inward-oriented patches)";
    case EFIE_ECUDA: return "CUDA error";
    case EFIE_ESTATE: return "call out of order";
    case EFIE_ETIMEOUT: return "device wait timed out";
    case EFIE_PENDING: return "request pending";
    default: return "unknown status";
  }
}

efie_status efie_default_options(efie_options *o) {
  if (!o) return EFIE_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->p = 1;
  o->level_m = 2;
  o->kappa = 1.0;
  o->q = 4;
  o->eta = 1.6;
  o->precision = EFIE_FP64;
  o->gmres_restart = 1500;
  o->gmres_tol = 1e-8;
  o->gmres_maxit = 10000;
  o->tol_is_relative = 1;
  return EFIE_OK;
}

efie_status efie_create(efie_ctx **out, const efie_options *opt, void *cuda_stream) {
  if (!out) return EFIE_EINVAL;
  *out = nullptr;
  if (check_options(opt) != EFIE_OK) return EFIE_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return EFIE_ECUDA;
  Ctx *c = new (std::nothrow) Ctx();
  if (!c) return EFIE_ENOMEM;
  c->opt = *opt;
  cudaGetDevice(&c->device);
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (c->nsm < 1) c->nsm = 1;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return EFIE_ECUDA;
    }
    c->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess) {
    delete c;
    return EFIE_ECUDA;
  }
  for (int i = 0; i < 8; ++i) cudaEventCreate(&c->tm.ev[i]);
  c->tm.made = true;
  if (pool_ref(c->device) != EFIE_OK) {
    efie_destroy(reinterpret_cast<efie_ctx *>(c));
    return EFIE_ECUDA;
  }
  c->pool_held = true;
  *out = reinterpret_cast<efie_ctx *>(c);
  return EFIE_OK;
}

efie_status efie_destroy(efie_ctx *ctx) {
  if (!ctx) return EFIE_OK;
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->stream2) cudaStreamSynchronize(c->stream2);
  release_device(c);
  if (c->stream) cudaStreamSynchronize(c->stream);  // the stream-ordered frees are done
  pinned_put(c->h_res);
  pinned_put(c->h_resB);
  c->h_res = nullptr;
  c->h_resB = nullptr;
  c->h_resB_cap = 0;
  if (c->pool_held) pool_unref(c->device);
  if (c->tm.made)
    for (int i = 0; i < 8; ++i) cudaEventDestroy(c->tm.ev[i]);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  if (c->stream2) cudaStreamDestroy(c->stream2);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return EFIE_OK;
}

efie_status efie_set_geometry(efie_ctx *ctx, int n_patches, const int *deg, const int *ncp, const double *knots,
                              const double *cp, const double *w) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || n_patches <= 0 || n_patches > 100000 || !deg || !ncp || !knots || !cp || !w) return EFIE_EINVAL;
  cudaSetDevice(c->device);
  std::vector<PatchDesc> P(n_patches);
  std::vector<double> kn, hw;
  size_t ko = 0, co = 0;
  for (int j = 0; j < n_patches; ++j) {
    PatchDesc &d = P[j];
    for (int t = 0; t < 2; ++t) {
      d.deg[t] = deg[2 * j + t];
      d.ncp[t] = ncp[2 * j + t];
      if (d.deg[t] < 1 || d.deg[t] > kMaxGeoDeg || d.ncp[t] < d.deg[t] + 1 || d.ncp[t] > kMaxGeoCp) return EFIE_EINVAL;
      int nk = d.ncp[t] + d.deg[t] + 1;
      d.kofs[t] = (int)kn.size();
      for (int i = 0; i < nk; ++i) {
        double v = knots[ko + i];
        if (!std::isfinite(v) || (i > 0 && v < knots[ko + i - 1])) return EFIE_EINVAL;
        kn.push_back(v);
      }
      if (knots[ko] != 0.0 || knots[ko + nk - 1] != 1.0) return EFIE_EINVAL;
      ko += nk;
    }
    // reciprocal knot differences, so that the device evaluator divides by no knot span
    for (int t = 0; t < 2; ++t) {
      const int nk = d.ncp[t] + d.deg[t] + 1;
      const double *kt = kn.data() + d.kofs[t];
      std::vector<double> inv((size_t)d.deg[t] * nk, 0.0);
      for (int dd = 1; dd <= d.deg[t]; ++dd)
        for (int f = 0; f + dd < nk; ++f) {
          const double den = kt[f + dd] - kt[f];
          inv[(size_t)(dd - 1) * nk + f] = den > 0.0 ? 1.0 / den : 0.0;
        }
      d.iofs[t] = (int)kn.size();
      kn.insert(kn.end(), inv.begin(), inv.end());
    }
    d.cofs = (int)(hw.size() / 4);
    int nc = d.ncp[0] * d.ncp[1];
    for (int i = 0; i < nc; ++i) {
      double wt = w[co + i];
      if (!(wt > 0.0) || !std::isfinite(wt)) return EFIE_EINVAL;
      for (int k = 0; k < 3; ++k) {
        double v = cp[3 * (co + i) + k];
        if (!std::isfinite(v)) return EFIE_EINVAL;
        hw.push_back(wt * v);
      }
      hw.push_back(wt);
    }
    co += nc;
  }
  release_device(c);
  c->setup_done = false;
  c->np = n_patches;
  c->patches = P;
  c->knots = kn;
  c->cpw = hw;
  EFIE_TRY(dalloc(c, &c->d_patches, P.size()));
  EFIE_TRY(dalloc(c, &c->d_knots, kn.size()));
  EFIE_TRY(dalloc(c, &c->d_cpw, hw.size() / 4));
  EFIE_CUDA(cudaMemcpyAsync(c->d_patches, P.data(), sizeof(PatchDesc) * P.size(), cudaMemcpyHostToDevice,
                            c->stream));
  EFIE_CUDA(cudaMemcpyAsync(c->d_knots, kn.data(), 8 * kn.size(), cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(c->d_cpw, hw.data(), 8 * hw.size(), cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  c->have_geometry = true;
  return EFIE_OK;
}

efie_status efie_setup(efie_ctx *ctx) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c) return EFIE_EINVAL;
  if (!c->have_geometry) return EFIE_ESTATE;
  cudaSetDevice(c->device);
  drop_product_graph(c);  // the setup rebuilds the buffers it names
  auto t0 = std::chrono::steady_clock::now();
  const efie_options &o = c->opt;
  c->p = o.p;
  c->m = o.level_m;
  c->n = 1 << c->m;
  c->q = o.q;
  c->q1 = o.q + 1;
  c->nI = c->q1 * c->q1;
  c->p1 = o.p + 1;
  c->nb = 2 * c->p1 * c->p1;
  c->kappa = o.kappa;
  c->eta = o.eta;
  c->gr = o.quad_regular > 0 ? o.quad_regular : o.p + 4;
  c->gs = o.quad_singular > 0 ? o.quad_singular : o.p + 4;
  c->nE = c->np * c->n * c->n;
  c->nsup = c->nE * c->nb;
  host_tables(c);

  // interfaces, orientation, DOF map and T
  std::vector<int> pid;
  std::vector<double> st, X, D;
  for (int j = 0; j < c->np; ++j)
    for (int k = 0; k < 4; ++k)
      for (int t = 0; t < 5; ++t) {
        double u = t / 4.0;
        double s1 = k == 0 ? 0.0 : (k == 1 ? 1.0 : u), s2 = k == 2 ? 0.0 : (k == 3 ? 1.0 : u);
        pid.push_back(j);
        st.push_back(s1);
        st.push_back(s2);
      }
  EFIE_TRY(dev_eval_points(c, pid, st, X, nullptr));
  std::vector<double> none;
  EFIE_TRY(host_build_space(c, X, none));
  // outward orientation: enclosed volume (1/3) int x . (d1F x d2F) ds > 0
  {
    pid.clear();
    st.clear();
    std::vector<double> gx, gw;
    gauss_legendre01(8, gx, gw);
    for (int j = 0; j < c->np; ++j)
      for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b) {
          pid.push_back(j);
          st.push_back(gx[a]);
          st.push_back(gx[b]);
        }
    EFIE_TRY(dev_eval_points(c, pid, st, X, &D));
    double vol = 0.0;
    for (size_t i = 0; i < pid.size(); ++i) {
      const double *x = &X[3 * i], *d1 = &D[6 * i], *d2 = &D[6 * i + 3];
      double nx = d1[1] * d2[2] - d1[2] * d2[1], ny = d1[2] * d2[0] - d1[0] * d2[2], nz = d1[0] * d2[1] - d1[1] * d2[0];
      int a = (int)((i / 8) % 8), b = (int)(i % 8);
      vol += gw[a] * gw[b] * (x[0] * nx + x[1] * ny + x[2] * nz) / 3.0;
    }
    if (!(vol > 0.0)) {
      c->err = "patches are oriented inwards (d1F x d2F must point out of the enclosed volume)";
      return EFIE_EGEOMETRY;
    }
  }
  // vertex grid of every patch, for the classification of touching element pairs
  pid.clear();
  st.clear();
  for (int j = 0; j < c->np; ++j)
    for (int v2 = 0; v2 <= c->n; ++v2)
      for (int v1 = 0; v1 <= c->n; ++v1) {
        pid.push_back(j);
        st.push_back((double)v1 / c->n);
        st.push_back((double)v2 / c->n);
      }
  std::vector<double> corners;
  EFIE_TRY(dev_eval_points(c, pid, st, corners, nullptr));

  // cluster tree, geometry at the interpolation nodes, block-cluster tree
  c->lev_off.assign(c->m + 2, 0);
  for (int l = 0; l <= c->m; ++l) c->lev_off[l + 1] = c->lev_off[l] + c->np * (1 << (2 * l));
  c->ncl = c->lev_off[c->m + 1];
  EFIE_TRY(dev_cluster_geometry(c));
  EFIE_TRY(host_build_trees(c));

  // near field
  std::vector<NearPair> pairs;
  std::vector<int> mirror;
  EFIE_TRY(host_classify_near(c, corners, pairs, mirror));
  EFIE_TRY(dev_near_quadrature(c, pairs, mirror));
  if (c->opt.precision == EFIE_MIXED_FP32) EFIE_TRY(dev_near_blocks_f32(c));
  EFIE_TRY(dev_alloc_work(c));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  c->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  c->setup_done = true;
  return EFIE_OK;
}

efie_status efie_num_dofs(const efie_ctx *ctx, int64_t *n) {
  const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
  if (!c || !n) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  *n = c->ndof;
  return EFIE_OK;
}

efie_status efie_block_counts(const efie_ctx *ctx, int64_t *nfar, int64_t *nnear, int64_t *ncl, int64_t *nsup) {
  const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
  if (!c) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  if (nfar) *nfar = c->nfar;
  if (nnear) *nnear = c->nnear;
  if (ncl) *ncl = c->ncl;
  if (nsup) *nsup = c->nsup;
  return EFIE_OK;
}

efie_status efie_export_blocks(const efie_ctx *ctx, int *far, int *near) {
  const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
  if (!c) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  if (far) std::memcpy(far, c->far.data(), 4 * c->far.size());
  if (near) std::memcpy(near, c->nearl.data(), 4 * c->nearl.size());
  return EFIE_OK;
}

efie_status efie_export_near_blocks(efie_ctx *ctx, double *blocks) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || !blocks) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  cudaSetDevice(c->device);
  const size_t nb2 = (size_t)c->nb * c->nb;
  std::vector<double2> tmp(nb2 * c->nnear);
  EFIE_CUDA(cudaMemcpyAsync(tmp.data(), c->d_nblk, 16 * tmp.size(), cudaMemcpyDeviceToHost, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  double2 *out = reinterpret_cast<double2 *>(blocks);
  for (int at = 0; at < c->nnear; ++at) {
    int k = c->near_perm[at];
    for (int cc = 0; cc < c->nb; ++cc)
      for (int rr = 0; rr < c->nb; ++rr) out[(size_t)k * nb2 + rr * c->nb + cc] = tmp[(size_t)at * nb2 + cc * c->nb + rr];
  }
  return EFIE_OK;
}

// device times of the phases of the last product (events recorded by dev_matvec and
// dev_matvec_batch): total, gather, near field, moments + M2M, M2L, L2L + evaluation, scatter
static void collect_timings(Ctx *c) {
  float ms[7];
  cudaEventElapsedTime(&ms[0], c->tm.ev[0], c->tm.ev[6]);
  cudaEventElapsedTime(&ms[1], c->tm.ev[0], c->tm.ev[1]);
  cudaEventElapsedTime(&ms[2], c->tm.ev[1], c->tm.ev[2]);
  cudaEventElapsedTime(&ms[3], c->tm.ev[1], c->tm.ev[3]);
  cudaEventElapsedTime(&ms[4], c->tm.ev[3], c->tm.ev[4]);
  cudaEventElapsedTime(&ms[5], c->tm.ev[4], c->tm.ev[5]);
  cudaEventElapsedTime(&ms[6], c->tm.ev[5], c->tm.ev[6]);
  for (int i = 0; i < 7; ++i) c->last_ms[i] = ms[i];
}

efie_status efie_matvec(efie_ctx *ctx, int nrhs, const double *x, double *y, int ptr_kind) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || nrhs < 0 || (nrhs > 0 && (!x || !y))) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  cudaSetDevice(c->device);
  const size_t N = c->ndof;
  if (nrhs > 1 && c->opt.precision == EFIE_MIXED_FP32) {
    // all right-hand sides in one pass, in chunks of 64
    for (int r0 = 0; r0 < nrhs; r0 += 64) {
      const int R = std::min(64, nrhs - r0);
      const double2 *xr = reinterpret_cast<const double2 *>(x) + r0 * N;
      double2 *yr = reinterpret_cast<double2 *>(y) + r0 * N;
      const double2 *xp[64];
      double2 *yp[64];
      if (ptr_kind == EFIE_PTR_HOST) {
        EFIE_TRY(dev_batch_alloc(c, R));
        for (int r = 0; r < R; ++r) {
          xp[r] = c->d_xB + r * N;
          yp[r] = c->d_yB + r * N;
        }
        EFIE_CUDA(cudaMemcpyAsync(c->d_xB, xr, 16 * N * R, cudaMemcpyHostToDevice, c->stream));
        EFIE_TRY(dev_matvec_batch(c, R, xp, yp));
        EFIE_CUDA(cudaMemcpyAsync(yr, c->d_yB, 16 * N * R, cudaMemcpyDeviceToHost, c->stream));
      } else {
        for (int r = 0; r < R; ++r) {
          xp[r] = xr + r * N;
          yp[r] = yr + r * N;
        }
        EFIE_TRY(dev_matvec_batch(c, R, xp, yp));
      }
    }
    EFIE_CUDA(cudaStreamSynchronize(c->stream));
    collect_timings(c);  // phases of the last pass
    return m2l_tc_check(c);
  }
  for (int r = 0; r < nrhs; ++r) {
    const double2 *xr = reinterpret_cast<const double2 *>(x) + r * N;
    double2 *yr = reinterpret_cast<double2 *>(y) + r * N;
    if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(c->d_x, xr, 16 * N, cudaMemcpyHostToDevice, c->stream));
      EFIE_TRY(dev_matvec(c, c->d_x, c->d_y));
      EFIE_CUDA(cudaMemcpyAsync(yr, c->d_y, 16 * N, cudaMemcpyDeviceToHost, c->stream));
    } else {
      EFIE_TRY(dev_matvec(c, xr, yr));
    }
  }
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  if (nrhs > 0) collect_timings(c);
  return EFIE_OK;
}

efie_status efie_near_apply(efie_ctx *ctx, const double *xs, double *ys, int ptr_kind) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || !xs || !ys) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  cudaSetDevice(c->device);
  const size_t S = c->nsup;
  const double2 *in = reinterpret_cast<const double2 *>(xs);
  double2 *out = reinterpret_cast<double2 *>(ys);
  DevTemp tmp;
  if (ptr_kind == EFIE_PTR_HOST) {
    double2 *ti = nullptr, *to = nullptr;
    EFIE_TRY(tmp.get(c, &ti, S));
    EFIE_TRY(tmp.get(c, &to, S));
    EFIE_CUDA(cudaMemcpyAsync(ti, xs, 16 * S, cudaMemcpyHostToDevice, c->stream));
    in = ti;
    out = to;
  }
  EFIE_CUDA(cudaEventRecord(c->tm.ev[0], c->stream));
  EFIE_TRY(dev_near_apply(c, in, out, c->stream));
  EFIE_CUDA(cudaEventRecord(c->tm.ev[1], c->stream));
  if (ptr_kind == EFIE_PTR_HOST) EFIE_CUDA(cudaMemcpyAsync(ys, out, 16 * S, cudaMemcpyDeviceToHost, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->tm.ev[0], c->tm.ev[1]);
  for (int i = 0; i < 7; ++i) c->last_ms[i] = 0.f;
  c->last_ms[0] = c->last_ms[2] = ms;
  return EFIE_OK;
}

efie_status efie_matvec_superspace(efie_ctx *ctx, const double *xs, double *ys, int ptr_kind) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || !xs || !ys) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  cudaSetDevice(c->device);
  const size_t S = c->nsup;
  double2 *in = c->d_xs, *out = c->d_ys;
  double2 *tmp_in = nullptr, *tmp_out = nullptr;
  DevTemp tmp;
  if (ptr_kind == EFIE_PTR_HOST) {
    EFIE_TRY(tmp.get(c, &tmp_in, S));
    EFIE_TRY(tmp.get(c, &tmp_out, S));
    EFIE_CUDA(cudaMemcpyAsync(tmp_in, xs, 16 * S, cudaMemcpyHostToDevice, c->stream));
    in = tmp_in;
    out = tmp_out;
  } else {
    in = reinterpret_cast<double2 *>(const_cast<double *>(xs));
    out = reinterpret_cast<double2 *>(ys);
  }
  EFIE_TRY(dev_matvec_super(c, in, out));
  if (ptr_kind == EFIE_PTR_HOST) EFIE_CUDA(cudaMemcpyAsync(ys, out, 16 * S, cudaMemcpyDeviceToHost, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  return EFIE_OK;
}

efie_status efie_matvec_superspace_batch(efie_ctx *ctx, int nrhs, const double *xs, double *ys, int ptr_kind) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || nrhs < 0 || (nrhs > 0 && (!xs || !ys))) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  if (nrhs == 0) return EFIE_OK;
  cudaSetDevice(c->device);
  const size_t S = c->nsup;
  const int chunk = std::min(64, nrhs);
  DevTemp tmp;
  double2 *din = nullptr, *dout = nullptr;
  if (ptr_kind == EFIE_PTR_HOST) {
    EFIE_TRY(tmp.get(c, &din, (size_t)chunk * S));
    EFIE_TRY(tmp.get(c, &dout, (size_t)chunk * S));
  }
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int R = std::min(chunk, nrhs - r0);
    const double2 *xr = reinterpret_cast<const double2 *>(xs) + r0 * S;
    double2 *yr = reinterpret_cast<double2 *>(ys) + r0 * S;
    const double2 *xp[64];
    double2 *yp[64];
    if (ptr_kind == EFIE_PTR_HOST)
      EFIE_CUDA(cudaMemcpyAsync(din, xr, 16 * S * R, cudaMemcpyHostToDevice, c->stream));
    for (int r = 0; r < R; ++r) {
      xp[r] = ptr_kind == EFIE_PTR_HOST ? din + r * S : xr + r * S;
      yp[r] = ptr_kind == EFIE_PTR_HOST ? dout + r * S : yr + r * S;
    }
    EFIE_TRY(dev_matvec_batch(c, R, xp, yp, true));
    if (ptr_kind == EFIE_PTR_HOST)
      EFIE_CUDA(cudaMemcpyAsync(yr, dout, 16 * S * R, cudaMemcpyDeviceToHost, c->stream));
  }
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  collect_timings(c);
  return m2l_tc_check(c);
}

efie_status efie_rhs_plane_waves(efie_ctx *ctx, int nrhs, const double *dir, const double *pol, double *g,
                                 int ptr_kind) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || nrhs < 0 || (nrhs > 0 && (!dir || !pol || !g))) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  cudaSetDevice(c->device);
  const size_t N = c->ndof;
  for (int r = 0; r < nrhs; ++r) {
    double2 *gr = reinterpret_cast<double2 *>(g) + r * N;
    double2 *dst = ptr_kind == EFIE_PTR_HOST ? c->d_y : gr;
    EFIE_TRY(dev_rhs(c, dir + 3 * r, pol + 3 * r, dst));
    if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(gr, c->d_y, 16 * N, cudaMemcpyDeviceToHost, c->stream));
      EFIE_CUDA(cudaStreamSynchronize(c->stream));
    }
  }
  return EFIE_OK;
}

// Several right-hand sides in the mixed form: lockstep GMRES over chunks of systems whose
// Krylov bases fit in the free device memory, so every step applies one batched matvec.
static efie_status solve_batched(Ctx *c, int nrhs, const double *b, double *x, int ptr_kind, const double *dir,
                                 const double *pol, int *its_max, int *all_conv, double *worst) {
  const size_t N = c->ndof;
  size_t fr = 0, tot = 0;
  EFIE_CUDA(cudaMemGetInfo(&fr, &tot));
  const size_t per = gmres_batch_bytes_per_system(c) + 32 * N + size_t(40) * c->nsup +
                     size_t(80) * c->ncl * c->nI;
  int chunk = (int)std::min<size_t>(64, (size_t)(0.8 * (double)fr) / std::max<size_t>(per, 1));
  if (chunk < 1) {
    c->err = "solve: the Krylov basis of one system does not fit in the free device memory";
    return EFIE_ENOMEM;
  }
  chunk = std::min(chunk, nrhs);
  EFIE_TRY(dev_batch_alloc(c, chunk));
  double2 *d_bb = nullptr, *d_xx = nullptr;
  DevTemp tmp;
  EFIE_TRY(tmp.get(c, &d_bb, (size_t)chunk * N));
  if (ptr_kind == EFIE_PTR_HOST) EFIE_TRY(tmp.get(c, &d_xx, (size_t)chunk * N));
  std::vector<const double2 *> bp(chunk);
  std::vector<double2 *> xp(chunk);
  std::vector<int> its(chunk), conv(chunk);
  std::vector<double> res(chunk);
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int R = std::min(chunk, nrhs - r0);
    for (int r = 0; r < R; ++r) {
      const int g = r0 + r;
      double2 *bd = d_bb + (size_t)r * N;
      if (dir) {
        EFIE_TRY(dev_rhs(c, dir + 3 * g, pol + 3 * g, bd));
        bp[r] = bd;
      } else if (ptr_kind == EFIE_PTR_HOST) {
        EFIE_CUDA(cudaMemcpyAsync(bd, reinterpret_cast<const double2 *>(b) + g * N, 16 * N, cudaMemcpyHostToDevice,
                                  c->stream));
        bp[r] = bd;
      } else {
        bp[r] = reinterpret_cast<const double2 *>(b) + g * N;
      }
      xp[r] = ptr_kind == EFIE_PTR_HOST ? d_xx + (size_t)r * N : reinterpret_cast<double2 *>(x) + g * N;
    }
    EFIE_TRY(dev_gmres_batch(c, R, bp.data(), xp.data(), its.data(), res.data(), conv.data()));
    if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(reinterpret_cast<double2 *>(x) + r0 * N, d_xx, 16 * N * R, cudaMemcpyDeviceToHost,
                                c->stream));
      EFIE_CUDA(cudaStreamSynchronize(c->stream));
    }
    for (int r = 0; r < R; ++r) {
      *its_max = std::max(*its_max, its[r]);
      *worst = std::max(*worst, res[r]);
      if (!conv[r]) *all_conv = 0;
    }
  }
  return EFIE_OK;
}

static efie_status solve_impl(Ctx *c, int nrhs, const double *b, double *x, int ptr_kind, efie_solve_info *info,
                              const double *dir, const double *pol) {
  const size_t N = c->ndof;
  if (!c->d_b) EFIE_TRY(dalloc(c, &c->d_b, N));
  efie_status result = EFIE_OK;
  int its_max = 0, all_conv = 1;
  double worst = 0.0;
  auto t0 = std::chrono::steady_clock::now();
  if (nrhs > 1 && c->opt.precision == EFIE_MIXED_FP32) {
    EFIE_TRY(solve_batched(c, nrhs, b, x, ptr_kind, dir, pol, &its_max, &all_conv, &worst));
    if (!all_conv) result = EFIE_NOT_CONVERGED;
    nrhs = 0;
  }
  for (int r = 0; r < nrhs; ++r) {
    double2 *xr = reinterpret_cast<double2 *>(x) + r * N;
    const double2 *br = b ? reinterpret_cast<const double2 *>(b) + r * N : nullptr;
    if (dir) {
      EFIE_TRY(dev_rhs(c, dir + 3 * r, pol + 3 * r, c->d_b));
    } else if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(c->d_b, br, 16 * N, cudaMemcpyHostToDevice, c->stream));
    } else {
      EFIE_CUDA(cudaMemcpyAsync(c->d_b, br, 16 * N, cudaMemcpyDeviceToDevice, c->stream));
    }
    double2 *dst = ptr_kind == EFIE_PTR_HOST ? c->d_x : xr;
    int its = 0, conv = 0;
    double res = 0.0;
    EFIE_TRY(dev_gmres(c, c->d_b, dst, &its, &res, &conv));
    if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(xr, c->d_x, 16 * N, cudaMemcpyDeviceToHost, c->stream));
      EFIE_CUDA(cudaStreamSynchronize(c->stream));
    }
    its_max = std::max(its_max, its);
    worst = std::max(worst, res);
    if (!conv) {
      all_conv = 0;
      result = EFIE_NOT_CONVERGED;
    }
  }
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  c->info.iterations = its_max;
  c->info.converged = all_conv;
  c->info.residual = worst;
  c->info.setup_ms = c->setup_ms;
  c->info.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = c->info;
  return result;
}

efie_status efie_solve(efie_ctx *ctx, int nrhs, const double *b, double *x, int ptr_kind, efie_solve_info *info) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || nrhs < 0 || (nrhs > 0 && (!b || !x))) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  cudaSetDevice(c->device);
  return solve_impl(c, nrhs, b, x, ptr_kind, info, nullptr, nullptr);
}

efie_status efie_solve_plane_waves(efie_ctx *ctx, int nrhs, const double *dir, const double *pol, double *w,
                                   int ptr_kind, efie_solve_info *info) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || nrhs < 0 || (nrhs > 0 && (!dir || !pol || !w))) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  cudaSetDevice(c->device);
  return solve_impl(c, nrhs, nullptr, w, ptr_kind, info, dir, pol);
}

efie_status efie_far_field(efie_ctx *ctx, int nrhs, const double *w, int ndir, const double *dirs, double *e_inf,
                           int ptr_kind) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || nrhs < 0 || ndir < 0 || (nrhs > 0 && ndir > 0 && (!w || !dirs || !e_inf))) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  if (ndir == 0 || nrhs == 0) return EFIE_OK;
  cudaSetDevice(c->device);
  const size_t N = c->ndof;
  double2 *d_out = nullptr;
  DevTemp tmp;
  EFIE_TRY(tmp.get(c, &d_out, 3 * (size_t)ndir));
  for (int r = 0; r < nrhs; ++r) {
    const double2 *wr = reinterpret_cast<const double2 *>(w) + r * N;
    double2 *er = reinterpret_cast<double2 *>(e_inf) + (size_t)r * ndir * 3;
    const double2 *src = wr;
    if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(c->d_x, wr, 16 * N, cudaMemcpyHostToDevice, c->stream));
      src = c->d_x;
    }
    EFIE_TRY(dev_far_field(c, src, ndir, dirs, ptr_kind == EFIE_PTR_HOST ? d_out : er));
    if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(er, d_out, 48 * (size_t)ndir, cudaMemcpyDeviceToHost, c->stream));
      EFIE_CUDA(cudaStreamSynchronize(c->stream));
    }
  }
  return EFIE_OK;
}

efie_status efie_exterior_field(efie_ctx *ctx, int nrhs, const double *w, int npts, const double *pts,
                                double *e_out, int ptr_kind) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || nrhs < 0 || npts < 0 || npts > 65535 || (nrhs > 0 && npts > 0 && (!w || !pts || !e_out)))
    return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  if (npts == 0 || nrhs == 0) return EFIE_OK;
  cudaSetDevice(c->device);
  const size_t N = c->ndof;
  double2 *d_out = nullptr;
  DevTemp tmp;
  EFIE_TRY(tmp.get(c, &d_out, 3 * (size_t)npts));
  for (int r = 0; r < nrhs; ++r) {
    const double2 *wr = reinterpret_cast<const double2 *>(w) + r * N;
    double2 *er = reinterpret_cast<double2 *>(e_out) + (size_t)r * npts * 3;
    const double2 *src = wr;
    if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(c->d_x, wr, 16 * N, cudaMemcpyHostToDevice, c->stream));
      src = c->d_x;
    }
    EFIE_TRY(dev_exterior_field(c, src, npts, pts, ptr_kind == EFIE_PTR_HOST ? d_out : er));
    if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(er, d_out, 48 * (size_t)npts, cudaMemcpyDeviceToHost, c->stream));
      EFIE_CUDA(cudaStreamSynchronize(c->stream));
    }
  }
  return EFIE_OK;
}

efie_status efie_rhs_dipole(efie_ctx *ctx, int nrhs, const double *x0, const double *p0, double *g, int ptr_kind) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || nrhs < 0 || (nrhs > 0 && (!x0 || !p0 || !g))) return EFIE_EINVAL;
  if (ptr_kind != EFIE_PTR_HOST && ptr_kind != EFIE_PTR_DEVICE) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  cudaSetDevice(c->device);
  const size_t N = c->ndof;
  for (int r = 0; r < nrhs; ++r) {
    double2 *gr = reinterpret_cast<double2 *>(g) + r * N;
    double2 *dst = ptr_kind == EFIE_PTR_HOST ? c->d_y : gr;
    EFIE_TRY(dev_rhs_dipole(c, x0 + 3 * r, p0 + 3 * r, dst));
    if (ptr_kind == EFIE_PTR_HOST) {
      EFIE_CUDA(cudaMemcpyAsync(gr, c->d_y, 16 * N, cudaMemcpyDeviceToHost, c->stream));
      EFIE_CUDA(cudaStreamSynchronize(c->stream));
    }
  }
  return EFIE_OK;
}

int efie_setup_timings(const efie_ctx *ctx, double *out, int n) {
  const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
  if (!c || !out) return 0;
  const double v[9] = {c->setup_ms, (double)c->near_quad_ms, (double)c->near_quad_points, (double)c->near_quad_pairs,
                       (double)c->near_sep_ms, (double)c->near_sep_pairs, (double)c->m2l_tune_ms[0],
                       (double)c->m2l_tune_ms[1], c->d_back ? 1.0 : 0.0};
  int k = n < 9 ? n : 9;
  for (int i = 0; i < k; ++i) out[i] = v[i];
  return k;
}

efie_status efie_device_bytes(const efie_ctx *ctx, int64_t *live, int64_t *peak) {
  Ctx *c = reinterpret_cast<Ctx *>(const_cast<efie_ctx *>(ctx));
  if (!c) return EFIE_EINVAL;
  std::lock_guard<std::mutex> lk(c->mem_mu);
  if (live) *live = (int64_t)c->live_bytes;
  if (peak) *peak = (int64_t)c->peak_bytes;
  return EFIE_OK;
}

int64_t efie_launch_count(const efie_ctx *ctx) {
  const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
  return c ? (int64_t)c->launches : -1;
}

int efie_last_timings(const efie_ctx *ctx, double *out, int n) {
  const Ctx *c = reinterpret_cast<const Ctx *>(ctx);
  if (!c || !out) return 0;
  int k = n < 7 ? n : 7;
  for (int i = 0; i < k; ++i) out[i] = c->last_ms[i];
  return k;
}

}  // extern "C"
