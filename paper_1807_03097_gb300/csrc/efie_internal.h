// Internal definitions of the GB300 EFIE library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/efie.h"

namespace efie {

constexpr int kMaxGeoDeg = 8;     // NURBS degree limit of the device evaluator
constexpr int kMaxGeoCp = 64;     // control points per direction
constexpr int kMaxQ1 = 17;        // q + 1 interpolation points per direction
constexpr int kMaxP1 = 7;         // p + 1 Bernstein functions per direction

// One NURBS patch as the device sees it: offsets into the packed knot and homogeneous
// control point arrays.
struct PatchDesc {
  int deg[2];
  int ncp[2];
  int kofs[2];  // offset of the s1 / s2 knot vector in the knot array
  int iofs[2];  // offset of the reciprocal knot differences 1 / (t_{f+d} - t_f) of each
                // direction in the knot array, [deg][ncp + deg + 1] (0 where t_{f+d} = t_f)
  int cofs;     // offset of the [ncp1][ncp0] homogeneous control net (w x, w y, w z, w)
};

// Quadrature meta data of one near-field element pair.
struct NearPair {
  int e, e2;    // target, source element
  int kind;     // 0 separated, 1 common vertex, 2 common edge, 3 identical
  int r1, r2;   // square symmetries taking the canonical Duffy coordinates to each element
};

struct Timers {
  cudaEvent_t ev[8];
  bool made = false;
};

// Per-level tables of the hierarchical interpolation (Sec. 4.2): constant across levels
// because every cluster is mapped onto its own parameter box.
struct Tables {
  std::vector<double> xcheb;  // q+1 Chebyshev nodes on [0,1]
  std::vector<double> M;      // [q1][p1]  int_0^1 L_m B_a
  std::vector<double> Md;     // [q1][p1]  int_0^1 L_m B_a'
  std::vector<double> E;      // [2][q1][q1]  E_c[m][m'] = L_m((c + x_m') / 2)
  std::vector<double> gx, gw;  // Gauss rule of quad_regular points
  std::vector<double> sx, sw;  // Gauss rule of quad_singular points
};

struct Ctx {
  efie_options opt{};
  int device = 0;
  int nsm = 152;  // streaming multiprocessors of the device
  cudaStream_t stream = nullptr;
  cudaStream_t stream2 = nullptr;  // near-field apply overlaps the far-field chain
  cudaEvent_t fork = nullptr, join = nullptr;
  bool own_stream = false;

  // geometry (host copy, homogeneous control points)
  int np = 0;
  std::vector<PatchDesc> patches;
  std::vector<double> knots;
  std::vector<double> cpw;  // [..][4]
  bool have_geometry = false;
  PatchDesc *d_patches = nullptr;
  double *d_knots = nullptr;
  double4 *d_cpw = nullptr;

  // discretisation
  int p = 1, m = 0, n = 1, q = 1, q1 = 2, nI = 4, p1 = 2, nb = 8;
  int nE = 0, nsup = 0, ndof = 0;
  int gr = 5, gs = 5;  // Gauss orders
  double kappa = 1.0, eta = 1.6;
  std::vector<int> edge_nbr;  // [np*4][3]: neighbour patch, edge, reversed

  // T (eq. superspace) as CSR in both directions
  int *d_tg_ptr = nullptr, *d_tg_col = nullptr;
  double *d_tg_val = nullptr;
  int *d_ts_ptr = nullptr, *d_ts_col = nullptr;
  double *d_ts_val = nullptr;
  int nT = 0;

  // clusters
  int ncl = 0;
  std::vector<int> lev_off;  // [m+2]
  std::vector<double> ball;  // [ncl][4]
  double *d_nodeX = nullptr;  // [ncl][nI][3]
  double *d_nodeD = nullptr;  // [ncl][nI][6]  (d1F, d2F)
  float *d_nodeXf = nullptr;  // [ncl][nI][3] offsets from the cluster centre (FP32 path)
  double *d_center = nullptr; // [ncl][3]

  // block-cluster tree (Algorithm 1)
  std::vector<int> far;   // [nfar][3] (level, target, source)
  std::vector<int> nearl; // [nnear][2]
  int nfar = 0, nnear = 0;
  int *d_far_ptr = nullptr, *d_far_src = nullptr;  // CSR by target cluster
  int *d_m2l_targets = nullptr;
  int n_m2l_targets = 0;
  int m2l_mode = 2;  // FP32 M2L phase: 0 direct kappa r - kappa r0, 1 split, 2 split + explicit reduction
  int *d_far_tgt = nullptr;   // target cluster of every far pair (CSR order)
  // unordered far pairs of the single right-hand-side FP32 M2L: each pair {t, s} is owned by
  // one of its clusters (balanced), which receives K_ts w_s; the other receives K_ts^T w_t
  // through the pair's slot of d_back, summed per cluster in a fixed order
  int npairs = 0;
  int *d_own_ptr = nullptr, *d_own_src = nullptr, *d_own_slot = nullptr;  // CSR by owner cluster
  int *d_own_targets = nullptr;  // owners with at least one pair, most pairs first
  int n_own_targets = 0;
  int *d_par_ptr = nullptr, *d_par_slot = nullptr;  // CSR by the non-owner cluster
  int *d_red = nullptr;          // clusters with any far pair
  int n_red = 0;
  float4 *d_own_pgeo = nullptr;  // per owned pair: c_owner - c_other, r0
  float2 *d_own_pph = nullptr;   // per owned pair: e^{i kappa r0} / (4 pi)
  float4 *d_back = nullptr;      // [npairs][nI][2]: K^T contributions to the non-owner
  float m2l_tune_ms[2] = {0.f, 0.f};  // autotuned M2L (m2l_pairs = 2): ordered, unordered
  void *d_K = nullptr;        // stored coupling matrices [pair][m'][m] (double2 or float2)
  bool k_stored = false;
  // several right-hand sides (mixed form)
  int batch_cap = 0;
  double *h_resB = nullptr;  // pinned residual estimates of a lockstep batch
  int h_resB_cap = 0;
  double2 *d_xB = nullptr, *d_yB = nullptr, *d_xsB = nullptr, *d_ysB = nullptr, *d_ysnB = nullptr;
  float2 *d_momB = nullptr, *d_srcB = nullptr, *d_accB = nullptr, *d_locB = nullptr;
  int *d_tc_err = nullptr;   // set by a tensor-core M2L whose pipeline wait ran out
  int *d_near_ptr = nullptr, *d_near_src = nullptr;  // CSR by target element
  double2 *d_nblk = nullptr;  // [nnear][nb (col)][nb (row)]
  float2 *d_nblkf = nullptr;  // FP32 copy of the blocks (mixed-precision apply)
  float2 *d_xsf = nullptr;    // x* in FP32 for the FP32 block product [nsup]
  std::vector<int> near_perm;  // CSR position -> index in nearl

  // tables on the device
  double *d_M = nullptr, *d_Md = nullptr, *d_E = nullptr;
  float *d_Mf = nullptr, *d_Mdf = nullptr, *d_Ef = nullptr;
  Tables tab;

  // work vectors (FP64)
  double2 *d_x = nullptr, *d_y = nullptr, *d_xs = nullptr, *d_ys = nullptr, *d_ysn = nullptr;
  double2 *d_mom = nullptr;  // [ncl][3][nI]
  double2 *d_src = nullptr;  // [ncl][4][nI]
  double2 *d_acc = nullptr;  // [ncl][4][nI]
  double2 *d_loc = nullptr;  // [ncl][3][nI]
  // work vectors (FP32 path)
  float2 *d_momf = nullptr, *d_locf = nullptr;
  float4 *d_srcf = nullptr;   // [ncl][nI][2]: (u_x, u_y), (u_z, nu) folded source fields
  float4 *d_accf = nullptr;   // [ncl][nI][2]: M2L results, same layout
  float4 *d_nodeX4 = nullptr; // [ncl][nI] node offsets from the cluster centre (x, y, z, 0)
  float4 *d_pgeo = nullptr;   // per far pair (CSR order): centre offset d = c_t - c_s, r0 = |d|
  float2 *d_pph = nullptr;    // per far pair: e^{i kappa r0} / (4 pi)
  double2 *d_accm = nullptr;

  // GMRES
  int kr = 0;  // allocated restart length
  double2 *d_V = nullptr;     // [kr+1][ndof]
  double2 *d_H = nullptr;     // [kr+1][kr]
  double2 *d_h = nullptr;     // [kr+1]
  double2 *d_h2 = nullptr;    // [kr+1]
  double2 *d_part = nullptr;  // partial dot products
  double *d_gs = nullptr;     // Givens / residual state
  double2 *d_w = nullptr, *d_r = nullptr, *d_b = nullptr, *d_sol = nullptr;
  double *h_res = nullptr;    // pinned host mirror of the residual estimate
  int part_cap = 0;
  // the product of the single-system solver as one graph: A d_mvin -> d_w (captured once per
  // setup; dropped whenever the buffers it names are released or rebuilt)
  cudaGraphExec_t g_mv = nullptr;
  double2 *d_mvin = nullptr;
  long long mv_kernels = 0;  // kernels in g_mv

  // device memory of this context (stream-ordered pool allocations, devmem.cpp)
  std::mutex mem_mu;
  std::unordered_map<void *, size_t> live;
  size_t live_bytes = 0, peak_bytes = 0;
  bool pool_held = false;

  bool setup_done = false;
  long long launches = 0;  // kernels launched by this context (all phases)
  Timers tm;
  float last_ms[7] = {0, 0, 0, 0, 0, 0, 0};
  double setup_ms = 0.0;
  // near-field quadrature of the last setup: kernel time (CUDA events), quadrature points
  // evaluated (parts x g^4 summed over the pairs integrated), pairs integrated
  float near_quad_ms = 0.f;
  long long near_quad_points = 0;
  int near_quad_pairs = 0;
  // separated pairs (element-table kernel): kernel time, pairs integrated
  float near_sep_ms = 0.f;
  int near_sep_pairs = 0;
  efie_solve_info info{};
  std::string err;
};

// drop the captured product graph of the single-system solver (gmres.cu)
void drop_product_graph(Ctx *c);

// helpers implemented in the .cu / .cpp files
efie_status host_build_space(Ctx *c, const std::vector<double> &edge_pts, const std::vector<double> &corner_pts);
efie_status host_build_trees(Ctx *c);
efie_status host_classify_near(Ctx *c, const std::vector<double> &corner_pts, std::vector<NearPair> &pairs,
                               std::vector<int> &mirror);
void host_tables(Ctx *c);
void gauss_legendre01(int g, std::vector<double> &x, std::vector<double> &w);

// device-side phases
efie_status dev_eval_points(Ctx *c, const std::vector<int> &patch, const std::vector<double> &st,
                            std::vector<double> &X, std::vector<double> *D);
efie_status dev_cluster_geometry(Ctx *c);
efie_status dev_near_quadrature(Ctx *c, const std::vector<NearPair> &pairs, const std::vector<int> &mirror);
efie_status dev_matvec_super(Ctx *c, const double2 *xs, double2 *ys);  // ys = (N + F) xs
efie_status dev_matvec(Ctx *c, const double2 *x, double2 *y);           // y = T^T (N+F) T x
efie_status dev_rhs(Ctx *c, const double *dir, const double *pol, double2 *g);
efie_status dev_far_field(Ctx *c, const double2 *w, int ndir, const double *dirs, double2 *out);
efie_status dev_gmres(Ctx *c, const double2 *b, double2 *x, int *its, double *res, int *conv);
efie_status dev_alloc_work(Ctx *c);
efie_status dev_near_blocks_f32(Ctx *c);
efie_status dev_near_apply_batch(Ctx *c, int R, const double2 *xs, double2 *ysn, size_t vstride, cudaStream_t st);
// Y[r] = A X[r] for r < R (host arrays of device pointers); one pass in the mixed form
// superspace: X[r], Y[r] are superspace vectors and Y[r] = (N + F) X[r]
efie_status dev_matvec_batch(Ctx *c, int R, const double2 *const *X, double2 *const *Y, bool superspace = false);
// R independent GMRES solves advanced in lockstep, one batched matvec per step
size_t gmres_batch_bytes_per_system(const Ctx *c);
// tensor-core M2L of a batch (m2l_tc.cu)
bool m2l_tc_supported(const Ctx *c);
efie_status m2l_tc_prepare(Ctx *c);
efie_status launch_m2l_tc(Ctx *c, cudaStream_t st, int F, int ld, const float2 *src, float2 *acc);
efie_status m2l_tc_check(Ctx *c);
efie_status dev_wait_selftest(Ctx *c, long long cycles);
// exterior field and the dipole right-hand side (exterior.cu)
efie_status dev_exterior_field(Ctx *c, const double2 *w, int npts, const double *pts, double2 *out);
efie_status dev_rhs_dipole(Ctx *c, const double *x0, const double *p0, double2 *g);
efie_status dev_gmres_batch(Ctx *c, int R, const double2 *const *b, double2 *const *x, int *its, double *res,
                            int *conv);

#define EFIE_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      c->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
      return (e_ == cudaErrorMemoryAllocation) ? EFIE_ENOMEM : EFIE_ECUDA;           \
    }                                                                                \
  } while (0)

#define EFIE_TRY(expr)             \
  do {                             \
    efie_status s_ = (expr);       \
    if (s_ < 0) return s_;         \
  } while (0)

// Device memory (devmem.cpp): stream-ordered allocations on the context's stream from one pool
// per device, counted per context.  pool_ref / pool_unref bracket the lifetime of a context or
// a server on a device; pinned_get / pinned_put hand out reusable pinned host buffers.
efie_status pool_ref(int dev);
void pool_unref(int dev);
efie_status pool_alloc(Ctx *c, void **p, size_t bytes);
void pool_free(Ctx *c, void *p);  // stream-ordered on c->stream
void *pinned_get(size_t bytes);
void pinned_put(void *p);

template <class T>
inline void dfree(Ctx *c, T *&p) {
  if (p) pool_free(c, (void *)p);
  p = nullptr;
}

template <class T>
inline efie_status dalloc(Ctx *c, T **p, size_t count) {
  dfree(c, *p);
  void *q = nullptr;
  efie_status s = pool_alloc(c, &q, (count ? count : 1) * sizeof(T));
  *p = static_cast<T *>(q);
  return s;
}

// Temporary device buffers of one call, returned to the pool (in stream order) when the owner
// goes out of scope, also on the early returns of EFIE_TRY / EFIE_CUDA.
struct DevTemp {
  Ctx *c = nullptr;
  std::vector<void *> p;
  DevTemp() = default;
  DevTemp(const DevTemp &) = delete;
  DevTemp &operator=(const DevTemp &) = delete;
  ~DevTemp() {
    for (void *q : p) pool_free(c, q);
  }
  template <class T>
  efie_status get(Ctx *ctx, T **out, size_t n) {
    c = ctx;
    void *q = nullptr;
    efie_status s = pool_alloc(ctx, &q, (n ? n : 1) * sizeof(T));
    *out = static_cast<T *>(q);
    if (s == EFIE_OK) p.push_back(q);
    return s;
  }
};

inline int morton2(int i1, int i2) {
  int k = 0;
  for (int b = 0; b < 15; ++b) k |= (((i1 >> b) & 1) << (2 * b)) | (((i2 >> b) & 1) << (2 * b + 1));
  return k;
}
inline void unmorton2(int k, int &i1, int &i2) {
  i1 = 0;
  i2 = 0;
  for (int b = 0; b < 15; ++b) {
    i1 |= ((k >> (2 * b)) & 1) << b;
    i2 |= ((k >> (2 * b + 1)) & 1) << b;
  }
}

}  // namespace efie
