/* efie.h -- C ABI of the GB300 isogeometric EFIE library.
 *
 * The library solves the electric field integral equation for perfectly conducting
 * scatterers bounded by multipatch NURBS surfaces (Doelz, Kurz, Schoeps, Wolf,
 * "Isogeometric Boundary Elements in Electromagnetism", arXiv 1807.03097):
 *
 *   find w_h in S^1 (div-conforming B-splines, Sec. 3.2) such that
 *   V_{kappa,h} w_h = -f_h                                   (eq. linsys)
 *
 * with the Galerkin matrix of eq. MSLtested applied through the superspace
 * transformation T^T V* T (eq. superspace) and the interpolation-based H^2 / fast multipole
 * compression of Sec. 4.2 (eq. FMMlr, Algorithm 1), inside a restarted GMRES (Sec. 5).
 * Every numerical step runs in CUDA kernels on one GPU; host code only builds index
 * structures (DOF map, cluster tree, block-cluster tree).
 *
 * Conventions
 *  - All functions return efie_status: 0 on success, > 0 for a completed call with a
 *    warning (EFIE_NOT_CONVERGED), < 0 on error.  No C++ exception crosses the ABI.
 *  - Complex numbers are interleaved (re, im) doubles; a vector of n complex values is
 *    2n doubles.  Several right-hand sides are stored one after the other ([nrhs][n]).
 *  - ptr_kind EFIE_PTR_HOST: pointers are host memory (pageable or pinned); the call
 *    copies in and out and returns after the result is in host memory.
 *    EFIE_PTR_DEVICE: pointers are device memory of the context's GPU; the call is ordered
 *    on the context's stream and returns once the result is complete on the device.
 *  - The caller owns every buffer it passes; the library deep-copies inputs and never
 *    keeps a caller pointer beyond the call.
 *  - DOF order: patch-major, then component (s1 then s2), then B-spline index i2, i1 (i1
 *    fastest); a function shared by two patches across an interface is numbered where it
 *    first occurs, and its part on the other patch carries the sign that keeps the normal
 *    flux continuous.
 *  - Thread safety: one context per host thread; contexts are independent.
 */
#ifndef EFIE_H
#define EFIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int efie_status;
#define EFIE_OK 0
#define EFIE_NOT_CONVERGED 1  /* GMRES reached gmres_maxit; output holds the last iterate */
#define EFIE_PENDING 2        /* efie_server_poll: the request has not finished yet */
#define EFIE_EINVAL -1        /* invalid argument (null pointer, size or option out of range) */
#define EFIE_ENOMEM -2        /* device or host allocation failed */
#define EFIE_EGEOMETRY -3     /* open, non-manifold, inward-oriented or mismatched patches */
#define EFIE_ECUDA -4         /* a CUDA call failed; the context should be destroyed */
#define EFIE_ESTATE -5        /* call out of order (e.g. matvec before efie_setup) */
#define EFIE_ETIMEOUT -6      /* a device-side wait gave up (status word set by a kernel) */

#define EFIE_FP64 0           /* every step in FP64 */
#define EFIE_MIXED_FP32 1     /* moments, M2M, M2L, L2L in FP32 (phase split, FP64 per-pair
                                 phase); the near-field blocks are integrated in FP64 and
                                 applied from an FP32 copy with compensated FP32 sums;
                                 geometry, right-hand side, far field and GMRES in FP64 */

#define EFIE_PTR_HOST 0
#define EFIE_PTR_DEVICE 1

typedef struct efie_ctx efie_ctx;

/* Discretisation and solver parameters (the paper's problem statement, Sec. 4.1, 4.2, 5). */
typedef struct {
  int p;             /* degree of S^0; S^1 uses (p, p-1) x (p-1, p), 1 <= p <= 4 (Sec. 3.2) */
  int level_m;       /* refinement level: 2^m equidistant elements per patch direction,
                        0 <= m <= 10 (Sec. 4.1) */
  double kappa;      /* wavenumber, > 0 (eq. HelmholtzGreen) */
  int q;             /* interpolation degree, q + 1 Chebyshev points per direction,
                        1 <= q <= 16 (Sec. 4.2) */
  double eta;        /* admissibility parameter, > 0 (eq. admissibility) */
  int precision;     /* EFIE_FP64 or EFIE_MIXED_FP32 */
  int quad_regular;  /* Gauss points per direction for separated near pairs, right-hand
                        side and far field; 0 selects p + 4 */
  int quad_singular; /* Gauss points per direction in each Duffy part of touching pairs;
                        0 selects p + 4 */
  int gmres_restart; /* restart length (the paper uses 1500), >= 1 */
  double gmres_tol;  /* residual tolerance */
  int gmres_maxit;   /* total iteration cap */
  int tol_is_relative; /* 1: ||r|| <= tol ||b||, 0: ||r|| <= tol */
  int m2l_store;     /* M2L coupling matrices: 0 automatic (FP64 form: kept in device memory
                        when they take at most half of the free memory; FP32 form: evaluated
                        in every product, which is faster than streaming them); 1 always
                        evaluate; 2 always keep (EFIE_ENOMEM if they do not fit) */
  int m2l_batch;     /* M2L of a product with several right-hand sides in the mixed form:
                        0 automatic (tensor cores when q <= 10, else FP32 on the CUDA cores),
                        1 FP32 on the CUDA cores, 2 tensor cores (split TF32 with FP32
                        accumulation, q <= 10; EFIE_EINVAL at setup otherwise) */
  int leaf_dense;    /* 0: the paper's block tree (Algorithm 1); 1: leaf-level variant, in which
                        an admissible pair of two elements is integrated as an element block
                        (tensor Gauss, quad_regular points) like a separated near pair instead of
                        being compressed, when (p+1)^2 < (q+1)^2.  A departure from the paper's
                        FMM (more accurate, more near-field storage, fewer M2L blocks). */
  int m2l_pairs;     /* M2L of one right-hand side in the mixed form: 0 every ordered admissible
                        pair (t, s) evaluates its coupling tile; 1 every unordered pair {t, s}
                        evaluates it once and applies it in both directions (K_st = K_ts^T),
                        with npairs x (q+1)^2 x 32 bytes of column sums (used when they fit in a
                        quarter of the free memory); 2 autotuned: setup times both kernels on
                        this problem's blocks (CUDA events, best of 3) and keeps the faster
                        (efie_setup_timings reports both times and the choice).  A variant of
                        the M2L's cost, same results within the mixed tolerance. */
} efie_options;

typedef struct {
  int iterations;        /* GMRES iterations (matrix-vector products) of the last solve */
  int converged;         /* 1 if the tolerance was met */
  double residual;       /* final ||b - A x|| (relative if tol_is_relative) */
  double setup_ms;       /* device time of efie_setup */
  double solve_ms;       /* wall time of the last solve on the device */
} efie_solve_info;

/* Fills *opt with defaults: p=1, m=2, kappa=1, q=4, eta=1.6, FP64, restart 1500,
 * tol 1e-8 relative, maxit 10000. */
efie_status efie_default_options(efie_options *opt);

/* Creates a context on the current CUDA device.  cuda_stream: a cudaStream_t to order
 * all work on, or NULL for a stream the context creates.  Errors: EFIE_EINVAL (bad
 * options), EFIE_ENOMEM, EFIE_ECUDA (no device). */
efie_status efie_create(efie_ctx **out, const efie_options *opt, void *cuda_stream);

/* Sets the geometry: n_patches NURBS patches F_j: [0,1]^2 -> R^3 (eq. def::geom).
 *  deg   [n][2]  degrees in s1 and s2 (>= 1)
 *  ncp   [n][2]  control points in s1 and s2 (<= 64 each)
 *  knots         per patch the s1 knot vector (ncp0 + deg0 + 1 values) followed by the s2
 *                knot vector, p-open on [0,1]
 *  cp            per patch [ncp1][ncp0][3] control points (s1 fastest)
 *  w             per patch [ncp1][ncp0] positive weights
 * Host pointers, deep-copied.  Interfaces are detected by matching patch edges (Sec. 3.1:
 * F_j(.,1) = F_i(.,0) up to orientation).  Errors: EFIE_EINVAL, EFIE_EGEOMETRY (an edge
 * without exactly one partner, or d1F x d2F not pointing out of the enclosed volume). */
efie_status efie_set_geometry(efie_ctx *ctx, int n_patches, const int *deg, const int *ncp,
                              const double *knots, const double *cp, const double *w);

/* Builds the discrete space and T (eq. superspace), cluster tree and block-cluster tree
 * (Algorithm 1), evaluates the geometry at the interpolation nodes and computes every
 * near-field element block by Sauter-Schwab / Gauss quadrature (eq. Vkh), all resident on
 * the device.  Errors: EFIE_ESTATE (no geometry), EFIE_EGEOMETRY, EFIE_ENOMEM, EFIE_ECUDA. */
efie_status efie_setup(efie_ctx *ctx);

/* Number of complex unknowns 2 N (n + p - 1)^2 of a closed surface. */
efie_status efie_num_dofs(const efie_ctx *ctx, int64_t *n);

/* y = T^T (N + F) T x for nrhs vectors of efie_num_dofs complex values each (the FMM
 * approximation of the Galerkin matrix of eq. MSLtested).  Errors: EFIE_ESTATE,
 * EFIE_EINVAL, EFIE_ECUDA. */
efie_status efie_matvec(efie_ctx *ctx, int nrhs, const double *x, double *y, int ptr_kind);

/* Right-hand side of eq. linsys for incident plane waves e_i = pol exp(i kappa dir.x):
 * g_j = -int_Gamma e_i . phi_j dsigma.  dir, pol: [nrhs][3] host arrays; g [nrhs][ndof]
 * complex in ptr_kind memory. */
efie_status efie_rhs_plane_waves(efie_ctx *ctx, int nrhs, const double *dir, const double *pol,
                                 double *g, int ptr_kind);

/* Solves A x = b by restarted GMRES (zero initial guess) for nrhs right-hand sides: one after
 * the other in the FP64 form; in the mixed form (nrhs > 1) in lockstep, with one batched
 * product of all unfinished systems per iteration.  Returns EFIE_NOT_CONVERGED (with the last
 * iterate in x) if some right-hand side reached gmres_maxit.  info may be NULL. */
efie_status efie_solve(efie_ctx *ctx, int nrhs, const double *b, double *x, int ptr_kind,
                       efie_solve_info *info);

/* Right-hand side plus solve: the scattering problem for incident plane waves. */
efie_status efie_solve_plane_waves(efie_ctx *ctx, int nrhs, const double *dir, const double *pol,
                                   double *w, int ptr_kind, efie_solve_info *info);

/* Far field of the scattered wave, e_s(r d) ~ E_inf(d) e^{i kappa r} / r, from the
 * representation formula (eq. ESLP): E_inf(d) = (1/4pi) (W - d (d.W)),
 * W = int_Gamma w(y) exp(-i kappa d.y) dsigma_y.  w: [nrhs][ndof] complex, dirs: [ndir][3]
 * unit vectors (host), e_inf: [nrhs][ndir][3] complex; w and e_inf in ptr_kind memory. */
efie_status efie_far_field(efie_ctx *ctx, int nrhs, const double *w, int ndir, const double *dirs,
                           double *e_inf, int ptr_kind);

/* Scattered electric field at points off the surface by the electric single-layer potential
 * (eq. ESLP): E(x) = int G w dsigma + kappa^-2 grad_x int G div_Gamma w dsigma.  w: [nrhs][ndof]
 * complex; pts: [npts][3] host array (1 <= npts <= 65535), points well separated from the
 * surface (tensor Gauss rule of quad_regular points per element direction, not adapted to near
 * points); e_out: [nrhs][npts][3] complex; w and e_out in ptr_kind memory. */
efie_status efie_exterior_field(efie_ctx *ctx, int nrhs, const double *w, int npts, const double *pts,
                                double *e_out, int ptr_kind);

/* Right-hand side of the manufactured solution of Sec. 5.2: incident field e_i = -DP, DP the
 * Hertz dipole at x0 with moment p0 (x0 inside the scatterer), so that the scattered field
 * outside is DP itself: g_j = +int_Gamma DP . phi_j dsigma.  x0, p0: [nrhs][3] host arrays;
 * g [nrhs][ndof] complex in ptr_kind memory. */
efie_status efie_rhs_dipole(efie_ctx *ctx, int nrhs, const double *x0, const double *p0, double *g,
                            int ptr_kind);

/* Introspection for verification.
 * efie_block_counts: far blocks, near element pairs, clusters, superspace size.
 * efie_export_blocks: far [nfar][3] = (level, target cluster, source cluster) and near
 *   [nnear][2] = (target element, source element), host memory; cluster ids are
 *   level offset + patch * 4^level + morton index, element ids patch * 4^m + morton index.
 * efie_export_near_blocks: near-field element blocks [nnear][nb][nb] complex (host),
 *   nb = 2 (p+1)^2, rows (alpha, b, a) of the target element, columns of the source.
 * efie_matvec_superspace: ys = (N + F) xs on superspace vectors [nE][2][p+1][p+1]
 *   complex (ptr_kind memory). */
efie_status efie_block_counts(const efie_ctx *ctx, int64_t *nfar, int64_t *nnear, int64_t *nclusters,
                              int64_t *nsuperspace);
efie_status efie_export_blocks(const efie_ctx *ctx, int *far, int *near);
efie_status efie_export_near_blocks(efie_ctx *ctx, double *blocks);
efie_status efie_matvec_superspace(efie_ctx *ctx, const double *xs, double *ys, int ptr_kind);
/* ys = N xs: the near-field part of the product alone (the element blocks of eq. Vkh of the
 * non-admissible leaf pairs, Sec. 4.1; FP32 blocks in the mixed form), on one superspace vector
 * (ptr_kind memory).  Its device time is reported by efie_last_timings (total and near field).
 * Errors: EFIE_ESTATE, EFIE_EINVAL, EFIE_ECUDA. */
efie_status efie_near_apply(efie_ctx *ctx, const double *xs, double *ys, int ptr_kind);
/* ys[r] = (N + F) xs[r] for nrhs superspace vectors, [nrhs][nE][2][p+1][p+1] complex in
 * ptr_kind memory: the product of several right-hand sides (eq. FMMlr) without the T gather
 * and scatter, in one batched pass per 64 vectors in the mixed form (the M2L chosen by
 * m2l_batch), one vector after the other in the FP64 form. */
efie_status efie_matvec_superspace_batch(efie_ctx *ctx, int nrhs, const double *xs, double *ys, int ptr_kind);

/* Device time in milliseconds of the named phases of the most recent efie_matvec
 * (CUDA events on the context stream): out[0] total, [1] gather, [2] near apply,
 * [3] moments + M2M, [4] M2L, [5] L2L + evaluation, [6] scatter.  Returns the number of
 * values written (<= n). */
int efie_last_timings(const efie_ctx *ctx, double *out, int n);

/* Figures of the last efie_setup: out[0] wall time of the setup (ms), [1] device time of the
 * near-field quadrature of touching element pairs (Sauter-Schwab kernel, ms, CUDA events on
 * the context stream), [2] quadrature points it evaluated (Duffy parts x g^4 summed over its
 * pairs), [3] touching pairs it integrated, [4] device time of the separated pairs (tensor
 * Gauss from element tables, ms), [5] separated pairs integrated; pairs (e', e) with e' > e
 * are mirrored, B(e', e) = B(e, e')^T; [6] M2L time of the ordered-pair kernel, [7] of the
 * unordered-pair kernel (ms, when m2l_pairs = 2 timed them, else 0), [8] the M2L kept (0
 * ordered pairs, 1 unordered pairs).  Returns the number of values written (<= n). */
int efie_setup_timings(const efie_ctx *ctx, double *out, int n);

/* Far field like efie_far_field, for callers that must not allocate device memory during
 * the call (a process running under a fixed device-memory budget owned by another
 * allocator, or one that cannot afford cudaMalloc / cudaFree synchronising the device while
 * its other work is in flight).  The paper has no counterpart; this is a library service.
 *  w_dev      [ndof] complex, device memory (one right-hand side)
 *  dirs_dev   [ndir][3] unit directions, device memory
 *  e_inf_dev  [ndir][3] complex output, device memory
 * Nothing is allocated: the T gather is fused into the kernel and the partial sums use one
 * file-scope device array of 2^18 complex doubles (4 MiB) that every GPU loading the library
 * holds until the process exits.  Limits: 3 * ndir * ceil(elements / 16) <= 2^18 and
 * ndir <= 65535, else EFIE_EINVAL.  The caller's current CUDA device is unchanged on return.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  All calls on a device share the array and each call rewrites the part it uses
 * in full; calls that overlap on the GPU (other streams or other contexts on the same
 * device) race on it.  Ordered on the context stream; returns when the result is complete. */
efie_status efie_far_field_noalloc(efie_ctx *ctx, const double *w_dev, int ndir, const double *dirs_dev,
                                   double *e_inf_dev);

/* Number of CUDA kernels this context has launched since efie_create (all phases);
 * -1 for a NULL context. */
int64_t efie_launch_count(const efie_ctx *ctx);

/* Device memory of the context: *live = bytes held now, *peak = the most held at any time
 * since efie_create (both may be NULL).  Device buffers come from one stream-ordered memory
 * pool per device (allocated and freed on the context's stream, so that no call of one
 * context synchronises the device or waits for another context).  The paper has no
 * counterpart; this is for admission control and tests.  EFIE_EINVAL for a NULL ctx. */
efie_status efie_device_bytes(const efie_ctx *ctx, int64_t *live, int64_t *peak);

/* Releases all device and host memory of the context (NULL is accepted). */
efie_status efie_destroy(efie_ctx *ctx);

/* ---------------------------------------------------------------------------------------
 * Serving: a request loop that admits scattering solves of different geometries, sizes and
 * wavenumbers while others run.  Requests wait in a queue; whenever a slot is free, among the
 * 8 oldest queued requests whose estimated device-memory footprint (near-field blocks, Krylov
 * bases, cluster data) fits the remaining budget, the one with the least estimated work
 * (directions x DOFs x local basis size x interpolation nodes) is admitted; so small requests
 * may pass larger ones, the oldest request goes first once 8 admissions have passed it, and a
 * request larger than the whole budget runs alone.
 * Each admitted request runs the ordinary per-context path (efie_create, set_geometry,
 * setup, solve_plane_waves, far_field) on its own worker thread and CUDA stream, so the
 * work of several requests overlaps on the GPU.  Results do not depend on what else runs:
 * every reduction has a fixed order. */
typedef struct efie_server efie_server;

typedef struct {
  int n_patches;           /* geometry as in efie_set_geometry (host, deep-copied at submit) */
  const int *deg, *ncp;
  const double *knots, *cp, *w;
  efie_options opt;        /* discretisation and solver options of this request */
  int nrhs;                /* incident plane waves */
  const double *dir, *pol; /* [nrhs][3] */
  int ndir;                /* far-field directions (0: none) */
  const double *ff_dirs;   /* [ndir][3] */
  double *w_out;           /* [nrhs][2 N (2^m + p - 1)^2] complex, caller-owned; must stay valid
                              until efie_server_poll has returned EFIE_OK for this ticket */
  double *e_inf_out;       /* [nrhs][ndir][3] complex, caller-owned (ndir > 0) */
} efie_request;

typedef struct {
  efie_status status;      /* status of the solve (EFIE_OK, EFIE_NOT_CONVERGED or an error) */
  int iterations;          /* largest GMRES iteration count over the request's waves */
  double residual;
  int64_t ndof;
  double queue_ms;         /* submit -> admitted */
  double latency_ms;       /* submit -> result in the caller's buffers */
  double setup_ms, solve_ms;
  int64_t footprint_bytes;   /* the admission's device-memory estimate of the request */
  int64_t device_peak_bytes; /* device memory the request's context held at its peak */
} efie_result;

/* Starts max_slots worker threads on the current CUDA device with a device-memory budget in
 * bytes.  Errors: EFIE_EINVAL (max_slots outside 1..64, zero budget), EFIE_ECUDA. */
efie_status efie_server_create(efie_server **out, size_t hbm_budget_bytes, int max_slots);
/* Queues a request (non-blocking) and returns its ticket.  Errors: EFIE_EINVAL. */
efie_status efie_server_submit(efie_server *srv, const efie_request *req, uint64_t *ticket);
/* EFIE_PENDING while the request is queued or running; EFIE_OK once its outputs are in the
 * caller's buffers, with *res filled (the ticket is then released); EFIE_EINVAL for an
 * unknown ticket. */
efie_status efie_server_poll(efie_server *srv, uint64_t ticket, efie_result *res);
/* Waits for every queued and running request, then stops the workers. */
efie_status efie_server_destroy(efie_server *srv);

/* Failure-detection check of the device-side waits (the mbarrier waits of the tensor-core M2L,
 * which give up after about 2^31 clock cycles and report EFIE_ETIMEOUT for the product).  Runs
 * one such wait, limited to `cycles` clocks (1 .. 2^32), on a barrier that nothing completes, so
 * the expected result is EFIE_ETIMEOUT with the detail in efie_last_error; the context stays
 * usable.  EFIE_EINVAL for a NULL ctx or cycles out of range.  The paper has no counterpart. */
efie_status efie_check_device_waits(efie_ctx *ctx, long long cycles);

/* Static description of a status code. */
const char *efie_status_string(efie_status s);
/* Detail of the last failed call on ctx (the failing CUDA call and its error string, or the
 * reason for EFIE_EINVAL / EFIE_ETIMEOUT); "" if none.  Owned by ctx, valid until the next
 * call on ctx. */
const char *efie_last_error(const efie_ctx *ctx);

/* ---------------------------------------------------------------------------------------
 * Groups of independent problems (restarted GMRES of Sec. 5 across problems).
 *
 * efie_setup_many runs efie_setup of nctx contexts on nthreads host threads (each context's
 * device work on its own stream, so the setups overlap on the GPU); status[i] (optional,
 * nctx entries) receives each context's status; the return value is the first error, else
 * EFIE_OK.
 *
 * A group holds nctx contexts that are set up on one device (each with its own geometry,
 * wavenumber, p, refinement and options).  efie_group_solve solves A_i x_i = b_i for every
 * context i in lockstep: each step is one CUDA-graph launch that holds the products of all
 * unfinished systems (one branch per context; the graph is captured again only when a tenth of
 * its branches belong to finished systems) and the Arnoldi (CGS2), Givens and update work of
 * all systems, one kernel per operation, with the arithmetic of efie_solve.  The
 * GMRES options (tolerance, restart, maximum iterations) are each context's own.
 *   b[i], x[i]: 2 ndof_i doubles each (ptr_kind memory); x[i] receives the solution.
 *   iterations, residuals, converged: nctx entries each (optional).
 * While a group solve runs, its contexts must not be used by other calls.  The contexts
 * stay owned by the caller and must outlive the group.
 * Returns EFIE_NOT_CONVERGED if any system did not converge; EFIE_ESTATE if a context is
 * not set up (or, at solve time, was set up again with another number of DOFs since the group
 * was made); EFIE_EINVAL for null pointers, repeated or mixed-device contexts.
 * efie_group_stats: [steps, product-graph captures, kernels launched (graph nodes counted),
 * solve wall time ms, kernel nodes of the product graph, vector chunks, device ms of the pre,
 * product and post graphs summed over the steps (CUDA events on the group's stream)] of the
 * last solve; returns the number of values written. */
typedef struct efie_group efie_group;
efie_status efie_setup_many(efie_ctx *const *ctxs, int nctx, int nthreads, efie_status *status);
efie_status efie_group_create(efie_group **g, efie_ctx *const *ctxs, int nctx);
efie_status efie_group_solve(efie_group *g, const double *const *b, double *const *x, int ptr_kind,
                             int *iterations, double *residuals, int *converged);
int efie_group_stats(const efie_group *g, double *out, int n);
const char *efie_group_last_error(const efie_group *g);
efie_status efie_group_destroy(efie_group *g);

#ifdef __cplusplus
}
#endif
#endif
