/* Oracle for the isogeometric EFIE with interpolation-based FMM (Doelz, Kurz, Schoeps,
 * Wolf, "Isogeometric Boundary Elements in Electromagnetism", arXiv 1807.03097).
 *
 * TEST INFRASTRUCTURE ONLY.  A plain, slow, serial FP64 CPU implementation of what the
 * library computes, written from the paper's equations.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no code with the
 * CUDA library.
 *
 * Conventions (the same ones the library follows, each implemented independently):
 *  - patch parameter s = (s1, s2) in [0,1]^2; control net [ncp1][ncp0], s1 index fastest;
 *  - n = 2^m elements per direction per patch; element e = patch*n*n + morton(i1, i2)
 *    with the bits of i1 in the even positions;
 *  - superspace coefficient index ((e*2 + alpha)*(p+1) + b)*(p+1) + a, alpha = component
 *    (0: s1, 1: s2), a / b = Bernstein indices in s1 / s2 on the element;
 *  - global DOFs: patch-major, component, i2, i1; an interface function is numbered at its
 *    first occurrence; its partner on the neighbouring patch carries the sign
 *    -sigma(edge)*sigma(edge') with sigma = -1 on the s=0 edges and +1 on the s=1 edges;
 *  - complex vectors are interleaved (re, im) doubles.
 */
#ifndef EFIE_ORACLE_H
#define EFIE_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_problem orc_problem;

/* Builds geometry, discrete space, transformation T, cluster tree and block-cluster tree.
 * deg/ncp: [np][2]; knots: per patch k0 then k1 concatenated; cp: [..][3]; w: [..].
 * Returns NULL on allocation failure; geometry errors are reported by orc_status(). */
orc_problem *orc_create(int np, const int *deg, const int *ncp, const double *knots,
                        const double *cp, const double *w, int p, int m, double kappa,
                        int q, double eta, int g_reg, int g_sing);
/* As orc_create, with the leaf-level variant of Algorithm 1 when leaf_dense = 1: admissible
 * pairs of two leaves are integrated as element blocks (tensor Gauss) instead of compressed. */
orc_problem *orc_create_variant(int np, const int *deg, const int *ncp, const double *knots,
                                const double *cp, const double *w, int p, int m, double kappa,
                                int q, double eta, int g_reg, int g_sing, int leaf_dense);
void orc_destroy(orc_problem *P);
int orc_status(const orc_problem *P, char *msg, int msglen);

int orc_num_dofs(const orc_problem *P);
int orc_num_elements(const orc_problem *P);
int orc_superspace_size(const orc_problem *P);
int orc_num_clusters(const orc_problem *P);

/* geometry: F, d1F, d2F at npts parameter points of one patch */
void orc_eval_patch(const orc_problem *P, int patch, int npts, const double *s, double *x,
                    double *d1, double *d2);

/* T as COO (superspace row, global column, value); returns nnz, fills up to cap */
int orc_T_coo(const orc_problem *P, int cap, int *row, int *col, double *val);

/* cluster bounding balls [ncl][4] = (cx, cy, cz, r) */
void orc_cluster_balls(const orc_problem *P, double *out);
/* block lists: far pairs [nfar][3] = (level, target id, source id), near [nnear][2] = (e, e') */
int orc_num_far(const orc_problem *P);
int orc_num_near(const orc_problem *P);
void orc_far_pairs(const orc_problem *P, int *out);
void orc_near_pairs(const orc_problem *P, int *out);

/* near-field element blocks [nnear][2(p+1)^2][2(p+1)^2] complex */
void orc_near_blocks(orc_problem *P, double *out);
/* one element-pair block with explicit quadrature orders (g_reg for separated pairs,
 * g_sing for touching pairs); out [2(p+1)^2][2(p+1)^2] complex */
void orc_pair_block(const orc_problem *P, int e, int e2, int g_reg, int g_sing, double *out);
/* scalar test integral int_e int_e2 G dsigma dsigma (surface measure included) */
void orc_pair_scalar(const orc_problem *P, int e, int e2, int g_reg, int g_sing, double kappa,
                     double *out2);
/* classification of an element pair: 0 separated, 1 vertex, 2 edge, 3 identical; -1 invalid */
int orc_pair_kind(const orc_problem *P, int e, int e2);

/* dense superspace matrix V* [S][S] complex (small problems only) */
void orc_dense_superspace(const orc_problem *P, double *out);
/* y = T^T V* T x with V* dense, nrhs vectors of length ndof */
void orc_dense_matvec(const orc_problem *P, int nrhs, const double *x, double *y);
/* y = T^T (N + F) T x through the non-nested interpolation FMM */
void orc_fmm_matvec(orc_problem *P, int nrhs, const double *x, double *y);
/* y* = (N + F) x* on superspace vectors [nE][2][p+1][p+1] complex */
void orc_fmm_matvec_superspace(orc_problem *P, const double *xs, double *ys);
/* the rows of y* = (N + F) x* belonging to the listed elements, out [nrows][2(p+1)^2]
 * (near blocks integrated on demand; for sampled checks and timing at large sizes) */
void orc_fmm_rows(orc_problem *P, const double *xs, int nrows, const int *elems, double *out);
/* the far-field part of those rows only (no near blocks): for timing the far field */
void orc_fmm_rows_far(orc_problem *P, const double *xs, int nrows, const int *elems, double *out);

/* right-hand side g = -T^T int e_i . phi for e_i = pol exp(i kappa d.x) */
void orc_rhs(const orc_problem *P, const double *dir, const double *pol, double *g);
/* restarted GMRES (MGS), zero initial guess; use_fmm selects FMM or dense operator;
 * returns 0 if converged */
int orc_gmres(orc_problem *P, int use_fmm, const double *b, double *x, int restart, double tol,
              int maxit, int *its, double *relres);
/* far field E_inf(d) = (1/4pi) (d x W) x d for ndir directions: out [ndir][3] complex */
void orc_far_field(const orc_problem *P, const double *coef, int ndir, const double *dirs,
                   double *out);
/* Hertz dipole field DP_{x0,p0} (Sec. 5.2) at npts points: out [npts][3] complex */
void orc_dipole_field(double kappa, const double *x0, const double *p0, int npts, const double *x, double *out);
/* right-hand side for e_i = -DP_{x0,p0} (scattered field = DP outside; manufactured solution) */
void orc_rhs_dipole(const orc_problem *P, const double *x0, const double *p0, double *g);
/* electric single-layer potential (eq. ESLP) of the field with global coefficients coef at
 * npts points off the surface: out [npts][3] complex */
void orc_exterior_field(const orc_problem *P, const double *coef, int npts, const double *x, double *out);
/* integral of the surface divergence of the field with global coefficients coef */
void orc_div_integral(const orc_problem *P, const double *coef, double *out2);
/* surface area (integral of tau) */
double orc_area(const orc_problem *P);
/* L2 error against the Mie current of a sphere (centre 0, radius a) for an x-polarised
 * plane wave travelling along +z: out[0] = ||w_h - w||, out[1] = ||w|| */
void orc_mie_l2(const orc_problem *P, const double *coef, double radius, double *out);

/* Mie series (PEC sphere, radius a, incident x exp(i kappa z)), at arbitrary points:
 * which = 0: incident E, 1: scattered E, 2: curl E_total, 3: surface current n x curl E_tot,
 * 4: far-field amplitude F(x/|x|) of the scattered field, e_s ~ F e^{i kappa r} / r */
void orc_mie_field(double kappa, double radius, int which, int npts, const double *x,
                   double *out);

/* 1-D tables used by tests: Gauss-Legendre on [0,1], Chebyshev nodes */
void orc_gauss01(int g, double *x, double *w);
void orc_cheb01(int q, double *x);

#ifdef __cplusplus
}
#endif
#endif
