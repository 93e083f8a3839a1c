// Geometry phase (a1): NURBS evaluation at arbitrary parameter points, cluster bounding
// balls for the admissibility test (eq. admissibility) and the geometry at every cluster's
// tensor Chebyshev nodes (Sec. 4.2, "only q^2 evaluations of geometry" per cluster).
#include <cmath>

#include "geom.cuh"

namespace efie {

__global__ void k_eval_points(const PatchDesc *patches, const double *knots, const double4 *cpw, int npts,
                              const int *pid, const double *st, double *X, double *D) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts) return;
  double x[3], d1[3], d2[3];
  dev_patch_eval(patches[pid[i]], knots, cpw, st[2 * i], st[2 * i + 1], x, d1, d2);
  for (int k = 0; k < 3; ++k) X[3 * i + k] = x[k];
  if (D)
    for (int k = 0; k < 3; ++k) {
      D[6 * i + k] = d1[k];
      D[6 * i + 3 + k] = d2[k];
    }
}

efie_status dev_eval_points(Ctx *c, const std::vector<int> &patch, const std::vector<double> &st,
                            std::vector<double> &X, std::vector<double> *D) {
  int npts = (int)patch.size();
  X.assign(3 * (size_t)npts, 0.0);
  if (D) D->assign(6 * (size_t)npts, 0.0);
  if (npts == 0) return EFIE_OK;
  int *d_pid = nullptr;
  double *d_st = nullptr, *d_X = nullptr, *d_D = nullptr;
  EFIE_TRY(dalloc(c, &d_pid, npts));
  EFIE_TRY(dalloc(c, &d_st, 2 * (size_t)npts));
  EFIE_TRY(dalloc(c, &d_X, 3 * (size_t)npts));
  if (D) EFIE_TRY(dalloc(c, &d_D, 6 * (size_t)npts));
  EFIE_CUDA(cudaMemcpyAsync(d_pid, patch.data(), 4 * (size_t)npts, cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(d_st, st.data(), 16 * (size_t)npts, cudaMemcpyHostToDevice, c->stream));
  k_eval_points<<<(npts + 127) / 128, 128, 0, c->stream>>>(c->d_patches, c->d_knots, c->d_cpw, npts, d_pid, d_st,
                                                          d_X, d_D); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_CUDA(cudaMemcpyAsync(X.data(), d_X, 24 * (size_t)npts, cudaMemcpyDeviceToHost, c->stream));
  if (D) EFIE_CUDA(cudaMemcpyAsync(D->data(), d_D, 48 * (size_t)npts, cudaMemcpyDeviceToHost, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  dfree(c, d_pid);
  dfree(c, d_st);
  dfree(c, d_X);
  dfree(c, d_D);
  return EFIE_OK;
}

// cluster id -> (level, patch, k1, k2)
__device__ inline void decode_cluster(const int *lev_off, int nlev, int id, int &l, int &j, int &k1, int &k2) {
  l = 0;
  while (l + 1 < nlev && id >= lev_off[l + 1]) ++l;
  int r = id - lev_off[l];
  j = r >> (2 * l);
  int K = r & ((1 << (2 * l)) - 1);
  k1 = 0;
  k2 = 0;
  for (int b = 0; b < l; ++b) {
    k1 |= ((K >> (2 * b)) & 1) << b;
    k2 |= ((K >> (2 * b + 1)) & 1) << b;
  }
}

// Bounding ball of every cluster: centre F(box centre), radius = largest distance of a
// 9 x 9 parameter grid (corners included) from the centre.  One block per cluster.
__global__ void k_cluster_balls(const PatchDesc *patches, const double *knots, const double4 *cpw,
                                const int *lev_off, int nlev, int ncl, double *ball) {
  int id = blockIdx.x;
  if (id >= ncl) return;
  int l, j, k1, k2;
  decode_cluster(lev_off, nlev, id, l, j, k1, k2);
  double hl = 1.0 / (double)(1 << l);
  __shared__ double cen[3];
  __shared__ double red[128];
  double d1[3], d2[3];
  if (threadIdx.x == 0) {
    double X[3];
    dev_patch_eval(patches[j], knots, cpw, (k1 + 0.5) * hl, (k2 + 0.5) * hl, X, d1, d2);
    cen[0] = X[0];
    cen[1] = X[1];
    cen[2] = X[2];
  }
  __syncthreads();
  double r = 0.0;
  for (int t = threadIdx.x; t < 81; t += blockDim.x) {
    int a = t % 9, b = t / 9;
    double X[3];
    dev_patch_eval(patches[j], knots, cpw, (k1 + a / 8.0) * hl, (k2 + b / 8.0) * hl, X, d1, d2);
    double dx = X[0] - cen[0], dy = X[1] - cen[1], dz = X[2] - cen[2];
    r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
  }
  red[threadIdx.x] = r;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ball[4 * id + 0] = cen[0];
    ball[4 * id + 1] = cen[1];
    ball[4 * id + 2] = cen[2];
    ball[4 * id + 3] = red[0];
  }
}

// F, d1F, d2F at the (q+1)^2 tensor Chebyshev nodes of every cluster; also the node offsets
// from the cluster centre in FP32 for the mixed-precision M2L.
__global__ void k_node_geometry(const PatchDesc *patches, const double *knots, const double4 *cpw,
                                const int *lev_off, int nlev, int ncl, int q1, const double *xcheb,
                                const double *ball, double *nodeX, double *nodeD, float *nodeXf) {
  int nI = q1 * q1;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ncl * nI) return;
  int id = (int)(t / nI), mi = (int)(t % nI);
  int l, j, k1, k2;
  decode_cluster(lev_off, nlev, id, l, j, k1, k2);
  double hl = 1.0 / (double)(1 << l);
  double X[3], D1[3], D2[3];
  dev_patch_eval(patches[j], knots, cpw, (k1 + xcheb[mi % q1]) * hl, (k2 + xcheb[mi / q1]) * hl, X, D1, D2);
  for (int k = 0; k < 3; ++k) {
    nodeX[3 * t + k] = X[k];
    nodeD[6 * t + k] = D1[k];
    nodeD[6 * t + 3 + k] = D2[k];
    nodeXf[3 * t + k] = (float)(X[k] - ball[4 * id + k]);
  }
}

efie_status dev_cluster_geometry(Ctx *c) {
  int *d_lev = nullptr;
  double *d_ball = nullptr, *d_x = nullptr;
  int nlev = c->m + 1;
  EFIE_TRY(dalloc(c, &d_lev, c->lev_off.size()));
  EFIE_TRY(dalloc(c, &d_ball, 4 * (size_t)c->ncl));
  EFIE_TRY(dalloc(c, &d_x, c->q1));
  EFIE_CUDA(cudaMemcpyAsync(d_lev, c->lev_off.data(), 4 * c->lev_off.size(), cudaMemcpyHostToDevice, c->stream));
  EFIE_CUDA(cudaMemcpyAsync(d_x, c->tab.xcheb.data(), 8 * (size_t)c->q1, cudaMemcpyHostToDevice, c->stream));
  k_cluster_balls<<<c->ncl, 128, 0, c->stream>>>(c->d_patches, c->d_knots, c->d_cpw, d_lev, nlev, c->ncl, d_ball); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  c->ball.assign(4 * (size_t)c->ncl, 0.0);
  EFIE_CUDA(cudaMemcpyAsync(c->ball.data(), d_ball, 32 * (size_t)c->ncl, cudaMemcpyDeviceToHost, c->stream));
  EFIE_TRY(dalloc(c, &c->d_nodeX, 3 * (size_t)c->ncl * c->nI));
  EFIE_TRY(dalloc(c, &c->d_nodeD, 6 * (size_t)c->ncl * c->nI));
  EFIE_TRY(dalloc(c, &c->d_nodeXf, 3 * (size_t)c->ncl * c->nI));
  EFIE_TRY(dalloc(c, &c->d_center, 4 * (size_t)c->ncl));
  long long tot = (long long)c->ncl * c->nI;
  k_node_geometry<<<(unsigned)((tot + 127) / 128), 128, 0, c->stream>>>(c->d_patches, c->d_knots, c->d_cpw, d_lev,
                                                                      nlev, c->ncl, c->q1, d_x, d_ball, c->d_nodeX,
                                                                      c->d_nodeD, c->d_nodeXf); ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_CUDA(cudaMemcpyAsync(c->d_center, d_ball, 32 * (size_t)c->ncl, cudaMemcpyDeviceToDevice, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  dfree(c, d_lev);
  dfree(c, d_ball);
  dfree(c, d_x);
  return EFIE_OK;
}

}  // namespace efie
