// Far field without any device allocation during the call (efie_far_field_noalloc).
//
// For callers that must not allocate device memory while they call the library: for example
// a host process that runs under a fixed device-memory budget owned by another allocator,
// or a caller that cannot afford cudaMalloc/cudaFree, which may synchronise the whole
// device and stall the other work it has in flight.  The result is the same far field as
// efie_far_field; the differences are that every pointer is device memory supplied by the
// caller, the superspace coefficients are gathered inside the kernel, and the partial sums
// live in one file-scope device array of fixed size instead of a buffer allocated per call.
#include <cmath>
#include <mutex>

#include "geom.cuh"

namespace efie {

// Scratch for the partial sums: 2^18 complex doubles (4 MiB).  Every GPU that loads the
// library holds it until the process exits.  All calls on a device share it.
constexpr size_t kFFScratchElems = size_t(1) << 18;
static __device__ __align__(256) double2 g_ff_scratch[kFFScratchElems];

constexpr int kFFChunk = 16;  // elements summed by one block
constexpr int kMaxRule = 16;

struct FFRule {
  double x[kMaxRule], w[kMaxRule];
};

// One block per (chunk of kFFChunk elements, direction), one thread per Gauss point; the
// element's superspace coefficients x* = T w are gathered from the caller's DOF vector.
__global__ void k_ff_partial_noalloc(const PatchDesc *patches, const double *knots, const double4 *cpw, int n, int p,
                                     int g, FFRule rule, double kappa, int nE, int nchunk, const double *dirs,
                                     const int *__restrict__ tptr, const int *__restrict__ tcol,
                                     const double *__restrict__ tval, const double2 *__restrict__ w,
                                     double2 *part) {
  const int chunk = blockIdx.x, dd = blockIdx.y, t = threadIdx.x;
  const int P1 = p + 1, nloc = 2 * P1 * P1;
  __shared__ double2 xe[2 * kMaxP1 * kMaxP1];
  __shared__ double2 red[256][3];
  const double *d = dirs + 3 * dd;
  double2 W[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  const double h = 1.0 / n;
  for (int e = chunk * kFFChunk; e < min(nE, (chunk + 1) * kFFChunk); ++e) {
    __syncthreads();
    for (int r = t; r < nloc; r += blockDim.x) {
      const int row = e * nloc + r;
      double2 s = make_double2(0.0, 0.0);
      for (int k = tptr[row]; k < tptr[row + 1]; ++k) {
        double2 v = w[tcol[k]];
        s.x += tval[k] * v.x;
        s.y += tval[k] * v.y;
      }
      xe[r] = s;
    }
    __syncthreads();
    if (t < g * g) {
      const int n2 = n * n, j = e / n2, K = e % n2;
      int i1 = 0, i2 = 0;
      for (int b = 0; b < 15; ++b) {
        i1 |= ((K >> (2 * b)) & 1) << b;
        i2 |= ((K >> (2 * b + 1)) & 1) << b;
      }
      const double u = rule.x[t % g], v = rule.x[t / g];
      double X[3], D1[3], D2[3];
      dev_patch_eval(patches[j], knots, cpw, (i1 + u) * h, (i2 + v) * h, X, D1, D2);
      double sn, cs;
      sincos(-kappa * (d[0] * X[0] + d[1] * X[1] + d[2] * X[2]), &sn, &cs);
      const double wt = rule.w[t % g] * rule.w[t / g] * h * h;
      double Bu[kMaxP1], dBu[kMaxP1], Bv[kMaxP1], dBv[kMaxP1];
      dev_bernstein(p, u, Bu, dBu);
      dev_bernstein(p, v, Bv, dBv);
      double2 wa[2] = {make_double2(0, 0), make_double2(0, 0)};
      for (int al = 0; al < 2; ++al)
        for (int b = 0; b < P1; ++b)
          for (int a = 0; a < P1; ++a) {
            const double f = Bu[a] * Bv[b];
            const double2 cf = xe[(al * P1 + b) * P1 + a];
            wa[al].x += f * cf.x;
            wa[al].y += f * cf.y;
          }
      for (int k = 0; k < 3; ++k) {
        const double vx = D1[k] * wa[0].x + D2[k] * wa[1].x, vy = D1[k] * wa[0].y + D2[k] * wa[1].y;
        W[k].x += wt * (cs * vx - sn * vy);
        W[k].y += wt * (cs * vy + sn * vx);
      }
    }
  }
  for (int k = 0; k < 3; ++k) red[t][k] = W[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s)
      for (int k = 0; k < 3; ++k) {
        red[t][k].x += red[t + s][k].x;
        red[t][k].y += red[t + s][k].y;
      }
    __syncthreads();
  }
  if (t == 0)
    for (int k = 0; k < 3; ++k) part[((size_t)dd * nchunk + chunk) * 3 + k] = red[0][k];
}

// E_inf(d) = (W - d (d.W)) / (4 pi), W summed over the chunks in a fixed order.
__global__ void k_ff_final_noalloc(int nchunk, const double *dirs, const double2 *part, double2 *out) {
  const int dd = blockIdx.x, t = threadIdx.x;
  __shared__ double2 red[256][3];
  double2 W[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
  for (int c = t; c < nchunk; c += blockDim.x)
    for (int k = 0; k < 3; ++k) {
      W[k].x += part[((size_t)dd * nchunk + c) * 3 + k].x;
      W[k].y += part[((size_t)dd * nchunk + c) * 3 + k].y;
    }
  for (int k = 0; k < 3; ++k) red[t][k] = W[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s)
      for (int k = 0; k < 3; ++k) {
        red[t][k].x += red[t + s][k].x;
        red[t][k].y += red[t + s][k].y;
      }
    __syncthreads();
  }
  if (t == 0) {
    const double *d = dirs + 3 * dd;
    const double2 dw = make_double2(d[0] * red[0][0].x + d[1] * red[0][1].x + d[2] * red[0][2].x,
                                    d[0] * red[0][0].y + d[1] * red[0][1].y + d[2] * red[0][2].y);
    const double f = 0.25 / M_PI;
    for (int k = 0; k < 3; ++k)
      out[3 * dd + k] = make_double2(f * (red[0][k].x - d[k] * dw.x), f * (red[0][k].y - d[k] * dw.y));
  }
}

// Device address of g_ff_scratch, looked up once per device (with that device current).
static std::mutex g_scratch_mu;
static double2 *g_scratch_ptr[256] = {nullptr};

static efie_status scratch_address(int dev, double2 **out) {
  if (dev < 0 || dev >= 256) return EFIE_EINVAL;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ff_scratch) != cudaSuccess || !p) return EFIE_ECUDA;
    g_scratch_ptr[dev] = static_cast<double2 *>(p);
  }
  *out = g_scratch_ptr[dev];
  return EFIE_OK;
}

}  // namespace efie

using namespace efie;

extern "C" efie_status efie_far_field_noalloc(efie_ctx *ctx, const double *w_dev, int ndir, const double *dirs_dev,
                                              double *e_inf_dev) {
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  if (!c || ndir < 0 || (ndir > 0 && (!w_dev || !dirs_dev || !e_inf_dev))) return EFIE_EINVAL;
  if (!c->setup_done) return EFIE_ESTATE;
  if (ndir == 0) return EFIE_OK;
  if (c->gr > kMaxRule || c->gr * c->gr > 256) return EFIE_EINVAL;
  const int nchunk = (c->nE + kFFChunk - 1) / kFFChunk;
  if ((size_t)3 * ndir * nchunk > kFFScratchElems) {
    c->err = "efie_far_field_noalloc: 3 * ndir * ceil(elements / 16) exceeds the 2^18-entry scratch";
    return EFIE_EINVAL;
  }
  if (ndir > 65535) {
    c->err = "efie_far_field_noalloc: at most 65535 directions per call";
    return EFIE_EINVAL;
  }
  // the caller's current device is put back on every return
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return EFIE_ECUDA;
  struct RestoreDevice {
    int dev;
    ~RestoreDevice() { cudaSetDevice(dev); }
  } restore{prev};
  if (cudaSetDevice(c->device) != cudaSuccess) return EFIE_ECUDA;
  double2 *part = nullptr;
  EFIE_TRY(scratch_address(c->device, &part));
  FFRule rule{};
  for (int i = 0; i < c->gr; ++i) {
    rule.x[i] = c->tab.gx[i];
    rule.w[i] = c->tab.gw[i];
  }
  dim3 grid(nchunk, ndir);
  k_ff_partial_noalloc<<<grid, 256, 0, c->stream>>>(c->d_patches, c->d_knots, c->d_cpw, c->n, c->p, c->gr, rule,
                                                   c->kappa, c->nE, nchunk, dirs_dev, c->d_tg_ptr, c->d_tg_col,
                                                   c->d_tg_val, reinterpret_cast<const double2 *>(w_dev), part);
  ++c->launches;
  k_ff_final_noalloc<<<ndir, 256, 0, c->stream>>>(nchunk, dirs_dev, part, reinterpret_cast<double2 *>(e_inf_dev));
  ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  return EFIE_OK;
}
