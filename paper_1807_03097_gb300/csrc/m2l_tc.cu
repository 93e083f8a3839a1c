// M2L of several right-hand sides on the tensor cores (a6, Sec. 4.2: the coupling of an
// admissible block is the kernel sampled at the tensor Chebyshev points of both clusters).
//
// For a target cluster t, a group of 64 fields (16 right-hand sides x {x, y, z, div}) and the
// far list of t, the contribution is C(i, f) = sum_s sum_j G_ts(i, j) S_s(j, f) with complex G
// and S.  On the tensor cores it runs transposed, with the fields on the 128 MMA rows:
//   A_s = [Re S_s^T; Im S_s^T]        (128 x nI, per source cluster),
//   D1  = A_s (Re G_ts)^T,  D2 = A_s (Im G_ts)^T      (128 x nI each, FP32 in tensor memory),
//   Re C^T = D1[0:64] - D2[64:128],  Im C^T = D1[64:128] + D2[0:64].
// Each FP32 operand is split as hi + lo with hi in TF32; the three products hi*hi, hi*lo and
// lo*hi carry about 21 bits.  The tensor core rounds its accumulator more coarsely than an
// FP32 add, so each block pair gets a fresh accumulator and the pair's result is added to
// FP32 registers (two tensor-memory buffers: the MMAs of pair p+1 run while pair p drains).
//
// Warp roles in a block of 288 threads: warps 0-7 stage operands (A from the folded moments,
// B by evaluating e^{i kappa |x - y|} / (4 pi |x - y|) with the same phase forms as the CUDA
// core kernels), drain the accumulators and write the result; warp 8 allocates tensor memory
// and one of its lanes issues the MMAs.  Operands go through two shared-memory stages of 32
// source nodes each, handed over with mbarriers; every wait is bounded and a wait that runs
// out sets an error flag for the host.
#include "efie_internal.h"
#include "tc.cuh"

namespace efie {

namespace {

constexpr int kTcFields = 64;       // fields per block (MMA rows = 2 x 64)
constexpr int kTcProducers = 256;   // threads of warps 0-7
constexpr int kTcThreads = kTcProducers + 32;
constexpr long long kTcWaitCycles = 1ll << 31;  // about a second

template <int NP>
struct TcLayout {
  static constexpr uint32_t kA = 128 * 128;            // one [128 x 32] FP32 tile
  static constexpr uint32_t kB = NP * 128;             // one [NP x 32] FP32 tile
  static constexpr uint32_t kStage = 2 * kA + 4 * kB;  // A hi, A lo, Re B hi/lo, Im B hi/lo
  static constexpr uint32_t kNodes = 2 * kStage;       // target node positions, float4 [NP]
  static constexpr uint32_t kBars = kNodes + 16 * NP;
  static constexpr uint32_t kBytes = kBars + 80;
  static constexpr uint32_t kCols = 4 * NP <= 256 ? 256 : 512;  // tensor-memory columns
  static_assert(2 * 128 * (NP + 1) * 4 <= 2 * kStage, "epilogue staging must fit in the stages");
};

__device__ __forceinline__ float2 kernel_entry(int mode, float4 g, float2 ph, float kappa, float4 xt, float4 xs) {
  const float inv2pi = 0.15915494309189535f, c1 = 6.28318548202514648f, c2 = -1.7484555e-7f;
  float ex = xt.x - xs.x, ey = xt.y - xs.y, ez = xt.z - xs.z, rinv, phs;
  if (mode == 0) {
    float vx = g.x + ex, vy = g.y + ey, vz = g.z + ez;
    float r2 = vx * vx + vy * vy + vz * vz;
    rinv = rsqrtf(r2);
    phs = fmaf(kappa, r2 * rinv, -kappa * g.w);
  } else {
    float num = fmaf(2.f, g.x * ex + g.y * ey + g.z * ez, ex * ex + ey * ey + ez * ez);
    float r2 = g.w * g.w + num;
    rinv = rsqrtf(r2);
    phs = kappa * __fdividef(num, r2 * rinv + g.w);
    if (mode == 2) {
      float q = rintf(phs * inv2pi);
      phs = fmaf(-q, c1, phs);
      phs = fmaf(-q, c2, phs);
    }
  }
  float sn, cs;
  __sincosf(phs, &sn, &cs);
  const float gr = cs * rinv, gi = sn * rinv;
  return make_float2(ph.x * gr - ph.y * gi, ph.x * gi + ph.y * gr);
}

__device__ __forceinline__ void st4(uint8_t *base, uint32_t off, const float *v) {
  *reinterpret_cast<float4 *>(base + off) = make_float4(v[0], v[1], v[2], v[3]);
}

__device__ __forceinline__ void producers_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

}  // namespace

template <int NP>
__global__ void __launch_bounds__(kTcThreads, 1) k_m2l_tc(
    const int *__restrict__ targets, const int *__restrict__ fptr, const int *__restrict__ fsrc,
    const float4 *__restrict__ pgeo, const float2 *__restrict__ pph, int nI, float kappa, int mode,
    const float4 *__restrict__ nodeX4, int F, int ld, const float2 *__restrict__ src, float2 *__restrict__ acc,
    int *__restrict__ err) {
  using L = TcLayout<NP>;
  extern __shared__ __align__(1024) uint8_t smem[];
  float4 *sXt = reinterpret_cast<float4 *>(smem + L::kNodes);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBars);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 8);
  const uint32_t b_full = tc::smem_u32(&bars[0]), b_empty = tc::smem_u32(&bars[2]);
  const uint32_t b_tfull = tc::smem_u32(&bars[4]), b_tempty = tc::smem_u32(&bars[6]);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t = targets[blockIdx.x];
  const int f0 = blockIdx.y * kTcFields;
  const int k0 = fptr[t], nsrc = fptr[t + 1] - k0;
  const int nchunk = (nI + 31) / 32, T = nsrc * nchunk;

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(b_full + 8 * i, kTcProducers);
      tc::mbar_init(b_empty + 8 * i, 1);
      tc::mbar_init(b_tfull + 8 * i, 1);
      tc::mbar_init(b_tempty + 8 * i, kTcProducers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < NP; i += blockDim.x) sXt[i] = i < nI ? nodeX4[(size_t)t * nI + i] : make_float4(0, 0, 0, 0);
  if (warp == 8) tc::tmem_alloc(tc::smem_u32(tslot), L::kCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;

  if (warp < 8) {
    // ---------------------------------------------------------------- producers + drain
    constexpr int NBH = NP / 32;  // 16-column blocks per thread and accumulator
    float d1[NBH][16], d2[NBH][16];
#pragma unroll
    for (int b = 0; b < NBH; ++b)
#pragma unroll
      for (int i = 0; i < 16; ++i) d1[b][i] = d2[b][i] = 0.f;
    const int q = warp & 3, h = warp >> 2;
    auto drain = [&](int p) {
      if (!tc::mbar_wait(b_tfull + 8 * (p & 1), (p >> 1) & 1, kTcWaitCycles)) atomicOr(err, 1);
      tc::fence_after_sync();
      const uint32_t col = tbase + ((uint32_t)(32 * q) << 16) + (p & 1) * 2 * NP;
#pragma unroll
      for (int b = 0; b < NBH; ++b) {
        float v[16];
        tc::tmem_ld16(col + 16 * (2 * b + h), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) d1[b][i] += v[i];
        tc::tmem_ld16(col + NP + 16 * (2 * b + h), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) d2[b][i] += v[i];
      }
      tc::fence_before_sync();
      tc::mbar_arrive(b_tempty + 8 * (p & 1));
    };
    for (int it = 0; it < T; ++it) {
      const int st = it & 1, p = it / nchunk, c = it - p * nchunk;
      if (it >= 2 && !tc::mbar_wait(b_empty + 8 * st, ((it >> 1) & 1) ^ 1, kTcWaitCycles)) atomicOr(err, 2);
      uint8_t *sAh = smem + st * L::kStage, *sAl = sAh + L::kA;
      uint8_t *sBrh = sAh + 2 * L::kA, *sBrl = sBrh + L::kB, *sBih = sBrl + L::kB, *sBil = sBih + L::kB;
      const int s = fsrc[k0 + p];
      // A: fields on rows (Re 0-63, Im 64-127), 32 source nodes on K
      for (int task = tid; task < kTcFields * 8; task += kTcProducers) {
        const int f = task & (kTcFields - 1), jq = task >> 6;
        float rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 32 * c + 4 * jq + e;
          float2 v = make_float2(0.f, 0.f);
          if (j < nI && f0 + f < F) v = src[((size_t)s * nI + j) * ld + f0 + f];
          tc::split_tf32(v.x, rh[e], rl[e]);
          tc::split_tf32(v.y, ih[e], il[e]);
        }
        st4(sAh, tc::tile_off(f, 4 * jq), rh);
        st4(sAl, tc::tile_off(f, 4 * jq), rl);
        st4(sAh, tc::tile_off(64 + f, 4 * jq), ih);
        st4(sAl, tc::tile_off(64 + f, 4 * jq), il);
      }
      // B: target nodes on rows, 32 source nodes on K
      const float4 g = pgeo[k0 + p];
      const float2 ph = pph[k0 + p];
      for (int task = tid; task < NP * 8; task += kTcProducers) {
        const int n = task % NP, jq = task / NP;
        float rh[4], rl[4], ih[4], il[4];
        const float4 xt = sXt[n];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 32 * c + 4 * jq + e;
          float2 v = make_float2(0.f, 0.f);
          if (n < nI && j < nI) v = kernel_entry(mode, g, ph, kappa, xt, nodeX4[(size_t)s * nI + j]);
          tc::split_tf32(v.x, rh[e], rl[e]);
          tc::split_tf32(v.y, ih[e], il[e]);
        }
        st4(sBrh, tc::tile_off(n, 4 * jq), rh);
        st4(sBrl, tc::tile_off(n, 4 * jq), rl);
        st4(sBih, tc::tile_off(n, 4 * jq), ih);
        st4(sBil, tc::tile_off(n, 4 * jq), il);
      }
      tc::fence_proxy_async();
      tc::mbar_arrive(b_full + 8 * st);
      if (c == nchunk - 1 && p >= 1) drain(p - 1);
    }
    if (nsrc >= 1) drain(nsrc - 1);
    // ------------------------------------------------------------------- epilogue
    // all MMAs are complete: the stage memory holds D1 and D2 as [128][NP + 1]
    producers_sync();
    float *sD1 = reinterpret_cast<float *>(smem), *sD2 = sD1 + 128 * (NP + 1);
    const int m = 32 * q + lane;
#pragma unroll
    for (int b = 0; b < NBH; ++b)
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = 16 * (2 * b + h) + i;
        sD1[m * (NP + 1) + col] = d1[b][i];
        sD2[m * (NP + 1) + col] = d2[b][i];
      }
    producers_sync();
    for (int idx = tid; idx < nI * kTcFields; idx += kTcProducers) {
      const int f = idx & (kTcFields - 1), i = idx >> 6;
      if (f0 + f >= F) continue;
      const float re = sD1[f * (NP + 1) + i] - sD2[(64 + f) * (NP + 1) + i];
      const float im = sD1[(64 + f) * (NP + 1) + i] + sD2[f * (NP + 1) + i];
      acc[((size_t)t * nI + i) * ld + f0 + f] = make_float2(re, im);
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------------- MMA issue
    const uint32_t idesc = tc::idesc_tf32(128, NP);
    for (int it = 0; it < T; ++it) {
      const int st = it & 1, p = it / nchunk, c = it - p * nchunk;
      if (c == 0 && p >= 2 && !tc::mbar_wait(b_tempty + 8 * (p & 1), ((p >> 1) & 1) ^ 1, kTcWaitCycles))
        atomicOr(err, 4);
      if (!tc::mbar_wait(b_full + 8 * st, (it >> 1) & 1, kTcWaitCycles)) atomicOr(err, 8);
      tc::fence_after_sync();
      const int ksteps = min(4, (nI - 32 * c + 7) / 8);
      const uint32_t ah = tc::smem_u32(smem + st * L::kStage), al = ah + L::kA;
      const uint32_t brh = ah + 2 * L::kA, brl = brh + L::kB, bih = brl + L::kB, bil = bih + L::kB;
      const uint32_t d1 = tbase + (p & 1) * 2 * NP, d2 = d1 + NP;
      for (int ks = 0; ks < ksteps; ++ks) {
        const uint32_t o = ks * tc::kKStepBytes, accum = (c > 0 || ks > 0) ? 1u : 0u;
        const uint64_t dah = tc::smem_desc(ah + o), dal = tc::smem_desc(al + o);
        tc::mma_tf32(d1, dah, tc::smem_desc(brh + o), idesc, accum);
        tc::mma_tf32(d1, dah, tc::smem_desc(brl + o), idesc, 1u);
        tc::mma_tf32(d1, dal, tc::smem_desc(brh + o), idesc, 1u);
        tc::mma_tf32(d2, dah, tc::smem_desc(bih + o), idesc, accum);
        tc::mma_tf32(d2, dah, tc::smem_desc(bil + o), idesc, 1u);
        tc::mma_tf32(d2, dal, tc::smem_desc(bih + o), idesc, 1u);
      }
      tc::mma_commit(b_empty + 8 * st);
      if (c == nchunk - 1) tc::mma_commit(b_tfull + 8 * (p & 1));
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 8) tc::tmem_dealloc(tbase, L::kCols);
}

template <int NP>
static efie_status tc_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TcLayout<NP>::kBytes);
  return e == cudaSuccess ? EFIE_OK : EFIE_ECUDA;
}

bool m2l_tc_supported(const Ctx *c) { return c->nI <= 128; }

efie_status m2l_tc_prepare(Ctx *c) {
  EFIE_TRY(tc_attr<64>());
  EFIE_TRY(tc_attr<96>());
  EFIE_TRY(tc_attr<128>());
  if (!c->d_tc_err) {
    EFIE_CUDA(cudaMalloc((void **)&c->d_tc_err, sizeof(int)));
    EFIE_CUDA(cudaMemset(c->d_tc_err, 0, sizeof(int)));
  }
  return EFIE_OK;
}

// acc[t][i][f] for the targets of the M2L, f < F = 4 R, row stride ld (float2 entries)
efie_status launch_m2l_tc(Ctx *c, cudaStream_t st, int F, int ld, const float2 *src, float2 *acc) {
  if (c->n_m2l_targets == 0) return EFIE_OK;
  const int nI = c->nI;
  dim3 grid(c->n_m2l_targets, (F + kTcFields - 1) / kTcFields);
  const float kf = (float)c->kappa;
#define EFIE_TC(NPV)                                                                                          \
  k_m2l_tc<NPV><<<grid, kTcThreads, TcLayout<NPV>::kBytes, st>>>(c->d_m2l_targets, c->d_far_ptr, c->d_far_src, \
                                                                 c->d_pgeo, c->d_pph, nI, kf, c->m2l_mode,     \
                                                                 c->d_nodeX4, F, ld, src, acc, c->d_tc_err)
  if (nI <= 64) EFIE_TC(64);
  else if (nI <= 96) EFIE_TC(96);
  else if (nI <= 128) EFIE_TC(128);
  else return EFIE_EINVAL;
#undef EFIE_TC
  ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

efie_status m2l_tc_check(Ctx *c) {
  if (!c->d_tc_err) return EFIE_OK;
  int e = 0;
  EFIE_CUDA(cudaMemcpyAsync(&e, c->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  EFIE_CUDA(cudaStreamSynchronize(c->stream));
  if (e) {
    c->err = "tensor-core M2L: a pipeline wait ran out (code " + std::to_string(e) + ")";
    cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream);
    return EFIE_ETIMEOUT;
  }
  return EFIE_OK;
}

}  // namespace efie
