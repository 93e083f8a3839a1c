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
// FP32 add, so every group of 4 block pairs gets a fresh accumulator D = [D1 D2] (one MMA of
// N = 2 NP against B = [Re G; Im G]), and the group's result is added to running sums S in
// tensor memory with FP32 adds on the CUDA cores.
//
// A block has 17 warps.  Warps 0-15 stage operands (A from the folded moments, B by evaluating
// e^{i kappa |x - y|} / (4 pi |x - y|) with the same phase forms as the CUDA-core kernels),
// fold D into S and write the result; warp 0 also allocates tensor memory.  Lane 0 of warp 16
// issues the MMAs of a stage once every staging warp has written it: the issuing thread
// stalls while the tensor pipe is busy, which a staging warp cannot afford.  Operands go through two
// shared-memory stages of 32 source nodes each, handed over with mbarriers; every wait is
// bounded and a wait that runs out sets an error flag for the host.
#include "efie_internal.h"
#include "tc.cuh"
#include "fastmath.cuh"

namespace efie {

namespace {

constexpr int kTcFields = 64;      // fields per block (MMA rows = 2 x 64)
constexpr int kTcWarps = 16;                    // staging warps
constexpr int kTcProducers = 32 * kTcWarps;
constexpr int kTcThreads = kTcProducers + 32;   // + the MMA-issue warp
constexpr long long kTcWaitCycles = 1ll << 31;  // about a second
constexpr int kTcGroup = 4;  // block pairs accumulated in D before it is folded into S

template <int NP>
struct TcLayout {
  static constexpr uint32_t kA = 128 * 128;            // one [128 x 32] FP32 tile
  static constexpr uint32_t kB = NP * 128;             // one [NP x 32] FP32 tile
  static constexpr uint32_t kStage = 2 * kA + 4 * kB;  // A hi, A lo, B hi, B lo (B: Re rows, Im rows)
  static constexpr uint32_t kNodes = 2 * kStage;       // target node positions, float4 [NP]
  static constexpr uint32_t kBars = kNodes + 16 * NP;
  static constexpr uint32_t kBytes = kBars + 64;
  static constexpr uint32_t kCols = 4 * NP <= 256 ? 256 : 512;  // D1, D2, S1, S2
  static_assert(2 * 128 * (NP + 1) * 4 <= 2 * kStage, "epilogue staging must fit in the stages");
};

// Two kernel entries (one target node, source nodes xs0 and xs1) with packed FP32 arithmetic
// (FFMA2 and friends: two lanes' worth of work per instruction), phase forms as in the CUDA-core
// kernels; ut = g + xt (pair offset plus target node) is used by the direct form (MODE 0) only.
// re = (Re G0, Re G1), im = (Im G0, Im G1).
template <int MODE>
__device__ __forceinline__ void kernel_entry2(float4 g, float2 ph, float kappa, float4 xt, float4 ut, float4 xs0,
                                              float4 xs1, float2 &re, float2 &im) {
  const float inv2pi = 0.15915494309189535f, c1 = 6.28318548202514648f, c2 = -1.7484555e-7f;
  float2 rinv, phs;
  if (MODE == 0) {
    const float2 vx = __fadd2_rn(make_float2(ut.x, ut.x), make_float2(-xs0.x, -xs1.x));
    const float2 vy = __fadd2_rn(make_float2(ut.y, ut.y), make_float2(-xs0.y, -xs1.y));
    const float2 vz = __fadd2_rn(make_float2(ut.z, ut.z), make_float2(-xs0.z, -xs1.z));
    const float2 r2 = __ffma2_rn(vz, vz, __ffma2_rn(vy, vy, __fmul2_rn(vx, vx)));
    rinv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
    phs = __ffma2_rn(make_float2(kappa, kappa), __fmul2_rn(r2, rinv), make_float2(-kappa * g.w, -kappa * g.w));
  } else {
    const float2 ex = __fadd2_rn(make_float2(xt.x, xt.x), make_float2(-xs0.x, -xs1.x));
    const float2 ey = __fadd2_rn(make_float2(xt.y, xt.y), make_float2(-xs0.y, -xs1.y));
    const float2 ez = __fadd2_rn(make_float2(xt.z, xt.z), make_float2(-xs0.z, -xs1.z));
    const float2 d1 = __ffma2_rn(make_float2(g.z, g.z), ez,
                                 __ffma2_rn(make_float2(g.y, g.y), ey, __fmul2_rn(make_float2(g.x, g.x), ex)));
    const float2 d2 = __ffma2_rn(ez, ez, __ffma2_rn(ey, ey, __fmul2_rn(ex, ex)));
    const float2 num = __ffma2_rn(make_float2(2.f, 2.f), d1, d2);
    const float2 r2 = __fadd2_rn(make_float2(g.w * g.w, g.w * g.w), num);
    rinv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
    const float2 den = __ffma2_rn(r2, rinv, make_float2(g.w, g.w));
    phs = __fmul2_rn(__fmul2_rn(make_float2(kappa, kappa), num), make_float2(rcp_ftz(den.x), rcp_ftz(den.y)));
    if (MODE == 2) {
      const float2 qq = __fmul2_rn(phs, make_float2(inv2pi, inv2pi));
      const float2 qn = make_float2(-rintf(qq.x), -rintf(qq.y));
      phs = __ffma2_rn(qn, make_float2(c1, c1), phs);
      phs = __ffma2_rn(qn, make_float2(c2, c2), phs);
    }
  }
  const float2 sn = make_float2(sin_ftz(phs.x), sin_ftz(phs.y)), cs = make_float2(cos_ftz(phs.x), cos_ftz(phs.y));
  const float2 gr = __fmul2_rn(cs, rinv), gi = __fmul2_rn(sn, rinv);
  re = __ffma2_rn(make_float2(ph.x, ph.x), gr, __fmul2_rn(make_float2(-ph.y, -ph.y), gi));
  im = __ffma2_rn(make_float2(ph.x, ph.x), gi, __fmul2_rn(make_float2(ph.y, ph.y), gr));
}

__device__ __forceinline__ void st2(uint8_t *base, uint32_t off, float a, float b) {
  *reinterpret_cast<float2 *>(base + off) = make_float2(a, b);
}

// Read-only loads issued where they stand (volatile: the scheduler does not sink them towards
// their use), so that the loads of the next stage overlap the evaluation of this one.
__device__ __forceinline__ float4 ldg_pin(const float4 *p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ldg_pin(const float2 *p) {
  float2 v;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ int ldg_pin(const int *p) {
  int v;
  asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

}  // namespace

// Staging map of a stage: lane l of warp w covers the source nodes j = 32 c + 4 (w % 8) +
// 2 ((l / 8) % 2) + e (e < 2) and the rows r = l % 8 + 8 (l / 16) + 16 (2 i + w / 8): fields
// f = r (A rows f and 64 + f, i < 2) and target nodes n = r (B rows, i < NP / 32).  A
// half-warp then writes 8 rows x 4 K-columns, 32 distinct banks.  Tensor memory: D1 [0, NP), D2 [NP, 2 NP) hold the group of block
// pairs in flight, S1 [2 NP, 3 NP), S2 [3 NP, 4 NP) the running sums over the far list.
template <int NP, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_m2l_tc(
    const int *__restrict__ targets, const int *__restrict__ fptr, const int *__restrict__ fsrc,
    const float4 *__restrict__ pgeo, const float2 *__restrict__ pph, int nI, float kappa,
    const float4 *__restrict__ nodeX4, int F, int ld, const float2 *__restrict__ src, float2 *__restrict__ acc,
    int *__restrict__ err) {
  using L = TcLayout<NP>;
  extern __shared__ __align__(1024) uint8_t smem[];
  float4 *sXt = reinterpret_cast<float4 *>(smem + L::kNodes);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L::kBars);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 6);
  const uint32_t b_full = tc::smem_u32(&bars[0]), b_empty = tc::smem_u32(&bars[2]);
  const uint32_t b_tfull = tc::smem_u32(&bars[4]), b_tempty = tc::smem_u32(&bars[5]);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int jq = warp & 7, jh = (lane >> 3) & 1;  // source nodes 4 jq + 2 jh + {0, 1}
  const int rbase = (lane & 7) + 8 * (lane >> 4) + 16 * (warp >> 3);  // rows rbase + 32 i
  const int t = targets[blockIdx.x];
  const int f0 = blockIdx.y * kTcFields;
  const int k0 = fptr[t], nsrc = fptr[t + 1] - k0;
  const int nchunk = (nI + 31) / 32, T = nsrc * nchunk;

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(b_full + 8 * i, kTcProducers);
      tc::mbar_init(b_empty + 8 * i, 1);
    }
    tc::mbar_init(b_tfull, 1);
    tc::mbar_init(b_tempty, kTcProducers);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < NP; i += kTcThreads) sXt[i] = i < nI ? nodeX4[(size_t)t * nI + i] : make_float4(0, 0, 0, 0);
  // B rows of target nodes n >= nI (padding up to NP, in the Re and the Im half) stay zero
  for (int i = tid; i < 2 * 2 * 2 * (NP - nI) * 8; i += kTcThreads) {
    const int kg = i & 7, n = nI + (i >> 3) % (NP - nI), tl = (i >> 3) / (NP - nI);
    // tl: stage (bit 2), hi/lo tile (bit 1), Re/Im half (bit 0)
    *reinterpret_cast<float4 *>(smem + (tl >> 2) * L::kStage + 2 * L::kA + ((tl >> 1) & 1) * 2 * L::kB +
                                tc::tile_off((tl & 1) * NP + n, 4 * kg)) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), L::kCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t idesc = tc::idesc_tf32(128, 2 * NP);
  const int q = warp & 3, r4 = warp >> 2;  // lane quadrant and column quarter of the drain
  const uint32_t tq = tbase + ((uint32_t)(32 * q) << 16);

  if (warp < kTcWarps) {
  // S += D for group g of block pairs (S = D for the first), then release D to the MMAs.
  // This thread covers lane 32 q + lane and the column blocks b = r4 + 4 i of D1/S1, D2/S2.
  auto drain = [&](int g) {
    constexpr int NB = NP / 32;
    const int p = g;
    if (!tc::mbar_wait(b_tfull, g & 1, kTcWaitCycles)) atomicOr(err, 1);
    tc::fence_after_sync();
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      uint32_t d[NB][8], sv[NB][8];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const uint32_t cd = tq + half * NP + 8 * (r4 + 4 * i);
        tc::tmem_ld8_async(cd, d[i]);
        if (p > 0) tc::tmem_ld8_async(cd + 2 * NP, sv[i]);
      }
      tc::tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        tc::touch8(d[i]);
        if (p > 0) {
          tc::touch8(sv[i]);
#pragma unroll
          for (int k = 0; k < 8; ++k) d[i][k] = __float_as_uint(__uint_as_float(d[i][k]) + __uint_as_float(sv[i][k]));
        }
        tc::tmem_st8_async(tq + half * NP + 8 * (r4 + 4 * i) + 2 * NP, d[i]);
      }
    }
    tc::tmem_wait_st();
    tc::fence_before_sync();
    tc::mbar_arrive(b_tempty);
  };

  float4 cx[2], nx[2];
  float2 ca[2][2], na[2][2];
  float4 cg, ng = make_float4(0, 0, 0, 1);
  float2 cph, nph = make_float2(0, 0);
  int s_next = nsrc > 0 ? ldg_pin(fsrc + k0) : 0;
  int lp = 0, lc = 0;  // (pair, chunk) that load_stage fetches next
  auto load_stage = [&]() {
    if (lp >= nsrc) return;
    const int p2 = lp, c2 = lc;
    if (++lc == nchunk) {
      lc = 0;
      ++lp;
    }
    const int s2 = s_next;
    if (lp < nsrc && lc == 0) s_next = ldg_pin(fsrc + k0 + lp);
    ng = ldg_pin(pgeo + k0 + p2);
    nph = ldg_pin(pph + k0 + p2);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int j = 32 * c2 + 4 * jq + 2 * jh + e;
      const bool jv = j < nI;
      nx[e] = jv ? ldg_pin(nodeX4 + (size_t)s2 * nI + j) : make_float4(0, 0, 0, 0);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int f = rbase + 32 * k;
        na[k][e] = (jv && f0 + f < F) ? ldg_pin(src + ((size_t)s2 * nI + j) * ld + f0 + f) : make_float2(0.f, 0.f);
      }
    }
  };
  load_stage();
  for (int it = 0, p = 0, c = 0; it < T; ++it, c = (c + 1 == nchunk) ? 0 : c + 1, p += (c == 0)) {
    const int st = it & 1;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      cx[e] = nx[e];
      ca[0][e] = na[0][e];
      ca[1][e] = na[1][e];
    }
    cg = ng;
    cph = nph;
    load_stage();
    if (it >= 2 && !tc::mbar_wait(b_empty + 8 * st, ((it >> 1) & 1) ^ 1, kTcWaitCycles)) atomicOr(err, 2);
    uint8_t *sAh = smem + st * L::kStage, *sAl = sAh + L::kA;
    uint8_t *sBh = sAh + 2 * L::kA, *sBl = sBh + 2 * L::kB;  // rows [0, NP) Re, [NP, 2 NP) Im
    const uint32_t kcol = 4 * jq + 2 * jh;
    // A: fields on rows (Re 0-63, Im 64-127), this warp's 2 source nodes on K
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int f = rbase + 32 * k;
      float rh[2], rl[2], ih[2], il[2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        tc::split_tf32(ca[k][e].x, rh[e], rl[e]);
        tc::split_tf32(ca[k][e].y, ih[e], il[e]);
      }
      st2(sAh, tc::tile_off(f, kcol), rh[0], rh[1]);
      st2(sAl, tc::tile_off(f, kcol), rl[0], rl[1]);
      st2(sAh, tc::tile_off(64 + f, kcol), ih[0], ih[1]);
      st2(sAl, tc::tile_off(64 + f, kcol), il[0], il[1]);
    }
    // B: target nodes on rows, this warp's 2 source nodes on K
    const int jb = 32 * c + (int)kcol;
#pragma unroll
    for (int k = 0; k < NP / 32; ++k) {
      const int n = rbase + 32 * k;
      if (n >= nI) continue;  // padding rows, zero since the start
      const float4 xt = sXt[n];
      const float4 ut = make_float4(cg.x + xt.x, cg.y + xt.y, cg.z + xt.z, 0.f);
      float rh[2], rl[2], ih[2], il[2];
      float2 gre, gim;
      kernel_entry2<MODE>(cg, cph, kappa, xt, ut, cx[0], cx[1], gre, gim);
      if (jb >= nI) gre.x = gim.x = 0.f;
      if (jb + 1 >= nI) gre.y = gim.y = 0.f;
      tc::split_tf32(gre.x, rh[0], rl[0]);
      tc::split_tf32(gim.x, ih[0], il[0]);
      tc::split_tf32(gre.y, rh[1], rl[1]);
      tc::split_tf32(gim.y, ih[1], il[1]);
      st2(sBh, tc::tile_off(n, kcol), rh[0], rh[1]);
      st2(sBl, tc::tile_off(n, kcol), rl[0], rl[1]);
      st2(sBh, tc::tile_off(NP + n, kcol), ih[0], ih[1]);
      st2(sBl, tc::tile_off(NP + n, kcol), il[0], il[1]);
    }
    tc::fence_proxy_async();
    tc::mbar_arrive(b_full + 8 * st);
    // the previous group's MMAs are done by now: fold it into the running sums
    const bool gstart = c == 0 && p % kTcGroup == 0;
    if (gstart && p >= 1) drain(p / kTcGroup - 1);
  }
  if (nsrc >= 1) drain((nsrc - 1) / kTcGroup);
  } else if (lane == 0) {
    // ------------------------------------------------------------------- MMA issue
    // One thread, so that its waits on the tensor pipe stall no staging warp.  Descriptors are
    // built once; the start address sits in the low bits, so stage st and K-step ks are
    // reached by adding (st kStage + 256 ks) / 16 (shared addresses stay below 2^18 bytes).
    const uint32_t a0 = tc::smem_u32(smem);
    const uint64_t dah0 = tc::smem_desc(a0), dal0 = tc::smem_desc(a0 + L::kA);
    const uint64_t dbh0 = tc::smem_desc(a0 + 2 * L::kA), dbl0 = tc::smem_desc(a0 + 2 * L::kA + 2 * L::kB);
    for (int it = 0, p = 0, c = 0; it < T; ++it, c = (c + 1 == nchunk) ? 0 : c + 1, p += (c == 0)) {
      const int st = it & 1;
      const bool gstart = c == 0 && p % kTcGroup == 0;
      // [D1 D2] (+)= A [Re B; Im B]^T, three split products per K-step
      if (gstart && p >= 1 && !tc::mbar_wait(b_tempty, (p / kTcGroup - 1) & 1, kTcWaitCycles)) atomicOr(err, 4);
      if (!tc::mbar_wait(b_full + 8 * st, (it >> 1) & 1, kTcWaitCycles)) atomicOr(err, 8);
      tc::fence_after_sync();
      const int ksteps = min(4, (nI - 32 * c + 7) / 8);
      for (int ks = 0; ks < ksteps; ++ks) {
        const uint64_t o = (uint64_t)(st * (L::kStage >> 4) + 16 * ks);
        tc::mma_tf32(tbase, dah0 + o, dbh0 + o, idesc, (gstart && ks == 0) ? 0u : 1u);
        tc::mma_tf32(tbase, dah0 + o, dbl0 + o, idesc, 1u);
        tc::mma_tf32(tbase, dal0 + o, dbh0 + o, idesc, 1u);
      }
      tc::mma_commit(b_empty + 8 * st);
      if (c == nchunk - 1 && (p % kTcGroup == kTcGroup - 1 || p == nsrc - 1)) tc::mma_commit(b_tfull);
    }
  }
  __syncwarp();
  // ------------------------------------------------------------------------- epilogue
  // every MMA is complete and drained: stage the sums as [128][NP + 1] in the stage memory
  __syncthreads();
  float *sS1 = reinterpret_cast<float *>(smem), *sS2 = sS1 + 128 * (NP + 1);
  const int m = 32 * q + lane;
  if (warp >= kTcWarps) {
    // the MMA-issue warp takes no part in staging the sums
  } else if (nsrc >= 1) {
    tc::fence_after_sync();
#pragma unroll 1
    for (int b = r4; b < NP / 8; b += 4) {
      float v[8];
      tc::tmem_ld8(tq + 2 * NP + 8 * b, v);
#pragma unroll
      for (int i = 0; i < 8; ++i) sS1[m * (NP + 1) + 8 * b + i] = v[i];
      tc::tmem_ld8(tq + 3 * NP + 8 * b, v);
#pragma unroll
      for (int i = 0; i < 8; ++i) sS2[m * (NP + 1) + 8 * b + i] = v[i];
    }
  } else {
    for (int b = r4; b < NP / 8; b += 4)
      for (int i = 0; i < 8; ++i) sS1[m * (NP + 1) + 8 * b + i] = sS2[m * (NP + 1) + 8 * b + i] = 0.f;
  }
  __syncthreads();
  for (int idx = tid; idx < nI * kTcFields; idx += kTcThreads) {
    const int f = idx & (kTcFields - 1), i = idx >> 6;
    if (f0 + f >= F) continue;
    const float re = sS1[f * (NP + 1) + i] - sS2[(64 + f) * (NP + 1) + i];
    const float im = sS1[(64 + f) * (NP + 1) + i] + sS2[f * (NP + 1) + i];
    acc[((size_t)t * nI + i) * ld + f0 + f] = make_float2(re, im);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, L::kCols);
}

template <int NP, int MODE>
static efie_status tc_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_m2l_tc<NP, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TcLayout<NP>::kBytes);
  return e == cudaSuccess ? EFIE_OK : EFIE_ECUDA;
}

template <int NP>
static efie_status tc_attrs() {
  efie_status e = tc_attr<NP, 0>();
  if (e == EFIE_OK) e = tc_attr<NP, 1>();
  if (e == EFIE_OK) e = tc_attr<NP, 2>();
  return e;
}

bool m2l_tc_supported(const Ctx *c) { return c->nI <= 128; }

efie_status m2l_tc_prepare(Ctx *c) {
  EFIE_TRY(tc_attrs<64>());
  EFIE_TRY(tc_attrs<96>());
  EFIE_TRY(tc_attrs<128>());
  if (!c->d_tc_err) {
    EFIE_TRY(dalloc(c, &c->d_tc_err, 1));
    EFIE_CUDA(cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream));
  }
  return EFIE_OK;
}

template <int NP>
static void launch_np(Ctx *c, cudaStream_t st, dim3 grid, int F, int ld, const float2 *src, float2 *acc) {
  const float kf = (float)c->kappa;
#define EFIE_TC(MV)                                                                                      \
  k_m2l_tc<NP, MV><<<grid, kTcThreads, TcLayout<NP>::kBytes, st>>>(c->d_m2l_targets, c->d_far_ptr,          \
                                                                   c->d_far_src, c->d_pgeo, c->d_pph, c->nI, \
                                                                   kf, c->d_nodeX4, F, ld, src, acc, c->d_tc_err)
  if (c->m2l_mode == 0) EFIE_TC(0);
  else if (c->m2l_mode == 1) EFIE_TC(1);
  else EFIE_TC(2);
#undef EFIE_TC
}

// acc[t][i][f] for the targets of the M2L, f < F = 4 R, row stride ld (float2 entries)
efie_status launch_m2l_tc(Ctx *c, cudaStream_t st, int F, int ld, const float2 *src, float2 *acc) {
  if (c->n_m2l_targets == 0) return EFIE_OK;
  const int nI = c->nI;
  dim3 grid(c->n_m2l_targets, (F + kTcFields - 1) / kTcFields);
  if (nI <= 64) launch_np<64>(c, st, grid, F, ld, src, acc);
  else if (nI <= 96) launch_np<96>(c, st, grid, F, ld, src, acc);
  else if (nI <= 128) launch_np<128>(c, st, grid, F, ld, src, acc);
  else return EFIE_EINVAL;
  ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return EFIE_OK;
}

// One bounded wait on an mbarrier that nothing ever completes (the situation of a stalled
// pipeline stage): the wait gives up after `cycles` clocks and sets the same error flag as the
// tensor-core M2L.  The barrier lives in shared memory and is abandoned when the block exits.
__global__ void k_wait_selftest(long long cycles, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!tc::mbar_wait(tc::smem_u32(&bar), 0, cycles)) atomicOr(err, 16);
  }
}

efie_status dev_wait_selftest(Ctx *c, long long cycles) {
  EFIE_TRY(m2l_tc_prepare(c));
  k_wait_selftest<<<1, 32, 0, c->stream>>>(cycles, c->d_tc_err);
  ++c->launches;
  EFIE_CUDA(cudaGetLastError());
  return m2l_tc_check(c);
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
