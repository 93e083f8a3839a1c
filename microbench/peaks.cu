// Compute-only throughput of the pipes the EFIE kernels are bound by, measured on the GPU the
// library runs on (no memory traffic):
//   FFMA     fma.rn.f32                (FP32 FMA pipe; 2 flop per lane)
//   FFMA2    fma.rn.f32x2              (packed FP32, two FMAs per lane per instruction)
//   DFMA     fma.rn.f64                (FP64 pipe)
//   MUFU     rsqrt / sin / cos approx  (special-function unit)
//   tcgen05  kind::tf32 and kind::f16 (bf16) MMAs, M = 128, issued back to back by one thread
//            per SM from descriptors built once (zero operands in shared memory).
// Each ALU kernel runs 16 independent dependency chains per thread on 4 blocks of 256
// threads per SM, so that latency is hidden and only the pipe's rate limits it.  Rates are
// operations per second over the whole GPU from CUDA events around one launch.
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "../paper_1807_03097_gb300/csrc/tc.cuh"

using namespace efie;

namespace {

constexpr int kChains = 16;

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long A = *reinterpret_cast<unsigned long long *>(&a);
  unsigned long long B = *reinterpret_cast<unsigned long long *>(&b);
  unsigned long long C = *reinterpret_cast<unsigned long long *>(&c);
  unsigned long long D;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D) : "l"(A), "l"(B), "l"(C));
  return *reinterpret_cast<float2 *>(&D);
}

__global__ void k_ffma(int iters, float b, float c, float *sink) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3f * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[i]) : "f"(b), "f"(c));
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == 1234.5f) sink[0] = s;
}

__global__ void k_ffma2(int iters, float b, float c, float *sink) {
  float2 x[kChains / 2];
#pragma unroll
  for (int i = 0; i < kChains / 2; ++i) x[i] = make_float2(1e-3f * (threadIdx.x + i), 2e-3f * i);
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains / 2; ++i) x[i] = ffma2(x[i], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains / 2; ++i) s += x[i].x + x[i].y;
  if (s == 1234.5f) sink[0] = s;
}

__global__ void k_dfma(int iters, double b, double c, float *sink) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(x[i]) : "d"(b), "d"(c));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == 1234.5) sink[0] = (float)s;
}

// OP 0 rsqrt, 1 sin, 2 cos (the approximate forms the kernels use)
template <int OP>
__global__ void k_mufu(int iters, float *sink) {
  float x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 0.5f + 1e-3f * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      if (OP == 0) asm volatile("rsqrt.approx.f32 %0, %0;" : "+f"(x[i]));
      if (OP == 1) asm volatile("sin.approx.f32 %0, %0;" : "+f"(x[i]));
      if (OP == 2) asm volatile("cos.approx.f32 %0, %0;" : "+f"(x[i]));
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == 1234.5f) sink[0] = s;
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d), "l"(a), "l"(b), "r"(idesc),
               "r"(acc)
               : "memory");
}

constexpr int kMmaSmem = 128 * 1024;

// KIND 0: tf32 (K = 8 per MMA), 1: bf16 (K = 16 per MMA); M = 128, N given; one accumulator.
template <int KIND>
__global__ void k_mma(int N, int iters, long long *cyc, int *err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kMmaSmem);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kMmaSmem / 4; i += blockDim.x) reinterpret_cast<float *>(smem)[i] = 0.f;
  if (threadIdx.x == 0) {
    tc::mbar_init(tc::smem_u32(bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), 256);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = *tslot;
  if (warp == 0 && lane == 0) {
    // bf16 instruction descriptor: FP32 accumulator, A and B bf16 (format 1), K-major
    const uint32_t idesc = KIND == 0 ? tc::idesc_tf32(128, N)
                                     : ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (8u << 24));
    const uint32_t a0 = tc::smem_u32(smem), b0 = a0 + 64 * 1024;
    uint64_t da[4], db[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      da[k] = tc::smem_desc(a0 + 256 * k);
      db[k] = tc::smem_desc(b0 + 256 * k);
    }
    const long long t0 = clock64();
    for (int i = 0; i < iters; i += 8) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (KIND == 0) tc::mma_tf32(tb, da[k & 3], db[k & 3], idesc, 1u);
        else mma_f16(tb, da[k & 3], db[k & 3], idesc, 1u);
      }
    }
    tc::mma_commit(tc::smem_u32(bar));
    if (!tc::mbar_wait(tc::smem_u32(bar), 0, 1ll << 32)) atomicOr(err, 1);
    cyc[blockIdx.x] = clock64() - t0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tb, 256);
}

struct Timer {
  cudaEvent_t a, b;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// Launch `launch(iters)` and grow iters until one launch takes at least 20 ms; returns the
// seconds of the last launch and the iterations it ran (negative seconds on a CUDA error).
template <class F>
double time_launch(F launch, int &iters) {
  Timer t;
  for (int round = 0; round < 8; ++round) {
    launch(iters);  // warm-up at this size
    cudaEventRecord(t.a);
    launch(iters);
    cudaEventRecord(t.b);
    if (cudaEventSynchronize(t.b) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    if (ms >= 20.f || round == 7) return ms * 1e-3;
    iters *= ms < 2.f ? 8 : 2;
  }
  return -1.0;
}

}  // namespace

extern "C" {

// Number of values peaks_measure writes.
int peaks_count(void) { return 10; }

// Measures on the current device and writes, in this order (operations per second over the
// GPU, one operation = one lane-level instruction result):
//  [0] FFMA flop/s (2 per FMA)  [1] FFMA2 flop/s (4 per packed instruction)  [2] DFMA flop/s
//  [3] rsqrt/s  [4] sin/s  [5] cos/s
//  [6] tcgen05 tf32 flop/s (M 128, N 256)  [7] tcgen05 bf16 flop/s (M 128, N 256)
//  [8] SM count  [9] error flag of the MMA kernels (0 = every wait completed).
// Returns 0, or -1 on a CUDA error.
int peaks_measure(double *out, int n) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  float *sink = nullptr;
  long long *cyc = nullptr;
  int *err = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess || cudaMalloc(&cyc, 8 * (size_t)nsm) != cudaSuccess ||
      cudaMalloc(&err, 4) != cudaSuccess)
    return -1;
  cudaMemset(err, 0, 4);
  const int blocks = 4 * nsm, threads = 256;
  const double lanes = (double)blocks * threads;
  double v[10] = {0};
  int it;
  double s;
  it = 4096;
  s = time_launch([&](int i) { k_ffma<<<blocks, threads>>>(i, 0.999999f, 1e-7f, sink); }, it);
  v[0] = s > 0 ? 2.0 * kChains * lanes * it / s : -1;
  it = 4096;
  s = time_launch([&](int i) { k_ffma2<<<blocks, threads>>>(i, 0.999999f, 1e-7f, sink); }, it);
  v[1] = s > 0 ? 2.0 * kChains * lanes * it / s : -1;
  it = 64;
  s = time_launch([&](int i) { k_dfma<<<blocks, threads>>>(i, 0.999999, 1e-7, sink); }, it);
  v[2] = s > 0 ? 2.0 * kChains * lanes * it / s : -1;
  it = 1024;
  s = time_launch([&](int i) { k_mufu<0><<<blocks, threads>>>(i, sink); }, it);
  v[3] = s > 0 ? kChains * lanes * it / s : -1;
  it = 1024;
  s = time_launch([&](int i) { k_mufu<1><<<blocks, threads>>>(i, sink); }, it);
  v[4] = s > 0 ? kChains * lanes * it / s : -1;
  it = 1024;
  s = time_launch([&](int i) { k_mufu<2><<<blocks, threads>>>(i, sink); }, it);
  v[5] = s > 0 ? kChains * lanes * it / s : -1;
  const int msm = kMmaSmem + 64;
  cudaFuncSetAttribute(k_mma<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, msm);
  cudaFuncSetAttribute(k_mma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, msm);
  const int N = 256;
  it = 2048;
  s = time_launch([&](int i) { k_mma<0><<<nsm, 128, msm>>>(N, i, cyc, err); }, it);
  v[6] = s > 0 ? 2.0 * 128 * N * 8 * (double)it * nsm / s : -1;
  it = 2048;
  s = time_launch([&](int i) { k_mma<1><<<nsm, 128, msm>>>(N, i, cyc, err); }, it);
  v[7] = s > 0 ? 2.0 * 128 * N * 16 * (double)it * nsm / s : -1;
  v[8] = nsm;
  int h = 0;
  cudaMemcpy(&h, err, 4, cudaMemcpyDeviceToHost);
  v[9] = h;
  cudaFree(sink);
  cudaFree(cyc);
  cudaFree(err);
  for (int i = 0; i < n && i < 10; ++i) out[i] = v[i];
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // extern "C"
