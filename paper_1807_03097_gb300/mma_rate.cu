// Throughput of tcgen05.mma on this GPU (measurement tool, not part of the library): one CTA
// per SM; lane 0 of warp 0 issues MMAs back to back from descriptors built once (zero
// operands in shared memory, no memory traffic) into one or several tensor-memory
// accumulators, in the K-major no-swizzle layout the tensor-core M2L uses and in the 128-byte
// swizzled layout.  Reports cycles per MMA and flop per clock per SM (clock64 on SM 0) and the
// whole-GPU rate (CUDA events).  Build and run on the GPU:
//   nvcc -O3 -std=c++17 -gencode arch=compute_103a,code=sm_103a -o /tmp/mma_rate \
//        paper_1807_03097_gb300/mma_rate.cu && /tmp/mma_rate
#include <cstdio>
#include <cuda_runtime.h>
#include "csrc/tc.cuh"
using namespace efie;

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
               : "memory");
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // 8 rows x 128 B
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

template <int KIND>  // 0 tf32, 1 bf16
__global__ void k_bench(int N, int iters, int nbuf, int nacc, int swz, long long *cyc, int *err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 200 * 1024);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < 200 * 1024 / 4; i += blockDim.x) reinterpret_cast<float *>(smem)[i] = 0.f;
  if (threadIdx.x == 0) { tc::mbar_init(tc::smem_u32(bar), 1); asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), 512);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tb = *tslot;
  if (warp == 0 && lane == 0) {
    // tf32: K=8 per MMA (32 B per row); bf16: K=16 per MMA (32 B per row).  Same layout, LBO 128, SBO 1024.
    const uint32_t idesc = KIND == 0 ? tc::idesc_tf32(128, N)
                                     : ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (8u << 24));
    const uint32_t a0 = tc::smem_u32(smem), b0 = a0 + 64 * 1024;
    long long t0 = clock64();
    uint64_t da[4], db[4];
    uint32_t dd[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t o = swz ? k * 32 : k * 256;
      da[k] = swz ? desc_sw128(a0 + o) : tc::smem_desc(a0 + o);
      db[k] = swz ? desc_sw128(b0 + o) : tc::smem_desc(b0 + o);
      dd[k] = tb + (k % nacc) * (uint32_t)N;
    }
    if (KIND == 0) {
      for (int i = 0; i < iters; i += 8) {
#pragma unroll
        for (int k = 0; k < 8; ++k) tc::mma_tf32(dd[k & 3], da[k & 3], db[k & 3], idesc, 1u);
      }
    } else {
      for (int i = 0; i < iters; i += 8) {
#pragma unroll
        for (int k = 0; k < 8; ++k) mma_bf16(dd[k & 3], da[k & 3], db[k & 3], idesc, 1u);
      }
    }
    tc::mma_commit(tc::smem_u32(bar));
    if (!tc::mbar_wait(tc::smem_u32(bar), 0, 1ll << 32)) atomicOr(err, 1);
    cyc[blockIdx.x] = clock64() - t0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tb, 512);
}

int main() {
  int nsm = 0; cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  long long *cyc; int *err; cudaMalloc(&cyc, 8 * nsm); cudaMalloc(&err, 4); cudaMemset(err, 0, 4);
  const int sm = 200 * 1024 + 64;
  cudaFuncSetAttribute(k_bench<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(k_bench<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  struct Cfg { int kind, N, nacc, swz; };
  const Cfg cfgs[] = {{0, 192, 1, 0}, {0, 192, 2, 0}, {0, 96, 4, 0}, {0, 128, 4, 0}, {0, 192, 1, 1}, {0, 256, 1, 1},
                      {0, 96, 4, 1}, {1, 192, 1, 1}, {1, 256, 1, 1}, {1, 256, 2, 0}};
  for (const Cfg &g : cfgs) {
    const int iters = 20000, N = g.N;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
      cudaEventRecord(e0);
      if (g.kind == 0) k_bench<0><<<nsm, 128, sm>>>(N, iters, 4, g.nacc, g.swz, cyc, err);
      else k_bench<1><<<nsm, 128, sm>>>(N, iters, 4, g.nacc, g.swz, cyc, err);
      cudaEventRecord(e1);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) { printf("error %s\n", cudaGetErrorString(e)); return 1; }
      float ms; cudaEventElapsedTime(&ms, e0, e1);
      long long c0; cudaMemcpy(&c0, cyc, 8, cudaMemcpyDeviceToHost);
      const double K = g.kind == 0 ? 8 : 16;
      const double fl = 2.0 * 128 * N * K * iters;
      if (rep == 1)
        printf("%s M128 N%d K%.0f acc%d swz%d: %.0f cycles/MMA, %.0f FLOP/clk/SM, %.1f TFLOP/s (event %.3f ms)\n",
               g.kind == 0 ? "tf32" : "bf16", N, K, g.nacc, g.swz, (double)c0 / iters, fl / c0,
               fl * nsm / (ms * 1e-3) / 1e12, ms);
    }
  }
  int h = 0; cudaMemcpy(&h, err, 4, cudaMemcpyDeviceToHost);
  printf("err flag %d\n", h);
  return h;
}
