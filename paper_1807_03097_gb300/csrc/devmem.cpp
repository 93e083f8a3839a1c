// Device and pinned host memory of the library.
//
// Device buffers come from one CUDA memory pool per device and are allocated and freed in
// stream order on the context's stream (cudaMallocFromPoolAsync / cudaFreeAsync), so that
// creating, setting up and destroying a context never synchronises the device: a request of
// the serving loop that starts or ends does not stall the kernels of the others.  Freed
// blocks stay in the pool for later allocations (of any context) while a context or a server
// holds a reference on the device; when the last reference is dropped the pool is trimmed.
// The pool never makes an allocating stream wait for another stream's frees.
//
// Small pinned host buffers (residual mirrors of GMRES) are kept on a free list and reused
// across contexts instead of cudaMallocHost / cudaFreeHost per context.
#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "efie_internal.h"

namespace efie {

namespace {

constexpr int kMaxDevices = 64;

struct PoolTable {
  std::mutex mu;
  cudaMemPool_t pool[kMaxDevices] = {};
  int refs[kMaxDevices] = {};
};

PoolTable &pools() {
  static PoolTable t;
  return t;
}

struct PinnedList {
  std::mutex mu;
  std::vector<std::pair<void *, size_t>> free;
  std::unordered_map<void *, size_t> size;
};

PinnedList &pinned() {
  static PinnedList l;
  return l;
}

cudaError_t make_pool(int dev, cudaMemPool_t *out) {
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaError_t e = cudaMemPoolCreate(out, &props);
  if (e != cudaSuccess) return e;
  uint64_t keep = UINT64_MAX;  // freed memory stays in the pool until it is trimmed
  e = cudaMemPoolSetAttribute(*out, cudaMemPoolAttrReleaseThreshold, &keep);
  int no = 0;  // no cross-stream waits inserted to reuse another stream's freed block
  if (e == cudaSuccess) e = cudaMemPoolSetAttribute(*out, cudaMemPoolReuseAllowInternalDependencies, &no);
  return e;
}

}  // namespace

efie_status pool_ref(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return EFIE_EINVAL;
  PoolTable &T = pools();
  std::lock_guard<std::mutex> lk(T.mu);
  if (!T.pool[dev]) {
    cudaMemPool_t p = nullptr;
    if (make_pool(dev, &p) != cudaSuccess) return EFIE_ECUDA;
    T.pool[dev] = p;
  }
  ++T.refs[dev];
  return EFIE_OK;
}

void pool_unref(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return;
  PoolTable &T = pools();
  std::lock_guard<std::mutex> lk(T.mu);
  if (T.refs[dev] > 0 && --T.refs[dev] == 0 && T.pool[dev]) cudaMemPoolTrimTo(T.pool[dev], 0);
}

efie_status pool_alloc(Ctx *c, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool = nullptr;
  {
    PoolTable &T = pools();
    std::lock_guard<std::mutex> lk(T.mu);
    if (c->device >= 0 && c->device < kMaxDevices) pool = T.pool[c->device];
  }
  if (!pool) {
    c->err = "device memory pool not initialised";
    return EFIE_ECUDA;
  }
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->err = std::string("cudaMallocFromPoolAsync(") + std::to_string(bytes) + " B): " + cudaGetErrorString(e);
    *p = nullptr;
    return EFIE_ENOMEM;
  }
  std::lock_guard<std::mutex> lk(c->mem_mu);
  c->live[*p] = bytes;
  c->live_bytes += bytes;
  if (c->live_bytes > c->peak_bytes) c->peak_bytes = c->live_bytes;
  return EFIE_OK;
}

void pool_free(Ctx *c, void *p) {
  if (!p) return;
  cudaFreeAsync(p, c->stream);
  std::lock_guard<std::mutex> lk(c->mem_mu);
  auto it = c->live.find(p);
  if (it != c->live.end()) {
    c->live_bytes -= it->second;
    c->live.erase(it);
  }
}

void *pinned_get(size_t bytes) {
  PinnedList &L = pinned();
  {
    std::lock_guard<std::mutex> lk(L.mu);
    for (size_t i = 0; i < L.free.size(); ++i)
      if (L.free[i].second >= bytes) {
        void *q = L.free[i].first;
        L.free.erase(L.free.begin() + (long)i);
        return q;
      }
  }
  const size_t sz = bytes < 65536 ? 65536 : bytes;
  void *q = nullptr;
  if (cudaMallocHost(&q, sz) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(L.mu);
  L.size[q] = sz;
  return q;
}

void pinned_put(void *p) {
  if (!p) return;
  PinnedList &L = pinned();
  std::lock_guard<std::mutex> lk(L.mu);
  L.free.emplace_back(p, L.size[p]);
}

}  // namespace efie
