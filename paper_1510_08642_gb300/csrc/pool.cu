// Workspace pool of the library (no counterpart in the paper): every
// temporary of a call (the recursion's S / T / P buffers, INT8 planes and
// products, LU scratch, batch plans) is taken from one stream-ordered memory
// pool per device that the library owns, apart from the device's default pool
// and from the caller's allocator.
//
// By default the pool keeps nothing between calls (release threshold 0:
// unused memory goes back to the device at the next synchronisation), like
// a plain cudaMallocAsync. A service that wants its temporaries mapped ahead
// of time reserves a size: the threshold is raised to it and the pool grown
// to it at once, so later calls are served without mapping new memory.
#include <mutex>
#include <string>

#include "kernels.cuh"

namespace ddg {

namespace {

constexpr int kMaxDev = 64;
std::mutex g_mu;
cudaMemPool_t g_pools[kMaxDev];
bool g_made[kMaxDev];

ddg_status pool_of(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= kMaxDev) return set_error(DDG_EINVAL, "workspace: device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_made[dev]) {
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || dev >= count) {
      cudaGetLastError();
      return set_error(DDG_EINVAL, "workspace: no device " + std::to_string(dev));
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&g_pools[dev], &props);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(DDG_ECUDA, std::string("workspace: cudaMemPoolCreate: ") + cudaGetErrorString(e));
    }
    g_made[dev] = true;
  }
  *out = g_pools[dev];
  return DDG_OK;
}

}  // namespace

cudaError_t ws_alloc(void** p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  if (pool_of(dev, &pool) != DDG_OK) return cudaErrorInvalidDevice;
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t ws_free(void* p, cudaStream_t s) { return cudaFreeAsync(p, s); }

}  // namespace ddg

extern "C" {

ddg_status ddg_workspace_reserve(int32_t device, uint64_t bytes) {
  using namespace ddg;
  clear_error();
  cudaMemPool_t pool;
  ddg_status st = pool_of(device, &pool);
  if (st != DDG_OK) return st;
  unsigned long long thr = bytes;
  cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(DDG_ECUDA, std::string("workspace: release threshold: ") + cudaGetErrorString(e));
  }
  unsigned long long have = 0;
  cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &have);
  if (bytes == 0 || have >= bytes) return DDG_OK;
  // grow the pool now: one allocation of the reserved size, freed at once
  int prev = 0;
  cudaGetDevice(&prev);
  if ((e = cudaSetDevice(device)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(DDG_ECUDA, std::string("workspace: cudaSetDevice: ") + cudaGetErrorString(e));
  }
  cudaStream_t s = nullptr;
  void* p = nullptr;
  st = DDG_OK;
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) {
    st = set_error(DDG_ECUDA, std::string("workspace: stream: ") + cudaGetErrorString(e));
  } else if ((e = cudaMallocFromPoolAsync(&p, bytes, pool, s)) != cudaSuccess) {
    st = set_error(DDG_ENOMEM, "workspace: cannot reserve " + std::to_string(bytes) + " bytes: " +
                                   cudaGetErrorString(e));
  } else if ((e = cudaFreeAsync(p, s)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    st = set_error(DDG_ECUDA, std::string("workspace: ") + cudaGetErrorString(e));
  }
  if (st != DDG_OK) {
    cudaGetLastError();
    thr = 0;  // a failed reservation holds nothing
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  return st;
}

ddg_status ddg_workspace_release(int32_t device) {
  using namespace ddg;
  clear_error();
  cudaMemPool_t pool;
  ddg_status st = pool_of(device, &pool);
  if (st != DDG_OK) return st;
  unsigned long long thr = 0;
  cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(DDG_ECUDA, std::string("workspace: release: ") + cudaGetErrorString(e));
  }
  return DDG_OK;
}

ddg_status ddg_workspace_stats(int32_t device, ddg_workspace_info* out) {
  using namespace ddg;
  clear_error();
  if (!out) return set_error(DDG_EINVAL, "workspace: out is null");
  cudaMemPool_t pool;
  ddg_status st = pool_of(device, &pool);
  if (st != DDG_OK) return st;
  unsigned long long v[4] = {0, 0, 0, 0};
  const cudaMemPoolAttr attr[4] = {cudaMemPoolAttrReservedMemCurrent, cudaMemPoolAttrUsedMemCurrent,
                                   cudaMemPoolAttrReleaseThreshold, cudaMemPoolAttrUsedMemHigh};
  for (int i = 0; i < 4; ++i) {
    cudaError_t e = cudaMemPoolGetAttribute(pool, attr[i], &v[i]);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(DDG_ECUDA, std::string("workspace: stats: ") + cudaGetErrorString(e));
    }
  }
  out->reserved_bytes = v[0];
  out->used_bytes = v[1];
  out->threshold_bytes = v[2];
  out->used_high_bytes = v[3];
  return DDG_OK;
}

}  // extern "C"
