// Cached launch shapes (see resident_shape_of in common.cuh).
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace wh {

cudaError_t resident_shape_of(const void* kernel, int threads, size_t smem, ResidentShape* out) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, size_t>, ResidentShape> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(kernel, dev, threads, smem);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out = it->second;
      return cudaSuccess;
    }
  }
  ResidentShape r{148, 1};
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&r.nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = r;
  }
  *out = r;
  return cudaSuccess;
}

}  // namespace wh
