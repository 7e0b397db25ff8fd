// Cached launch shapes (see resident_shape_of in common.cuh).
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace wh {

cudaError_t resident_shape_of(const void* kernel, int threads, size_t smem, ResidentShape* out,
                              int carveout) {
  // The dynamic shared-memory limit is a property of the kernel, so it is only
  // ever raised, to the largest size requested for that kernel on that device;
  // every cached launch shape then stays launchable.
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, size_t>, ResidentShape> cache;
  static std::map<std::pair<const void*, int>, size_t> smem_limit;
  static std::map<std::pair<const void*, int>, int> carve;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(kernel, dev, threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  if (carveout >= 0) {
    int& c = carve[std::make_pair(kernel, dev)];
    if (c != carveout + 1) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
      if (e != cudaSuccess) return e;
      c = carveout + 1;
    }
  }
  size_t& limit = smem_limit[std::make_pair(kernel, dev)];
  if (smem > limit) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    limit = smem;
  }
  ResidentShape r{148, 1};
  e = cudaDeviceGetAttribute(&r.nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r.per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  cache[key] = r;
  *out = r;
  return cudaSuccess;
}

}  // namespace wh
