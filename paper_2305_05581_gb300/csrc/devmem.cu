// devmem.cu -- device memory accounting of the library.
//
// Every device allocation of the library goes through dmalloc / dfree.  They
// keep the bytes in use per device (and the high-water mark), and refuse,
// before cudaMalloc is called, an allocation that would take the device above
// its budget (tns_set_memory_budget; 0 = no budget).  The engine reads these
// numbers to decide when to move operator catalogues off the device.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "cuda_backend.h"

namespace tns {

namespace {
constexpr int kMaxDev = 64;
struct DevMemState {
  std::mutex mu;
  std::unordered_map<void*, std::pair<int, size_t>> live;  // pointer -> (device, bytes)
  long long used[kMaxDev] = {};
  long long peak[kMaxDev] = {};
  long long budget[kMaxDev] = {};
};
DevMemState& state() {
  static DevMemState s;
  return s;
}
int cur_dev() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDev) d = 0;
  return d;
}
}  // namespace

cudaError_t dmalloc_raw(void** p, size_t bytes) {
  *p = nullptr;
  const int dev = cur_dev();
  DevMemState& s = state();
  {
    std::lock_guard<std::mutex> g(s.mu);
    if (s.budget[dev] > 0 && s.used[dev] + (long long)bytes > s.budget[dev]) return cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> g(s.mu);
  s.live[*p] = {dev, bytes};
  s.used[dev] += (long long)bytes;
  if (s.used[dev] > s.peak[dev]) s.peak[dev] = s.used[dev];
  return cudaSuccess;
}

void dfree(void* p) {
  if (!p) return;
  DevMemState& s = state();
  {
    std::lock_guard<std::mutex> g(s.mu);
    auto it = s.live.find(p);
    if (it != s.live.end()) {
      s.used[it->second.first] -= (long long)it->second.second;
      s.live.erase(it);
    }
  }
  cudaFree(p);
}

DevMem dmem(int dev) {
  DevMem m;
  if (dev < 0 || dev >= kMaxDev) return m;
  DevMemState& s = state();
  std::lock_guard<std::mutex> g(s.mu);
  m.used = s.used[dev];
  m.peak = s.peak[dev];
  m.budget = s.budget[dev];
  return m;
}

void dmem_set_budget(int dev, long long bytes) {
  if (dev < 0 || dev >= kMaxDev) return;
  DevMemState& s = state();
  std::lock_guard<std::mutex> g(s.mu);
  s.budget[dev] = bytes > 0 ? bytes : 0;
}

void dmem_reset_peak(int dev) {
  if (dev < 0 || dev >= kMaxDev) return;
  DevMemState& s = state();
  std::lock_guard<std::mutex> g(s.mu);
  s.peak[dev] = s.used[dev];
}

}  // namespace tns
