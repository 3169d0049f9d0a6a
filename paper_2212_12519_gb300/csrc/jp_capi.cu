// Error reporting and small host utilities of the C ABI.
#include <cuda_runtime.h>

#include <atomic>
#include <string>

#include "jp_internal.cuh"

namespace jp {

namespace {
thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};
}

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return JP_ERR_CUDA;
}

void clear_error() { g_err.clear(); }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 152;
  return n;
}

}  // namespace jp

extern "C" const char* jp_last_error(void) { return jp::g_err.c_str(); }

extern "C" uint64_t jp_launch_count(void) { return jp::g_launches.load(std::memory_order_relaxed); }

extern "C" const char* jp_version(void) { return "libjoseph 0.1 (sm_103a)"; }
