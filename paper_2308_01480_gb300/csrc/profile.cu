// Kernel accounting for benchmarks: launch counts per kernel family and,
// optionally, CUDA-event durations with algorithmic bytes and flops.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace ttr {

namespace {
struct Acc {
  int64_t launches = 0;
  double ms = 0, bytes = 0, flops = 0;
};
struct Rec {
  std::string fam;
  cudaEvent_t a, b;
};
std::mutex g_mu;
std::atomic<bool> g_on{false};
bool g_timing = false;
std::map<std::string, Acc> g_acc;
std::vector<Rec> g_recs;
}  // namespace

void note_launch(const char* family, int count) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_acc[family].launches += count;
}

ProfScope::ProfScope(const char* family, cudaStream_t st, double bytes, double flops)
    : fam_(family), st_(st) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Acc& a = g_acc[family];
  a.bytes += bytes;
  a.flops += flops;
  if (g_timing && cudaEventCreate(&a_) == cudaSuccess && cudaEventCreate(&b_) == cudaSuccess) {
    cudaEventRecord(a_, st);
    timed_ = true;
  }
}

ProfScope::~ProfScope() {
  if (!timed_) return;
  cudaEventRecord(b_, st_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({fam_, a_, b_});
}

cudaError_t raise_smem_limit_ptr(const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, cudaError_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find({dev, kernel});
  if (it != done.end()) return it->second;
  cudaFuncAttributes fa;
  int optin = 0;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  done[{dev, kernel}] = e;
  return e;
}

}  // namespace ttr

extern "C" {

tt_status tt_rbki_profile_begin(int event_timing) {
  std::lock_guard<std::mutex> lk(ttr::g_mu);
  for (auto& r : ttr::g_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ttr::g_recs.clear();
  ttr::g_acc.clear();
  ttr::g_timing = event_timing != 0;
  ttr::g_on.store(true);
  return TT_OK;
}

tt_status tt_rbki_profile_end(tt_kernel_stat* stats, int max_stats, int* n_stats) {
  ttr::g_on.store(false);
  std::lock_guard<std::mutex> lk(ttr::g_mu);
  for (auto& r : ttr::g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
      ttr::g_acc[r.fam].ms += ms;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ttr::g_recs.clear();
  std::vector<std::pair<std::string, ttr::Acc>> v(ttr::g_acc.begin(), ttr::g_acc.end());
  std::sort(v.begin(), v.end(), [](const auto& x, const auto& y) { return x.second.ms > y.second.ms; });
  int n = 0;
  for (auto& kv : v) {
    if (stats && n < max_stats) {
      tt_kernel_stat& s = stats[n];
      std::memset(&s, 0, sizeof(s));
      std::strncpy(s.name, kv.first.c_str(), sizeof(s.name) - 1);
      s.launches = kv.second.launches;
      s.ms = kv.second.ms;
      s.bytes = kv.second.bytes;
      s.flops = kv.second.flops;
    }
    ++n;
  }
  if (n_stats) *n_stats = std::min(n, max_stats);
  return TT_OK;
}

}  // extern "C"
