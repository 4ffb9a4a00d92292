// Kernel tracing: CUDA events around each launch, accumulated per kernel name;
// every launch also opens an NVTX range of the kernel's name for profilers.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pc.h"
#include "pc_internal.cuh"

namespace pcx {
namespace {

struct Entry {
  const char *name;
  uint64_t launches;
  double ms;
};
struct Pending {
  const char *name;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Entry> g_entries;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free;

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void add(const char *name, double ms) {
  for (auto &e : g_entries)
    if (std::strcmp(e.name, name) == 0) {
      e.launches += 1;
      e.ms += ms;
      return;
    }
  g_entries.push_back(Entry{name, 1, ms});
}

}  // namespace

TraceScope::TraceScope(const char *name, cudaStream_t st) : name_(name), st_(st), a_(nullptr), b_(nullptr) {
  nvtxRangePushA(name);  // a range per launch for profilers (no-op without one)
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  a_ = take_event();
  b_ = take_event();
  if (a_ && b_) cudaEventRecord(static_cast<cudaEvent_t>(a_), st_);
}

TraceScope::~TraceScope() {
  nvtxRangePop();
  if (!a_ || !b_) return;
  cudaEventRecord(static_cast<cudaEvent_t>(b_), st_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_pending.push_back(Pending{name_, static_cast<cudaEvent_t>(a_), static_cast<cudaEvent_t>(b_)});
}

bool trace_enabled() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

void trace_flush() {
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<Pending> keep;
  for (auto &p : g_pending) {
    if (cudaEventQuery(p.b) != cudaSuccess) {
      keep.push_back(p);
      continue;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) add(p.name, double(ms));
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.swap(keep);
  (void)cudaGetLastError();  // a pending query is not an error of the caller
}

}  // namespace pcx

extern "C" {

int pc_trace_enable(int on) {
  std::lock_guard<std::mutex> lk(pcx::g_mu);
  pcx::g_on = on != 0;
  return PC_OK;
}

int pc_trace_reset(void) {
  pcx::trace_flush();
  std::lock_guard<std::mutex> lk(pcx::g_mu);
  pcx::g_entries.clear();
  return PC_OK;
}

int pc_trace_count(void) {
  pcx::trace_flush();
  std::lock_guard<std::mutex> lk(pcx::g_mu);
  return int(pcx::g_entries.size());
}

int pc_trace_get(int i, const char **name, uint64_t *launches, double *total_ms) {
  std::lock_guard<std::mutex> lk(pcx::g_mu);
  if (i < 0 || size_t(i) >= pcx::g_entries.size() || !name || !launches || !total_ms) return PC_ERR_ARG;
  *name = pcx::g_entries[size_t(i)].name;
  *launches = pcx::g_entries[size_t(i)].launches;
  *total_ms = pcx::g_entries[size_t(i)].ms;
  return PC_OK;
}

}  // extern "C"
