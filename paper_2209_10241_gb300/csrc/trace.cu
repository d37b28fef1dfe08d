// Kernel timing trace: when enabled, each census kernel launch and each ingest
// phase is bracketed by CUDA events recorded on the stream it is launched on,
// so a caller can attribute device time to kernels without a profiler.
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

#include "hm_internal.cuh"

namespace hm {
namespace {

struct Entry {
  const char* name;
  cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Entry> g_entries;
std::vector<cudaEvent_t> g_pool;  // events read back, reused by later spans

cudaEvent_t take_event() {
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_pool.empty()) {
      cudaEvent_t e = g_pool.back();
      g_pool.pop_back();
      return e;
    }
  }
  cudaEvent_t e;
  HM_CUDA(cudaEventCreate(&e));
  return e;
}

}  // namespace

std::string g_only;  // traced span name; empty = every span

bool trace_on(const char* name) {
  if (!g_on) return false;
  std::lock_guard<std::mutex> lock(g_mu);
  return g_only.empty() || (name && g_only == name);
}

static std::atomic<uint64_t> g_launches{0};
uint64_t launch_count_add(uint64_t n) { return g_launches.fetch_add(n) + n; }

void trace_begin(cudaStream_t s, cudaEvent_t* a) {
  *a = take_event();
  HM_CUDA(cudaEventRecord(*a, s));
}

void trace_end(const char* name, cudaStream_t s, cudaEvent_t a) {
  cudaEvent_t b = take_event();
  HM_CUDA(cudaEventRecord(b, s));
  std::lock_guard<std::mutex> lock(g_mu);
  g_entries.push_back(Entry{name, a, b});
}

}  // namespace hm

extern "C" {

uint64_t hm_launch_count(void) { return hm::launch_count_add(0); }

hm_status hm_trace_enable(int on) {
  return hm::guarded([&] {
    std::lock_guard<std::mutex> lock(hm::g_mu);
    hm::g_on = on != 0;
  });
}

hm_status hm_trace_only(const char* name) {
  return hm::guarded([&] {
    std::lock_guard<std::mutex> lock(hm::g_mu);
    hm::g_only = name ? name : "";
  });
}

hm_status hm_trace_read(int max_entries, char* names, int name_len, float* ms, int* count) {
  return hm::guarded([&] {
    HM_CHECK(count, HM_EINVAL, "NULL count");
    std::lock_guard<std::mutex> lock(hm::g_mu);
    int n = 0;
    for (auto& e : hm::g_entries) {
      if (n < max_entries) {
        float t = 0.f;
        HM_CUDA(cudaEventSynchronize(e.b));
        HM_CUDA(cudaEventElapsedTime(&t, e.a, e.b));
        if (ms) ms[n] = t;
        if (names && name_len > 0) {
          std::strncpy(names + (size_t)n * name_len, e.name, name_len - 1);
          names[(size_t)n * name_len + name_len - 1] = 0;
        }
        ++n;
      }
      hm::g_pool.push_back(e.a);
      hm::g_pool.push_back(e.b);
    }
    hm::g_entries.clear();
    *count = n;
  });
}

}  // extern "C"
