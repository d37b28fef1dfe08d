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

namespace {

// Each thread reads its 16-byte words of the buffer `reps` times with loads
// cached in L2 only; the XOR of the words keeps the loads alive.
__global__ void __launch_bounds__(256)
    k_l2_read(const uint4* __restrict__ buf, size_t n16, int reps,
              unsigned long long* __restrict__ sink) {
  uint32_t acc = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
      const uint4 v = __ldcg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);
}

}  // namespace

}  // namespace hm

extern "C" {

uint64_t hm_launch_count(void) { return hm::launch_count_add(0); }

hm_status hm_l2_read_bandwidth(size_t bytes, int reps, double* gbs, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(gbs != nullptr, HM_EINVAL, "NULL result");
    HM_CHECK(bytes > 0 && bytes <= ((size_t)64 << 20) && bytes % 16 == 0, HM_EINVAL,
             "bytes must be a positive multiple of 16, at most 64 MiB");
    HM_CHECK(reps >= 1, HM_EINVAL, "reps must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)hm::k_l2_read, 256, 0));
    const unsigned blocks = (unsigned)(sms * (per > 0 ? per : 1));
    const size_t n16 = bytes / 16;
    hm::DBuf<unsigned char> buf(bytes + 256, s);
    unsigned long long* sink = reinterpret_cast<unsigned long long*>(buf.p + bytes);
    HM_CUDA(cudaMemsetAsync(buf.p, 0x5A, bytes + 256, s));
    const uint4* b = reinterpret_cast<const uint4*>(buf.p);
    hm::k_l2_read<<<blocks, 256, 0, s>>>(b, n16, 1, sink);
    HM_KCHECK();
    struct Events {  // destroyed on every exit
      cudaEvent_t a = nullptr, b = nullptr;
      ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
      }
    } ev;
    HM_CUDA(cudaEventCreate(&ev.a));
    HM_CUDA(cudaEventCreate(&ev.b));
    HM_CUDA(cudaEventRecord(ev.a, s));
    hm::k_l2_read<<<blocks, 256, 0, s>>>(b, n16, reps, sink);
    HM_KCHECK();
    HM_CUDA(cudaEventRecord(ev.b, s));
    HM_CUDA(cudaEventSynchronize(ev.b));
    float ms = 0.f;
    HM_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
    *gbs = (double)bytes * reps / (ms * 1e-3) / 1e9;
  });
}

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
