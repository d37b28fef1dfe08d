// Device primitives used by graph ingest: exclusive scan, stable LSD radix
// sort (8-bit digits, warp-match ranking), unique, CSR offsets.
#include <mutex>

#include <atomic>

#include "hm_internal.cuh"

namespace hm {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_IPT;

template <class T>
__device__ T block_exclusive_scan(T v, T* warp_tot, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : T(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  T before = warp > 0 ? warp_tot[warp - 1] : T(0);
  if (total) *total = warp_tot[SCAN_THREADS / 32 - 1];
  return before + x - v;
}

// per-tile sums
template <class T>
__global__ void k_tile_sums(const T* in, int64_t n, T* sums) {
  __shared__ T wt[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  T s = 0;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
    int64_t idx = base + i;
    if (idx < n) s += in[idx];
  }
  T tot;
  block_exclusive_scan<T>(s, wt, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// exclusive scan of a tile plus the tile's offset; the last tile also writes out[n]
template <class T>
__global__ void k_tile_scan(const T* in, T* out, int64_t n, const T* tile_off) {
  __shared__ T buf[SCAN_TILE];
  __shared__ T wt[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
    int64_t idx = base + i;
    buf[i] = idx < n ? in[idx] : T(0);
  }
  __syncthreads();
  T loc[SCAN_IPT];
  T s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j) {
    loc[j] = buf[threadIdx.x * SCAN_IPT + j];
    s += loc[j];
  }
  T tot;
  T run = block_exclusive_scan<T>(s, wt, &tot) + (tile_off ? tile_off[blockIdx.x] : T(0));
  __syncthreads();
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j) {
    buf[threadIdx.x * SCAN_IPT + j] = run;
    run += loc[j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = buf[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    out[n] = (tile_off ? tile_off[blockIdx.x] : T(0)) + tot;
}

template <class T>
void scan_exclusive(const T* in, T* out, int64_t n, cudaStream_t s) {
  if (n == 0) {
    HM_CUDA(cudaMemsetAsync(out, 0, sizeof(T), s));
    return;
  }
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  HM_CHECK(tiles < (1ll << 31), HM_EINVAL, "scan too large");
  if (tiles == 1) {
    k_tile_scan<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
    HM_KCHECK();
    return;
  }
  DBuf<T> sums(tiles, s), offs(tiles + 1, s);
  k_tile_sums<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums.p);
  HM_KCHECK();
  scan_exclusive<T>(sums.p, offs.p, tiles, s);
  k_tile_scan<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, offs.p);
  HM_KCHECK();
}

// Same scan with its tile sums / offsets carved from caller scratch.
template <class T>
void scan_exclusive_in(const T* in, T* out, int64_t n, cudaStream_t s, T* scratch,
                       size_t scratch_elems) {
  if (n == 0) {
    HM_CUDA(cudaMemsetAsync(out, 0, sizeof(T), s));
    return;
  }
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    k_tile_scan<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
    HM_KCHECK();
    return;
  }
  HM_CHECK((size_t)(2 * tiles + 1) <= scratch_elems, HM_EINVAL, "scan scratch too small");
  T* sums = scratch;
  T* offs = scratch + tiles;
  k_tile_sums<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums);
  HM_KCHECK();
  scan_exclusive_in<T>(sums, offs, tiles, s, scratch + 2 * tiles + 1,
                       scratch_elems - (size_t)(2 * tiles + 1));
  k_tile_scan<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, offs);
  HM_KCHECK();
}

unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

}  // namespace

uint64_t* pinned_words() {
  thread_local uint64_t* p = nullptr;
  if (!p) HM_CUDA(cudaMallocHost((void**)&p, 512 * sizeof(uint64_t)));
  return p;
}

// ------------------------------------------------------------------ fork-join
namespace {
std::mutex g_side_mu;
cudaStream_t g_side[64][Fork::kSide] = {};

// Events of this host thread on one device, created once: [0] marks the
// fork, [1 + i] the end of side stream i.
struct ForkEvents {
  cudaEvent_t e[1 + Fork::kSide] = {};
};
ForkEvents& fork_events(int dev) {
  thread_local ForkEvents ev[64];
  ForkEvents& f = ev[dev];
  if (!f.e[0])
    for (auto& e : f.e) HM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return f;
}
}  // namespace

// hm_serialize_launches: forked work runs in order on the parent stream
std::atomic<bool> g_serial{false};

Fork::Fork(cudaStream_t s, int w) : main(s), width(w < 1 ? 1 : w > kSide ? kSide : w) {
  if (g_serial.load(std::memory_order_relaxed)) {
    for (int i = 0; i < kSide; ++i) side[i] = main;
    width = 0;
    return;
  }
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev));
  HM_CHECK(dev >= 0 && dev < 64, HM_ECUDA, "device ordinal above 63");
  {
    std::lock_guard<std::mutex> lock(g_side_mu);
    for (int i = 0; i < kSide; ++i) {
      if (!g_side[dev][i])
        HM_CUDA(cudaStreamCreateWithFlags(&g_side[dev][i], cudaStreamNonBlocking));
      side[i] = g_side[dev][i];
    }
  }
  ForkEvents& ev = fork_events(dev);
  HM_CUDA(cudaEventRecord(ev.e[0], main));
  for (int i = 0; i < width; ++i) HM_CUDA(cudaStreamWaitEvent(side[i], ev.e[0], 0));
}

void Fork::join() {
  if (joined) return;
  joined = true;
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev));
  ForkEvents& ev = fork_events(dev);
  for (int i = 0; i < width; ++i) {
    HM_CUDA(cudaEventRecord(ev.e[1 + i], side[i]));
    HM_CUDA(cudaStreamWaitEvent(main, ev.e[1 + i], 0));
  }
}

Fork::~Fork() {
  if (joined) return;
  joined = true;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  ForkEvents& ev = fork_events(dev);
  for (int i = 0; i < width; ++i)
    if (cudaEventRecord(ev.e[1 + i], side[i]) == cudaSuccess)
      cudaStreamWaitEvent(main, ev.e[1 + i], 0);
}

void scan_exclusive_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s) {
  scan_exclusive<uint64_t>(in, out, n, s);
}
void scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s) {
  scan_exclusive<uint32_t>(in, out, n, s);
}
void scan_exclusive_u64_in(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s,
                           uint64_t* scratch, size_t scratch_elems) {
  scan_exclusive_in<uint64_t>(in, out, n, s, scratch, scratch_elems);
}
size_t scan_scratch_elems(int64_t n) {
  // tile sums + offsets at every level of the recursion
  size_t need = 0;
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  while (tiles > 1) {
    need += (size_t)(2 * tiles + 1);
    tiles = (tiles + SCAN_TILE - 1) / SCAN_TILE;
  }
  return need;
}

}  // namespace hm

extern "C" hm_status hm_serialize_launches(int on) {
  hm::g_serial.store(on != 0);
  return HM_OK;
}
