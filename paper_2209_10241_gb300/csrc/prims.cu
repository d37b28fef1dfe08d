// Device primitives used by graph ingest: exclusive scan, stable LSD radix
// sort (8-bit digits, warp-match ranking), unique, CSR offsets.
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

// ------------------------------------------------------------------ radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_IPT = 8;
constexpr int RS_TILE = RS_THREADS * RS_IPT;

__global__ void k_rs_hist(const uint64_t* src, int shift, int64_t n, uint32_t* counts, int nb) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    int64_t idx = base + i;
    if (idx < n) atomicAdd(&h[(src[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: the rank of an item among equal digits of its tile is the
// count in earlier warps + earlier iterations of its warp + earlier lanes.
__global__ void k_rs_scatter(const uint64_t* src, int shift, const uint64_t* a, const uint64_t* b,
                             uint64_t* a2, uint64_t* b2, int64_t n, const uint32_t* offs, int nb) {
  __shared__ uint32_t wcnt[RS_WARPS][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE + warp * (32 * RS_IPT);
  const unsigned lt = (1u << lane) - 1u;
  uint32_t dig[RS_IPT], rank[RS_IPT];
#pragma unroll
  for (int it = 0; it < RS_IPT; ++it) {
    int64_t idx = base + it * 32 + lane;
    bool valid = idx < n;
    uint32_t d = valid ? (uint32_t)((src[idx] >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = valid ? wcnt[warp][d] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
    dig[it] = d;
    rank[it] = before + __popc(peers & lt);
  }
  __syncthreads();
  {
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      uint32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < RS_IPT; ++it) {
    int64_t idx = base + it * 32 + lane;
    if (idx < n) {
      uint32_t d = dig[it];
      uint64_t pos = (uint64_t)offs[(int64_t)d * nb + blockIdx.x] + wcnt[warp][d] + rank[it];
      a2[pos] = a[idx];
      if (b) b2[pos] = b[idx];
    }
  }
}

// passes: (array index 0 = a / 1 = b, shift)
void radix_core(uint64_t* a, uint64_t* b, int64_t n, const std::vector<std::pair<int, int>>& passes,
                cudaStream_t s) {
  if (n <= 1 || passes.empty()) return;
  HM_CHECK(n < (1ll << 31), HM_EINVAL, "radix sort input too large");
  const int nb = (int)((n + RS_TILE - 1) / RS_TILE);
  DBuf<uint64_t> ta(n, s), tb(b ? n : 0, s);
  DBuf<uint32_t> counts((size_t)256 * nb, s), offs((size_t)256 * nb + 1, s);
  uint64_t *ca = a, *cb = b, *na = ta.p, *nb_ = tb.p;
  for (auto& ps : passes) {
    const uint64_t* src = ps.first == 0 ? ca : cb;
    k_rs_hist<<<nb, RS_THREADS, 0, s>>>(src, ps.second, n, counts.p, nb);
    HM_KCHECK();
    scan_exclusive<uint32_t>(counts.p, offs.p, (int64_t)256 * nb, s);
    k_rs_scatter<<<nb, RS_THREADS, 0, s>>>(src, ps.second, ca, cb, na, nb_, n, offs.p, nb);
    HM_KCHECK();
    std::swap(ca, na);
    std::swap(cb, nb_);
  }
  if (ca != a) {
    HM_CUDA(cudaMemcpyAsync(a, ca, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    if (b) HM_CUDA(cudaMemcpyAsync(b, cb, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  }
}

__global__ void k_unique_flags(const uint64_t* hi, const uint64_t* lo, int64_t n, uint32_t* f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    bool keep = i == 0 || lo[i] != lo[i - 1] || (hi && hi[i] != hi[i - 1]);
    f[i] = keep ? 1u : 0u;
  }
}

__global__ void k_unique_scatter(const uint64_t* hi, const uint64_t* lo, int64_t n,
                                 const uint32_t* f, const uint32_t* pos, uint64_t* hi2,
                                 uint64_t* lo2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (f[i]) {
      lo2[pos[i]] = lo[i];
      if (hi) hi2[pos[i]] = hi[i];
    }
  }
}

__global__ void k_set_u32(uint32_t* p, uint32_t v) { *p = v; }

__global__ void k_csr_offsets(const uint64_t* keys, int64_t n, int shift, int32_t nn,
                              int64_t* off) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t cur = i < n ? (int64_t)(keys[i] >> shift) : (int64_t)nn;
    int64_t prev = i > 0 ? (int64_t)(keys[i - 1] >> shift) : -1;
    for (int64_t v = prev + 1; v <= cur && v <= nn; ++v) off[v] = i;
  }
}

unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

}  // namespace

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

void radix_sort_u64(uint64_t* keys, uint64_t* vals, int64_t n, int bits, cudaStream_t s) {
  std::vector<std::pair<int, int>> passes;
  for (int sh = 0; sh < bits; sh += 8) passes.push_back({0, sh});
  radix_core(keys, vals, n, passes, s);
}

void radix_sort_u128(uint64_t* hi, uint64_t* lo, int64_t n, int hi_bits, int lo_bits,
                     cudaStream_t s) {
  std::vector<std::pair<int, int>> passes;
  for (int sh = 0; sh < lo_bits; sh += 8) passes.push_back({0, sh});
  for (int sh = 0; sh < hi_bits; sh += 8) passes.push_back({1, sh});
  radix_core(lo, hi, n, passes, s);
}

int64_t unique_sorted(uint64_t* hi, uint64_t* lo, int64_t n, cudaStream_t s) {
  if (n <= 1) return n;
  DBuf<uint32_t> f(n, s), pos(n + 1, s);
  DBuf<uint64_t> lo2(n, s), hi2(hi ? n : 0, s);
  k_unique_flags<<<grid_for(n, 256), 256, 0, s>>>(hi, lo, n, f.p);
  HM_KCHECK();
  scan_exclusive<uint32_t>(f.p, pos.p, n, s);
  k_unique_scatter<<<grid_for(n, 256), 256, 0, s>>>(hi, lo, n, f.p, pos.p, hi2.p, lo2.p);
  HM_KCHECK();
  uint32_t kept = 0;
  HM_CUDA(cudaMemcpyAsync(&kept, pos.p + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  HM_CUDA(cudaMemcpyAsync(lo, lo2.p, kept * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  if (hi) HM_CUDA(cudaMemcpyAsync(hi, hi2.p, kept * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  return kept;
}

void unique_sorted_async(uint64_t* hi, uint64_t* lo, int64_t n, uint32_t* d_kept,
                         cudaStream_t s) {
  if (n <= 1) {
    k_set_u32<<<1, 1, 0, s>>>(d_kept, (uint32_t)n);
    HM_KCHECK();
    return;
  }
  DBuf<uint32_t> f(n, s), pos(n + 1, s);
  DBuf<uint64_t> lo2(n, s), hi2(hi ? n : 0, s);
  k_unique_flags<<<grid_for(n, 256), 256, 0, s>>>(hi, lo, n, f.p);
  HM_KCHECK();
  scan_exclusive<uint32_t>(f.p, pos.p, n, s);
  k_unique_scatter<<<grid_for(n, 256), 256, 0, s>>>(hi, lo, n, f.p, pos.p, hi2.p, lo2.p);
  HM_KCHECK();
  HM_CUDA(cudaMemcpyAsync(d_kept, pos.p + n, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  // the first `kept` entries are the distinct keys; the rest is left over
  HM_CUDA(cudaMemcpyAsync(lo, lo2.p, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  if (hi) HM_CUDA(cudaMemcpyAsync(hi, hi2.p, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
}

void csr_offsets(const uint64_t* keys, int64_t n, int shift, int32_t num_nodes, int64_t* off,
                 cudaStream_t s) {
  k_csr_offsets<<<grid_for(n + 1, 256), 256, 0, s>>>(keys, n, shift, num_nodes, off);
  HM_KCHECK();
}

}  // namespace hm
