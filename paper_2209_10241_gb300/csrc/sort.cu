// Batched stable LSD radix sort (8-bit digits) with an optional unique +
// unpack step, for up to SORT_MAX_JOBS independent key arrays at once.
//
// One launch takes the digit histograms of every pass of every job (a
// digit's total does not depend on the key order); then one launch per pass
// index serves every job that still has a pass, each tile finding its offset
// for every digit by decoupled look-back over the tiles before it; a final
// launch drops repeated keys (again with look-back, for the output position)
// and writes the kept keys in their final layout. Temporaries come from one
// allocation, so a batch costs a handful of runtime calls whatever its size.
//
// Tiles take ids from an atomic counter in the order their blocks start, so a
// tile only ever waits on tiles that already run; every wait is still bounded
// and one that gives up counts into g_wait_timeouts (read by the host).
#include <algorithm>
#include <atomic>
#include <vector>

#include "hm_internal.cuh"

namespace hm {

// device-side bounded waits that gave up (see look_back)
__device__ unsigned int g_wait_timeouts;

namespace {

constexpr int SORT_MAX_JOBS = 4;
constexpr int SORT_MAX_PASSES = 16;
constexpr int TPB = 256;               // threads per block
constexpr int IPT = 8;                 // keys per thread
constexpr int TILE = TPB * IPT;        // keys per tile
constexpr uint64_t ST_AGG = 1ull << 62, ST_PREFIX = 2ull << 62, ST_VALUE = (1ull << 62) - 1;
constexpr uint32_t SPIN_LIMIT = 1u << 20;
// back-off between polls of a status word that is not published yet, so
// that waiting tiles leave issue slots to the tiles they wait on and to
// kernels running beside the sort (0: poll without pause; with 100 ns a
// build + order-4 census of 10^6 nodes and 2*10^6 hyperedges went from 2.139
// to 2.131 ms)
#ifndef HM_LB_SLEEP_NS
#define HM_LB_SLEEP_NS 100
#endif

struct JobDev {
  uint64_t* a[2];  // primary word: [0] = caller's array, [1] = temporary
  uint64_t* b[2];  // second word (high key word or values), may be null
  int64_t n, tiles;
  int np;
  int8_t arr[SORT_MAX_PASSES];
  int8_t shift[SORT_MAX_PASSES];
  int b_is_key;       // unique compares b too
  int unique;         // 0: sort only
  int unpack;         // SortJob::Unpack
  int member_bits;
  void* out;
  uint64_t* out_b;
  uint32_t* d_kept;
  uint32_t* ghist;    // [np][256]
  uint32_t* gbase;    // [np][256]
  uint64_t* status[2];  // [tiles][256] per pass parity
  uint64_t* ustatus;    // [tiles] for unique
  uint32_t* ctr;        // [np + 1] tile tickets (last one: unique)
  uint32_t* rank;       // small jobs: [n] ranks (zeroed)
};

struct Batch {
  int nj;
  JobDev j[SORT_MAX_JOBS];
};

// Blocks of a launch covering several jobs: job k owns blocks [first[k], first[k+1]).
struct Grid {
  int nj;
  int job[SORT_MAX_JOBS];
  int8_t on_b[SORT_MAX_JOBS];   // pass launches: digit of word b
  int8_t shift[SORT_MAX_JOBS];  // pass launches: digit shift
  int64_t first[SORT_MAX_JOBS + 1];
};

// Grid entry e of block blk: its job is G.job[e], its blocks G.first[e]..G.first[e+1).
__device__ __forceinline__ int grid_entry(const Grid& G, int64_t blk) {
  int e = 0;
  while (e + 1 < G.nj && blk >= G.first[e + 1]) ++e;
  return e;
}

__device__ __forceinline__ uint64_t ld_status(const uint64_t* p) {
  return *(const volatile uint64_t*)p;
}
__device__ __forceinline__ void st_status(uint64_t* p, uint64_t v) { *(volatile uint64_t*)p = v; }

// Sum of the values published by tiles before `tile` (tile >= 1) in a
// [tiles][stride] status array, column col: aggregates are added until an
// inclusive prefix is met. With HM_LB_WINDOW > 1 the words of that many tiles
// are read at once (independent loads), so a walk over w tiles costs about
// w / HM_LB_WINDOW memory round trips.
#ifndef HM_LB_WINDOW
#define HM_LB_WINDOW 1
#endif
__device__ uint64_t look_back(const uint64_t* status, int64_t tile, int stride, int col) {
  uint64_t excl = 0;
  int64_t j = tile - 1;
  uint32_t spins = 0;
  while (j >= 0) {
    uint64_t v[HM_LB_WINDOW];
#pragma unroll
    for (int k = 0; k < HM_LB_WINDOW; ++k)  // before tile 0: an inclusive prefix of 0
      v[k] = j - k >= 0 ? ld_status(status + (j - k) * stride + col) : ST_PREFIX;
    bool stop = false, done = false;
    int used = 0;
#pragma unroll
    for (int k = 0; k < HM_LB_WINDOW; ++k) {
      if (stop) continue;
      if ((v[k] & ~ST_VALUE) == 0) {  // not published yet: read it again
        stop = true;
      } else {
        excl += v[k] & ST_VALUE;
        ++used;
        if (v[k] & ST_PREFIX) stop = done = true;
      }
    }
    if (done) break;
    if (used == 0) {
      if (++spins > SPIN_LIMIT) {  // cannot happen with in-order tile tickets
        atomicAdd(&g_wait_timeouts, 1u);
        break;
      }
      if (HM_LB_SLEEP_NS) __nanosleep(HM_LB_SLEEP_NS);
    }
    j -= used;
  }
  return excl;
}

// Warp-wide look-back for one status word per tile (stride 1): lanes read the
// 32 tiles before the window's end at once; the sum of their aggregates up to
// the nearest inclusive prefix is the tile's exclusive prefix. All 32 lanes of
// the calling warp must call it; every lane gets the result. Bounded like
// look_back.
__device__ uint64_t look_back_warp(const uint64_t* status, int64_t tile) {
  const int lane = threadIdx.x & 31;
  uint64_t excl = 0;
  int64_t end = tile;  // window: tiles [end - 32, end)
  uint32_t spins = 0;
  while (end > 0) {
    const int64_t j = end - 1 - lane;
    uint64_t v = j >= 0 ? ld_status(status + j) : ST_PREFIX;  // before tile 0: prefix 0
    // wait until every tile of the window has published something
    while (__any_sync(0xffffffffu, (v & ~ST_VALUE) == 0)) {
      if (++spins > SPIN_LIMIT) {  // cannot happen with in-order tile tickets
        if (lane == 0) atomicAdd(&g_wait_timeouts, 1u);
        return __shfl_sync(0xffffffffu, excl, 0);
      }
      if (HM_LB_SLEEP_NS) __nanosleep(HM_LB_SLEEP_NS);
      if ((v & ~ST_VALUE) == 0) v = ld_status(status + j);
    }
    // nearest inclusive prefix in the window (lowest lane = highest tile)
    const unsigned pre = __ballot_sync(0xffffffffu, (v & ST_PREFIX) != 0);
    const int stop = pre ? __ffs(pre) - 1 : 32;
    uint64_t mine = lane <= stop && j >= 0 ? (v & ST_VALUE) : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    excl += mine;
    if (pre) break;
    end -= 32;
  }
  return excl;
}

// Histograms of all passes of all jobs; the last block to finish turns them
// into exclusive digit offsets (one warp per (job, pass)) and writes 0 kept
// keys for empty unique jobs.
__global__ void __launch_bounds__(TPB)
    k_sort_hist(const __grid_constant__ Batch B, const __grid_constant__ Grid G, uint32_t* done) {
  __shared__ uint32_t h[SORT_MAX_PASSES][256];
  __shared__ bool last;
  if (G.nj) {
    const int e = grid_entry(G, blockIdx.x);
    const JobDev& J = B.j[G.job[e]];
    const int64_t lb = blockIdx.x - G.first[e], jblocks = G.first[e + 1] - G.first[e];
    for (int i = threadIdx.x; i < J.np * 256; i += TPB) (&h[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = lb * TPB + threadIdx.x; i < J.n; i += jblocks * TPB) {
      const uint64_t ka = J.a[0][i], kb = J.b[0] ? J.b[0][i] : 0;
      for (int p = 0; p < J.np; ++p)
        atomicAdd(&h[p][((J.arr[p] ? kb : ka) >> J.shift[p]) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < J.np * 256; i += TPB)
      if ((&h[0][0])[i]) atomicAdd(&J.ghist[i], (&h[0][0])[i]);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int total = 0;
  for (int k = 0; k < B.nj; ++k) total += B.j[k].np;
  for (int w = warp; w < total; w += TPB / 32) {
    int k = 0, p = w;
    while (p >= B.j[k].np) p -= B.j[k++].np;
    const JobDev& J = B.j[k];
    const volatile uint32_t* src = J.ghist + p * 256 + lane * 8;
    uint32_t v[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      v[i] = src[i];
      sum += v[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      J.gbase[p * 256 + lane * 8 + i] = run;
      run += v[i];
    }
  }
  if (threadIdx.x < B.nj) {
    const JobDev& J = B.j[threadIdx.x];
    if (J.unique && J.n == 0 && J.d_kept) *J.d_kept = 0;
  }
}

// Pass p of every job in the grid.
__global__ void __launch_bounds__(TPB) k_sort_pass(const __grid_constant__ Batch B, const __grid_constant__ Grid G, int p) {
  __shared__ uint32_t wcnt[TPB / 32][256];
  __shared__ uint64_t toff[256];
  __shared__ uint32_t tile_s;
  const int e = grid_entry(G, blockIdx.x);
  const JobDev& J = B.j[G.job[e]];
  if (threadIdx.x == 0) tile_s = atomicAdd(&J.ctr[p], 1u);
  for (int i = threadIdx.x; i < (TPB / 32) * 256; i += TPB) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = tile_s;
  // the next pass's status array was the previous pass's: clear this row
  J.status[(p + 1) & 1][tile * 256 + threadIdx.x] = 0;
  const int shift = G.shift[e];
  const bool on_b = G.on_b[e] != 0;
  const uint64_t* sa = J.a[p & 1];
  const uint64_t* sb = J.b[0] ? J.b[p & 1] : nullptr;
  uint64_t* da = J.a[(p + 1) & 1];
  uint64_t* db = J.b[0] ? J.b[(p + 1) & 1] : nullptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = tile * TILE + warp * (32 * IPT);
  const unsigned lt = (1u << lane) - 1u;
  uint32_t dig[IPT], rank[IPT];
  uint64_t ka[IPT], kb[IPT];
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int64_t idx = base + it * 32 + lane;
    ka[it] = idx < J.n ? sa[idx] : 0;
    kb[it] = (sb && idx < J.n) ? sb[idx] : 0;
  }
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int64_t idx = base + it * 32 + lane;
    const bool valid = idx < J.n;
    const uint32_t d = valid ? (uint32_t)(((on_b ? kb[it] : ka[it]) >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? wcnt[warp][d] : 0u;
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
    for (int w = 0; w < TPB / 32; ++w) {
      const uint32_t c = wcnt[w][d];
      wcnt[w][d] = run;
      run += c;
    }
    uint64_t* status = J.status[p & 1];
    uint64_t excl = 0;
    if (tile == 0) {
      st_status(status + d, ST_PREFIX | run);
    } else {
      st_status(status + tile * 256 + d, ST_AGG | run);
      excl = look_back(status, tile, 256, d);
      st_status(status + tile * 256 + d, ST_PREFIX | (excl + run));
    }
    toff[d] = (uint64_t)J.gbase[p * 256 + d] + excl;
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int64_t idx = base + it * 32 + lane;
    if (idx < J.n) {
      const uint32_t d = dig[it];
      const uint64_t pos = toff[d] + wcnt[warp][d] + rank[it];
      da[pos] = ka[it];
      if (db) db[pos] = kb[it];
    }
  }
}

// Unique + unpack of every unique job in the grid: a key is kept when it
// differs from its predecessor; its output position is the number of kept
// keys before it (block scan + look-back over tiles).
__global__ void __launch_bounds__(TPB) k_sort_unique(const __grid_constant__ Batch B, const __grid_constant__ Grid G) {
  __shared__ uint32_t wtot[TPB / 32];
  __shared__ uint64_t tile_excl;
  __shared__ uint32_t tile_s;
  const JobDev& J = B.j[G.job[grid_entry(G, blockIdx.x)]];
  if (threadIdx.x == 0) tile_s = atomicAdd(&J.ctr[J.np], 1u);
  __syncthreads();
  const int64_t tile = tile_s;
  const uint64_t* sa = J.a[J.np & 1];
  const uint64_t* sb = J.b[0] ? J.b[J.np & 1] : nullptr;
  const int64_t i0 = tile * TILE + (int64_t)threadIdx.x * IPT;
  uint32_t keep = 0, cnt = 0;
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int64_t i = i0 + it;
    if (i < J.n) {
      bool k = i == 0 || sa[i] != sa[i - 1];
      if (!k && J.b_is_key && sb) k = sb[i] != sb[i - 1];
      if (k) {
        keep |= 1u << it;
        ++cnt;
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t before = 0, total = 0;
#pragma unroll
  for (int w = 0; w < TPB / 32; ++w) {
    before += w < warp ? wtot[w] : 0u;
    total += wtot[w];
  }
  if (threadIdx.x < 32) {
    uint64_t excl = 0;
    if (tile == 0) {
      if (threadIdx.x == 0) st_status(J.ustatus, ST_PREFIX | total);
    } else {
      if (threadIdx.x == 0) st_status(J.ustatus + tile, ST_AGG | total);
      excl = look_back_warp(J.ustatus, tile);
      if (threadIdx.x == 0) st_status(J.ustatus + tile, ST_PREFIX | (excl + total));
    }
    if (threadIdx.x == 0) {
      tile_excl = excl;
      if (tile == J.tiles - 1 && J.d_kept) *J.d_kept = (uint32_t)(excl + total);
    }
  }
  __syncthreads();
  uint64_t pos = tile_excl + before + incl - cnt;
  const int mb = J.member_bits;
  const uint64_t mask = (1ull << mb) - 1;
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    if (!((keep >> it) & 1u)) continue;
    const int64_t i = i0 + it;
    const uint64_t ka = sa[i], kb = sb ? sb[i] : 0;
    if (J.unpack == SortJob::RAW) {
      static_cast<uint64_t*>(J.out)[pos] = ka;
      if (J.out_b) J.out_b[pos] = kb;
    } else if (J.unpack == SortJob::PAIR) {
      static_cast<uint64_t*>(J.out)[pos] = ((ka >> mb) << 32) | (ka & mask);
    } else {
      // members most significant first: the last member in the lowest bits
      unsigned __int128 key = ((unsigned __int128)kb << 64) | ka;
      const int32_t m3 = (int32_t)((uint64_t)key & mask);
      key >>= mb;
      const int32_t m2 = (int32_t)((uint64_t)key & mask);
      key >>= mb;
      const int32_t m1 = (int32_t)((uint64_t)key & mask);
      key >>= mb;
      const int32_t m0 = (int32_t)((uint64_t)key & mask);
      static_cast<int4*>(J.out)[pos] = J.unpack == SortJob::TRIPLE
                                           ? make_int4(m1, m2, m3, -1)
                                           : make_int4(m0, m1, m2, m3);
    }
    ++pos;
  }
}

// Jobs of at most SMALL_KEYS keys, sorted by counting ranks over the whole
// GPU: a key's place is the number of keys ordered before it, comparing only
// the bits the job's digit passes cover (the high word b first) and breaking
// ties by index, which keeps the sort stable. k_sort_rank: job k of G owns
// T_k^2 blocks, T_k = ceil(n / RANK_T); block (it, jt) compares the keys of
// tile it with those of tile jt (kept in shared memory) and adds the partial
// ranks with atomics. k_sort_place: one block per job puts the keys at their
// ranks in shared memory, drops repeats and writes the output. O(n^2)
// comparisons, 67M at 8,192 keys, spread over every SM instead of the
// latency chain of one block's radix passes.
constexpr int RANK_T = 256;  // keys per tile = threads per block of k_sort_rank
constexpr int PLACE_T = 1024;  // threads per block of k_sort_place
constexpr int64_t SMALL_KEYS = 8192;
constexpr size_t PLACE_SMEM = (size_t)SMALL_KEYS * 16 + 32 * 4;

__device__ __forceinline__ void rank_masks(const JobDev& J, uint64_t& ma, uint64_t& mb) {
  ma = 0;
  mb = 0;
  for (int p = 0; p < J.np; ++p) {
    const uint64_t m = 0xFFull << J.shift[p];
    if (J.arr[p])
      mb |= m;
    else
      ma |= m;
  }
}

__global__ void __launch_bounds__(RANK_T) k_sort_rank(const __grid_constant__ Batch B, const __grid_constant__ Grid G) {
  __shared__ __align__(16) uint64_t ja[RANK_T];
  __shared__ uint64_t jb[RANK_T];
  const int e = grid_entry(G, blockIdx.x);
  const JobDev& J = B.j[G.job[e]];
  const int n = (int)J.n;
  const int T = (n + RANK_T - 1) / RANK_T;
  const int q = (int)(blockIdx.x - G.first[e]);
  const int it = q / T, jt = q - (q / T) * T;
  uint64_t ma, mb;
  rank_masks(J, ma, mb);
  const bool has_b = J.b[0] != nullptr;
  const int j0 = jt * RANK_T, m = min(RANK_T, n - j0);
  const int i = it * RANK_T + threadIdx.x;
  if (mb == 0 && (ma >> 51) == 0) {
    // the sorted bits and the index fit one word: (key << 13) | index orders
    // like (key, index) and is unique, so one compare per pair; slots past
    // the tile hold the largest word, which ranks before nothing
    const uint64_t cj = threadIdx.x < m
                            ? ((J.a[0][j0 + threadIdx.x] & ma) << 13) | (uint64_t)(j0 + threadIdx.x)
                            : ~0ull;
    ja[threadIdx.x] = cj;
    const uint64_t ci = i < n ? ((J.a[0][i] & ma) << 13) | (uint64_t)i : 0;
    __syncthreads();
    if (i < n) {
      uint32_t c = 0;
      const ulonglong2* j2 = reinterpret_cast<const ulonglong2*>(ja);
#pragma unroll 8
      for (int t = 0; t < RANK_T / 2; ++t) {
        const ulonglong2 w = j2[t];
        c += (w.x < ci ? 1u : 0u) + (w.y < ci ? 1u : 0u);
      }
      if (c) atomicAdd(&J.rank[i], c);
    }
    return;
  }
  if (threadIdx.x < m) {
    ja[threadIdx.x] = J.a[0][j0 + threadIdx.x] & ma;
    jb[threadIdx.x] = has_b ? (J.b[0][j0 + threadIdx.x] & mb) : 0;
  }
  uint64_t ai = 0, bi = 0;
  if (i < n) {
    ai = J.a[0][i] & ma;
    bi = has_b ? (J.b[0][i] & mb) : 0;
  }
  __syncthreads();
  if (i < n) {
    uint32_t c = 0;
    for (int t = 0; t < m; ++t) {
      const uint64_t aj = ja[t], bj = jb[t];
      const bool before = bj < bi || (bj == bi && (aj < ai || (aj == ai && j0 + t < i)));
      c += before ? 1u : 0u;
    }
    if (c) atomicAdd(&J.rank[i], c);
  }
}

__global__ void __launch_bounds__(PLACE_T) k_sort_place(const __grid_constant__ Batch B, const __grid_constant__ Grid G) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* ka_s = reinterpret_cast<uint64_t*>(smem);
  uint64_t* kb_s = ka_s + SMALL_KEYS;
  uint32_t* wtot = reinterpret_cast<uint32_t*>(kb_s + SMALL_KEYS);
  const JobDev& J = B.j[G.job[blockIdx.x]];
  const int n = (int)J.n;
  const bool has_b = J.b[0] != nullptr;
  // ranks are a permutation of [0, n) (each counts fewer than n keys); a
  // thread's (at most 8) ranks and keys are loaded before any is stored, so
  // their loads overlap
  {
    constexpr int PER = (int)(SMALL_KEYS / PLACE_T);
    uint32_t r[PER];
    uint64_t va[PER], vb[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int k = threadIdx.x + u * PLACE_T;
      if (k < n) {
        r[u] = J.rank[k];
        va[u] = J.a[0][k];
        vb[u] = has_b ? J.b[0][k] : 0;
      }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int k = threadIdx.x + u * PLACE_T;
      if (k < n) {
        ka_s[r[u]] = va[u];
        kb_s[r[u]] = vb[u];
      }
    }
  }
  __syncthreads();
  if (!J.unique) {
    for (int k = threadIdx.x; k < n; k += PLACE_T) {
      J.a[0][k] = ka_s[k];
      if (has_b) J.b[0][k] = kb_s[k];
    }
    return;
  }
  // unique: a key is kept when it differs from its predecessor; thread t owns
  // keys [t * ipt, (t + 1) * ipt), ipt <= 8
  const int ipt = (n + PLACE_T - 1) / PLACE_T;
  const int i0 = threadIdx.x * ipt;
  uint32_t keep = 0, cnt = 0;
  for (int u = 0; u < ipt; ++u) {
    const int k = i0 + u;
    if (k >= n) break;
    bool kp = k == 0 || ka_s[k] != ka_s[k - 1];
    if (!kp && J.b_is_key && has_b) kp = kb_s[k] != kb_s[k - 1];
    if (kp) {
      keep |= 1u << u;
      ++cnt;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = wtot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    wtot[lane] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0 && J.d_kept) *J.d_kept = wtot[PLACE_T / 32 - 1];
  uint64_t pos = (warp ? wtot[warp - 1] : 0u) + incl - cnt;
  const int mbits = J.member_bits;
  const uint64_t mask = (1ull << mbits) - 1;
  for (int u = 0; u < ipt; ++u) {
    if (!((keep >> u) & 1u)) continue;
    const int k = i0 + u;
    const uint64_t ka = ka_s[k], kb = kb_s[k];
    if (J.unpack == SortJob::RAW) {
      static_cast<uint64_t*>(J.out)[pos] = ka;
      if (J.out_b) J.out_b[pos] = kb;
    } else if (J.unpack == SortJob::PAIR) {
      static_cast<uint64_t*>(J.out)[pos] = ((ka >> mbits) << 32) | (ka & mask);
    } else {
      unsigned __int128 key = ((unsigned __int128)kb << 64) | ka;
      const int32_t m3 = (int32_t)((uint64_t)key & mask);
      key >>= mbits;
      const int32_t m2 = (int32_t)((uint64_t)key & mask);
      key >>= mbits;
      const int32_t m1 = (int32_t)((uint64_t)key & mask);
      key >>= mbits;
      const int32_t m0 = (int32_t)((uint64_t)key & mask);
      static_cast<int4*>(J.out)[pos] = J.unpack == SortJob::TRIPLE
                                           ? make_int4(m1, m2, m3, -1)
                                           : make_int4(m0, m1, m2, m3);
    }
    ++pos;
  }
}

// k_sort_place's shared memory is above the default 48 KB: opt in once per
// device.
void place_smem_attr() {
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  HM_CUDA(cudaFuncSetAttribute(k_sort_place, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)PLACE_SMEM));
  done.fetch_or(bit, std::memory_order_acq_rel);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Layout of a batch's scratch: [zeroed: per job status[0] | ustatus | ghist |
// ctr | rank ; done] [per job: status[1] | gbase | temporaries].
struct SortPlan {
  Batch B{};
  std::vector<size_t> zoff, off;
  size_t zbytes = 0, bytes = 0;
};

void plan_sort(const SortJob* jobs, int njobs, SortPlan& P) {
  HM_CHECK(njobs >= 1 && njobs <= SORT_MAX_JOBS, HM_EINVAL, "sort batch of 1-4 jobs");
  Batch& B = P.B;
  B.nj = njobs;
  size_t zbytes = 0, bytes = 0;
  std::vector<size_t>& zoff = P.zoff;
  std::vector<size_t>& off = P.off;
  zoff.assign(njobs, 0);
  off.assign(njobs, 0);
  for (int k = 0; k < njobs; ++k) {
    const SortJob& S = jobs[k];
    HM_CHECK(S.n >= 0 && S.n < (1ll << 31), HM_EINVAL, "sort input too large");
    HM_CHECK(S.passes >= 0 && S.passes <= SORT_MAX_PASSES, HM_EINVAL, "too many radix passes");
    HM_CHECK(!S.unique || S.out || S.n == 0, HM_EINVAL, "unique sort without an output");
    JobDev& J = B.j[k];
    J.n = S.n;
    J.tiles = (S.n + TILE - 1) / TILE;
    J.np = S.n > 1 ? S.passes : 0;
    for (int p = 0; p < S.passes; ++p) {
      J.arr[p] = S.arr[p];
      J.shift[p] = S.shift[p];
    }
    J.b_is_key = S.b_is_key;
    J.unique = S.unique;
    J.unpack = S.unpack;
    J.member_bits = S.member_bits;
    J.out = S.out;
    J.out_b = S.out_b;
    J.d_kept = S.d_kept;
    zoff[k] = zbytes;
    zbytes += align256((size_t)J.tiles * 256 * 8) + align256((size_t)J.tiles * 8) +
              align256((size_t)SORT_MAX_PASSES * 256 * 4) + align256((SORT_MAX_PASSES + 1) * 4);
    if (J.n >= 1 && J.n <= SMALL_KEYS) zbytes += align256((size_t)J.n * 4);
  }
  zbytes += 256;  // done counter
  bytes = zbytes;
  for (int k = 0; k < njobs; ++k) {
    off[k] = bytes;
    const JobDev& J = B.j[k];
    bytes += align256((size_t)J.tiles * 256 * 8) + align256((size_t)SORT_MAX_PASSES * 256 * 4);
    if (J.np > 0) bytes += align256((size_t)J.n * 8) * (jobs[k].b ? 2 : 1);
  }
  P.zbytes = zbytes;
  P.bytes = bytes;
}

}  // namespace

size_t sort_batch_scratch(const SortJob* jobs, int njobs, size_t* zero_bytes) {
  SortPlan P;
  plan_sort(jobs, njobs, P);
  if (zero_bytes) *zero_bytes = P.zbytes;
  return P.bytes;
}

void sort_batch(const SortJob* jobs, int njobs, cudaStream_t s, unsigned char* ext_scratch,
                bool zeroed) {
  SortPlan P;
  plan_sort(jobs, njobs, P);
  Batch& B = P.B;
  const size_t zbytes = P.zbytes, bytes = P.bytes;
  const std::vector<size_t>& zoff = P.zoff;
  const std::vector<size_t>& off = P.off;
  DBuf<unsigned char> scratch(ext_scratch ? 0 : bytes, s);
  unsigned char* base = ext_scratch ? ext_scratch : scratch.p;
  for (int k = 0; k < njobs; ++k) {
    JobDev& J = B.j[k];
    const SortJob& S = jobs[k];
    unsigned char* z = base + zoff[k];
    J.status[0] = reinterpret_cast<uint64_t*>(z);
    z += align256((size_t)J.tiles * 256 * 8);
    J.ustatus = reinterpret_cast<uint64_t*>(z);
    z += align256((size_t)J.tiles * 8);
    J.ghist = reinterpret_cast<uint32_t*>(z);
    z += align256((size_t)SORT_MAX_PASSES * 256 * 4);
    J.ctr = reinterpret_cast<uint32_t*>(z);
    z += align256((SORT_MAX_PASSES + 1) * 4);
    J.rank = (J.n >= 1 && J.n <= SMALL_KEYS) ? reinterpret_cast<uint32_t*>(z) : nullptr;
    unsigned char* q = base + off[k];
    J.status[1] = reinterpret_cast<uint64_t*>(q);
    q += align256((size_t)J.tiles * 256 * 8);
    J.gbase = reinterpret_cast<uint32_t*>(q);
    q += align256((size_t)SORT_MAX_PASSES * 256 * 4);
    J.a[0] = S.a;
    J.b[0] = S.b;
    J.a[1] = J.np > 0 ? reinterpret_cast<uint64_t*>(q) : S.a;
    if (J.np > 0) q += align256((size_t)J.n * 8);
    J.b[1] = (J.np > 0 && S.b) ? reinterpret_cast<uint64_t*>(q) : S.b;
  }
  uint32_t* done = reinterpret_cast<uint32_t*>(base + zbytes - 256);
  if (!(ext_scratch && zeroed)) HM_CUDA(cudaMemsetAsync(base, 0, zbytes, s));
  // jobs of up to SMALL_KEYS keys: ranks by counting, all such jobs in one
  // launch (T^2 blocks per job, T = ceil(n / RANK_T))
  auto small = [&](int k) { return B.j[k].n >= 1 && B.j[k].n <= SMALL_KEYS; };
  {
    Grid G{};
    int64_t blocks = 0;
    for (int k = 0; k < njobs; ++k) {
      if (!small(k)) continue;
      const int64_t T = (B.j[k].n + RANK_T - 1) / RANK_T;
      G.job[G.nj] = k;
      G.first[G.nj] = blocks;
      blocks += T * T;
      ++G.nj;
    }
    G.first[G.nj] = blocks;
    if (G.nj) {
      k_sort_rank<<<(unsigned)blocks, RANK_T, 0, s>>>(B, G);
      HM_KCHECK();
      place_smem_attr();
      k_sort_place<<<(unsigned)G.nj, PLACE_T, PLACE_SMEM, s>>>(B, G);
      HM_KCHECK();
    }
  }

  // histograms (at least one block, for the offsets and empty jobs)
  {
    Grid G{};
    int64_t blocks = 0;
    for (int k = 0; k < njobs; ++k) {
      if (B.j[k].np == 0 || small(k)) continue;
      int64_t hb = (B.j[k].n + 4095) / 4096;
      if (hb > 152 * 2) hb = 152 * 2;
      G.job[G.nj] = k;
      G.first[G.nj] = blocks;
      blocks += hb;
      ++G.nj;
    }
    G.first[G.nj] = blocks;
    bool empty_unique = false;
    for (int k = 0; k < njobs; ++k) empty_unique |= B.j[k].unique && B.j[k].n == 0;
    if (blocks > 0 || empty_unique) {
      k_sort_hist<<<(unsigned)(blocks > 0 ? blocks : 1), TPB, 0, s>>>(B, G, done);
      HM_KCHECK();
    }
  }
  int maxp = 0;
  for (int k = 0; k < njobs; ++k)
    if (!small(k)) maxp = std::max(maxp, B.j[k].np);
  for (int p = 0; p < maxp; ++p) {
    Grid G{};
    int64_t blocks = 0;
    for (int k = 0; k < njobs; ++k) {
      if (B.j[k].np <= p || small(k)) continue;
      G.job[G.nj] = k;
      G.on_b[G.nj] = B.j[k].arr[p];
      G.shift[G.nj] = B.j[k].shift[p];
      G.first[G.nj] = blocks;
      blocks += B.j[k].tiles;
      ++G.nj;
    }
    G.first[G.nj] = blocks;
    k_sort_pass<<<(unsigned)blocks, TPB, 0, s>>>(B, G, p);
    HM_KCHECK();
  }
  {
    Grid G{};
    int64_t blocks = 0;
    for (int k = 0; k < njobs; ++k) {
      if (!B.j[k].unique || B.j[k].n == 0 || small(k)) continue;
      G.job[G.nj] = k;
      G.first[G.nj] = blocks;
      blocks += B.j[k].tiles;
      ++G.nj;
    }
    G.first[G.nj] = blocks;
    if (blocks) {
      k_sort_unique<<<(unsigned)blocks, TPB, 0, s>>>(B, G);
      HM_KCHECK();
    }
  }
  // sort-only jobs whose last pass ended in the temporaries: copy back
  for (int k = 0; k < njobs; ++k) {
    const JobDev& J = B.j[k];
    if (J.unique || (J.np & 1) == 0 || small(k)) continue;
    HM_CUDA(cudaMemcpyAsync(J.a[0], J.a[1], J.n * 8, cudaMemcpyDeviceToDevice, s));
    if (J.b[0]) HM_CUDA(cudaMemcpyAsync(J.b[0], J.b[1], J.n * 8, cudaMemcpyDeviceToDevice, s));
  }
}

namespace {

// Self-test of the bounded waits: the last of `tiles` tiles looks back over
// the others, one of which (tile 0) never publishes, with both look-back
// forms; each wait gives up after SPIN_LIMIT polls and counts a timeout.
__global__ void k_wait_selftest(const uint64_t* status, int64_t tiles, uint64_t* out) {
  if (threadIdx.x == 0) out[0] = look_back(status, tiles - 1, 1, 0);
  __syncwarp();
  const uint64_t v = look_back_warp(status, tiles - 1);
  if (threadIdx.x == 0) out[1] = v;
}

}  // namespace

void wait_selftest(cudaStream_t s) {
  constexpr int64_t tiles = 4;
  DBuf<uint64_t> buf(tiles + 2, s);
  std::vector<uint64_t> h(tiles + 2, 0);
  for (int64_t t = 1; t < tiles; ++t) h[t] = ST_AGG | 1;  // tiles 1..3 publish an aggregate
  HM_CUDA(cudaMemcpyAsync(buf.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, s));
  k_wait_selftest<<<1, 32, 0, s>>>(buf.p, tiles, buf.p + tiles);
  HM_KCHECK();
  unsigned* timeouts = (unsigned*)(pinned_words() + 80);
  *timeouts = 0;
  wait_timeouts_async(timeouts, s);
  HM_CUDA(cudaStreamSynchronize(s));
  wait_timeouts_check(*timeouts, s);
  HM_CHECK(false, HM_EINVAL, "bounded wait self-test: no wait gave up");
}

void wait_timeouts_async(unsigned* h_count, cudaStream_t s) {
  HM_CUDA(cudaMemcpyFromSymbolAsync(h_count, g_wait_timeouts, sizeof(unsigned), 0,
                                    cudaMemcpyDeviceToHost, s));
}

void wait_timeouts_check(unsigned count, cudaStream_t s) {
  if (!count) return;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_wait_timeouts) == cudaSuccess)
    cudaMemsetAsync(p, 0, sizeof(unsigned), s);
  HM_CHECK(false, HM_ETIMEOUT, "a device-side wait gave up (decoupled look-back)");
}

void radix_sort_u64(uint64_t* keys, uint64_t* vals, int64_t n, int bits, cudaStream_t s,
                    int lo_bit) {
  SortJob J{};
  J.a = keys;
  J.b = vals;
  J.n = n;
  for (int sh = 0; sh < bits; sh += 8) {
    J.arr[J.passes] = 0;
    J.shift[J.passes++] = (int8_t)(lo_bit + sh);
  }
  if (n <= 1 || J.passes == 0) return;
  sort_batch(&J, 1, s);
}

void radix_sort_u128(uint64_t* hi, uint64_t* lo, int64_t n, int hi_bits, int lo_bits,
                     cudaStream_t s) {
  SortJob J{};
  J.a = lo;
  J.b = hi;
  J.n = n;
  J.b_is_key = 1;
  J.passes = 0;
  for (int sh = 0; sh < lo_bits; sh += 8) {
    J.arr[J.passes] = 0;
    J.shift[J.passes++] = (int8_t)sh;
  }
  for (int sh = 0; sh < hi_bits; sh += 8) {
    J.arr[J.passes] = 1;
    J.shift[J.passes++] = (int8_t)sh;
  }
  if (n <= 1 || J.passes == 0) return;
  sort_batch(&J, 1, s);
}

}  // namespace hm

// ------------------------------------------------------------------ batched scan
namespace hm {
namespace {

constexpr int SCAN_JOBS = 8;

struct ScanDev {
  uint64_t* a;
  int64_t n, tiles;
  uint64_t* total;
  uint64_t* status;  // [tiles]
  uint32_t* ctr;
};
struct ScanBatch {
  int nj;
  int single;  // every job is one tile: no tickets, no look-back, no scratch
  ScanDev j[SCAN_JOBS];
  int64_t first[SCAN_JOBS + 1];
};

// In place: a[i] = sum of the input a[0..i), a[n] = total (and *total). Each
// tile reads its 2048 inputs before anything of it is written, and no tile
// reads another's inputs, so in-place is safe. The tile moves through shared
// memory both ways, so that global loads and stores are coalesced while each
// thread scans IPT consecutive values.
__global__ void __launch_bounds__(TPB) k_scan_batch(const __grid_constant__ ScanBatch B) {
  __shared__ uint64_t wtot[TPB / 32];
  __shared__ uint64_t tile_excl;
  __shared__ uint32_t tile_s;
  __shared__ uint64_t stage[TILE];
  int e = 0;
  while (e + 1 < B.nj && (int64_t)blockIdx.x >= B.first[e + 1]) ++e;
  const ScanDev& J = B.j[e];
  if (threadIdx.x == 0) tile_s = B.single ? 0u : atomicAdd(J.ctr, 1u);
  __syncthreads();
  const int64_t tile = tile_s;
  const int64_t t0 = tile * TILE;
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int64_t i = t0 + it * TPB + threadIdx.x;
    stage[it * TPB + threadIdx.x] = i < J.n ? J.a[i] : 0;
  }
  __syncthreads();
  uint64_t v[IPT], sum = 0;
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    v[it] = stage[threadIdx.x * IPT + it];
    sum += v[it];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint64_t before = 0, total = 0;
#pragma unroll
  for (int w = 0; w < TPB / 32; ++w) {
    before += w < warp ? wtot[w] : 0ull;
    total += wtot[w];
  }
  if (threadIdx.x < 32) {
    uint64_t excl = 0;
    if (tile == 0) {
      if (threadIdx.x == 0 && !B.single) st_status(J.status, ST_PREFIX | total);
    } else {
      if (threadIdx.x == 0) st_status(J.status + tile, ST_AGG | total);
      excl = look_back_warp(J.status, tile);
      if (threadIdx.x == 0) st_status(J.status + tile, ST_PREFIX | (excl + total));
    }
    if (threadIdx.x == 0) {
      tile_excl = excl;
      if (tile == J.tiles - 1) {
        J.a[J.n] = excl + total;
        if (J.total) *J.total = excl + total;
      }
    }
  }
  __syncthreads();
  uint64_t run = tile_excl + before + incl - sum;
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    stage[threadIdx.x * IPT + it] = run;
    run += v[it];
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int64_t i = t0 + it * TPB + threadIdx.x;
    if (i < J.n) J.a[i] = stage[it * TPB + threadIdx.x];
  }
}

}  // namespace

// Scratch of a multi-tile scan batch: per array its tile status words and
// ticket counter, all of it to be zeroed; 0 when every array is one tile.
size_t scan_batch_scratch(const ScanJob* jobs, int njobs) {
  size_t bytes = 256;
  int64_t blocks = 0;
  for (int k = 0; k < njobs; ++k) {
    const int64_t tiles = std::max<int64_t>(1, (jobs[k].n + TILE - 1) / TILE);
    bytes += align256((size_t)tiles * 8) + 256;
    blocks += tiles;
  }
  return blocks == njobs ? 0 : bytes;
}

void scan_batch_inplace(const ScanJob* jobs, int njobs, cudaStream_t s, unsigned char* ext_scratch,
                        bool zeroed) {
  HM_CHECK(njobs >= 1 && njobs <= SCAN_JOBS, HM_EINVAL, "scan batch of 1-8 arrays");
  ScanBatch B{};
  B.nj = njobs;
  size_t bytes = 256;
  std::vector<size_t> off(njobs);
  int64_t blocks = 0;
  for (int k = 0; k < njobs; ++k) {
    HM_CHECK(jobs[k].n >= 0 && jobs[k].a, HM_EINVAL, "bad scan array");
    ScanDev& J = B.j[k];
    J.a = jobs[k].a;
    J.n = jobs[k].n;
    J.tiles = std::max<int64_t>(1, (J.n + TILE - 1) / TILE);
    J.total = jobs[k].total;
    off[k] = bytes;
    bytes += align256((size_t)J.tiles * 8) + 256;
    B.first[k] = blocks;
    blocks += J.tiles;
  }
  B.first[njobs] = blocks;
  HM_CHECK(blocks < (1ll << 31), HM_EINVAL, "scan too large");
  if (blocks == njobs) {
    // one tile each: a block per array, nothing to allocate
    B.single = 1;
    k_scan_batch<<<(unsigned)blocks, TPB, 0, s>>>(B);
    HM_KCHECK();
    return;
  }
  DBuf<unsigned char> scratch(ext_scratch ? 0 : bytes, s);
  unsigned char* base = ext_scratch ? ext_scratch : scratch.p;
  for (int k = 0; k < njobs; ++k) {
    B.j[k].status = reinterpret_cast<uint64_t*>(base + off[k]);
    B.j[k].ctr = reinterpret_cast<uint32_t*>(base + off[k] + align256((size_t)B.j[k].tiles * 8));
  }
  if (!(ext_scratch && zeroed)) HM_CUDA(cudaMemsetAsync(base, 0, bytes, s));
  k_scan_batch<<<(unsigned)blocks, TPB, 0, s>>>(B);
  HM_KCHECK();
}

}  // namespace hm

extern "C" hm_status hm_selftest_wait(void* stream) {
  return hm::guarded([&] { hm::wait_selftest((cudaStream_t)stream); });
}
