// Graph ingest on the device: normalisation of hyperedges into sets (Def. 1),
// deduplication (E is a set), the per-size hyperedge hash sets that make the
// fill-in of Sec. 4.3 a constant number of probes, and the CSR neighbourhoods
// the candidate generators walk.
#include <cstdlib>
#include <mutex>
#include <tuple>

#include "hm_internal.cuh"

namespace hm {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

namespace {

constexpr int T256 = 256;

unsigned grid1d(int64_t n, int threads = T256) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

int bits_for(int64_t maxval) {
  int b = 1;
  while (b < 62 && (1ll << b) <= maxval) ++b;
  return b;
}

enum { ERR_RANGE = 1, ERR_OFFSETS = 2, ERR_TABLE = 4 };

// column of node b in the bitmap row of node a (rows span a's block of ids)
__device__ __forceinline__ int32_t bit_col(int32_t a, int32_t b, int32_t block, uint64_t inv) {
  return block ? b - (int32_t)__umul64hi((uint64_t)(uint32_t)a, inv) * block : b;
}

// Dense bitmaps written while normalising (graphs with pair bitmaps): pair
// rows, co-occurrence rows of 3- and 4-hyperedges, exact triple rows (may be
// NULL: the 3-hyperedges then go to sort keys).
struct BitsOut {
  uint32_t* bits2;
  uint32_t* bits3;
  uint32_t* bits4;
  uint32_t* tri3;
  int32_t bw, block, n;
  uint64_t inv;
};

__device__ __forceinline__ void set_bit(const BitsOut& o, uint32_t* bm, int32_t a, int32_t b) {
  const int32_t c = bit_col(a, b, o.block, o.inv);
  atomicOr(bm + (size_t)a * o.bw + (c >> 5), 1u << (c & 31));
}

// Normalisation: hyperedge j's members (sorted, repeats collapsed) as long as
// it has at most kmax distinct members; hyperedges with more are only counted
// (size kmax + 1). Every mode counts the hyperedges per size into cnt; MODE 1
// emits the packed sort key of each kept hyperedge of size >= 2 (members
// concatenated with b bits each, most significant first) into arrays sized
// for the worst case; MODE 2 sets the bitmap bits of each kept hyperedge
// instead (pairs, co-occurrence, exact triple rows) and emits sort keys only
// for 3- and 4-hyperedges.
//
// A block takes NORM_ITEMS * 256 consecutive hyperedges, each warp 32 *
// NORM_ITEMS of them, whose members are one contiguous range of the input:
// the warp stages up to NORM_STAGE of them in shared memory with coalesced
// loads (the rest are read directly), then each lane normalises NORM_ITEMS
// hyperedges. Output slots come from per-block counts in shared memory and
// one global atomic per size per block: same-address atomics serialise in
// L2, so one per warp and size (a quarter of a million on 2M hyperedges) cost
// more than the rest of the kernel.
constexpr int NORM_THREADS = 256;
constexpr int NORM_ITEMS = 4;
constexpr int NORM_STAGE = 1024;  // staged members per warp (4 KB)
constexpr int64_t NORM_TILE = (int64_t)NORM_THREADS * NORM_ITEMS;

unsigned norm_grid(int64_t m) { return (unsigned)((m + NORM_TILE - 1) / NORM_TILE); }

template <int MODE>
__global__ void __launch_bounds__(NORM_THREADS)
    k_normalize(const int32_t* __restrict__ mem, const int64_t* __restrict__ off, int64_t m,
                int32_t n, int kmax, int b, unsigned long long* __restrict__ cnt,
                int* __restrict__ err, uint64_t* __restrict__ c2, uint64_t* __restrict__ c3hi,
                uint64_t* __restrict__ c3lo, uint64_t* __restrict__ c4hi,
                uint64_t* __restrict__ c4lo, const BitsOut bo) {
  __shared__ int32_t stage[NORM_THREADS / 32][NORM_STAGE];
  __shared__ unsigned int scnt[8];
  __shared__ unsigned long long sbase[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < 8) scnt[threadIdx.x] = 0;
  const int64_t w0 = (int64_t)blockIdx.x * NORM_TILE + (int64_t)warp * 32 * NORM_ITEMS;
  const int64_t wend = min(w0 + 32 * NORM_ITEMS, m);
  // the warp's member range, clamped to the input (offsets[m] members)
  int64_t lo = 0, len = 0;
  if (w0 < m) {
    lo = off[w0];
    const int64_t hi = min(off[wend], off[m]);
    if (lo >= 0 && hi > lo) len = min(hi - lo, (int64_t)NORM_STAGE);
  }
  for (int64_t i = lane; i < len; i += 32) stage[warp][i] = mem[lo + i];
  __syncwarp();
  int32_t v[NORM_ITEMS][5];
  int sz[NORM_ITEMS];  // 0: nothing to count or emit
#pragma unroll
  for (int it = 0; it < NORM_ITEMS; ++it) {
    const int64_t j = w0 + it * 32 + lane;
    sz[it] = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i) v[it][i] = 0;
    if (j >= m) continue;
    const int64_t s0 = off[j], s1 = off[j + 1];
    if (s1 < s0 || s0 < 0) {
      atomicOr(err, ERR_OFFSETS);
      continue;
    }
    int cntd = 0;
    bool big = false, bad = false;
    for (int64_t p = s0; p < s1; ++p) {
      const int64_t q = p - lo;
      const int32_t x = (q >= 0 && q < len) ? stage[warp][q] : mem[p];
      if (x < 0 || x >= n) {
        bad = true;
        continue;
      }
      if (big) continue;
      bool present = false;
      int pos = 0;
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        present |= (i < cntd && v[it][i] == x);
        pos += (i < cntd && v[it][i] < x) ? 1 : 0;
      }
      if (present) continue;
#pragma unroll
      for (int i = 4; i > 0; --i)
        if (i > pos && i <= cntd) v[it][i] = v[it][i - 1];
#pragma unroll
      for (int i = 0; i < 5; ++i)
        if (i == pos) v[it][i] = x;
      ++cntd;
      if (cntd > kmax) big = true;
    }
    if (bad) {
      atomicOr(err, ERR_RANGE);
      continue;
    }
    if (big) {
      sz[it] = kmax + 1;
      continue;
    }
    if (cntd < 2) continue;
    if (MODE == 2) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (i < cntd && k < cntd && i != k)
            set_bit(bo, cntd == 2 ? bo.bits2 : cntd == 3 ? bo.bits3 : bo.bits4, v[it][i],
                    v[it][k]);
      if (cntd == 3 && bo.tri3) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            if (i == k) continue;
            const int32_t c = v[it][3 - i - k];
            atomicOr(bo.tri3 + ((size_t)v[it][i] * bo.n + v[it][k]) * bo.bw + (c >> 5),
                     1u << (c & 31));
          }
      }
    }
    sz[it] = cntd;
  }
  __syncthreads();  // scnt zeroed
  // slots: lanes with the same size share one shared-memory atomic per item
  unsigned loc[NORM_ITEMS];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int it = 0; it < NORM_ITEMS; ++it) {
    const unsigned peers = __match_any_sync(0xffffffffu, sz[it]);
    const int leader = __ffs(peers) - 1;
    unsigned base = 0;
    if (sz[it] && lane == leader) base = atomicAdd(&scnt[sz[it]], (unsigned)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    loc[it] = base + (unsigned)__popc(peers & lt);
  }
  __syncthreads();
  if (threadIdx.x < 8 && scnt[threadIdx.x])
    sbase[threadIdx.x] = atomicAdd(&cnt[threadIdx.x], (unsigned long long)scnt[threadIdx.x]);
  __syncthreads();
#pragma unroll
  for (int it = 0; it < NORM_ITEMS; ++it) {
    const int cntd = sz[it];
    if (cntd < (MODE == 2 ? 3 : 2) || cntd > kmax) continue;  // counted only
    const unsigned long long slot = sbase[cntd] + loc[it];
    unsigned __int128 key = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < cntd) key = (key << b) | (uint32_t)v[it][i];
    if (cntd == 2) {
      c2[slot] = (uint64_t)key;
    } else if (cntd == 3) {
      c3lo[slot] = (uint64_t)key;
      c3hi[slot] = (uint64_t)(key >> 64);
    } else {
      c4lo[slot] = (uint64_t)key;
      c4hi[slot] = (uint64_t)(key >> 64);
    }
  }
}

__device__ __forceinline__ void insert_pair(uint64_t key, uint64_t* table, uint64_t mask,
                                            int* err) {
  uint64_t slot = hash_pair(key) & mask;
  for (uint64_t it = 0; it <= mask; ++it) {
    const unsigned long long old = atomicCAS((unsigned long long*)(table + slot),
                                             (unsigned long long)EMPTY64, (unsigned long long)key);
    if (old == EMPTY64) return;
    slot = (slot + 1) & mask;
  }
  atomicOr(err, ERR_TABLE);
}

// Keys are distinct, so a slot is claimed by a CAS on its first 8 bytes and
// the second half is then stored plainly; probes run in later kernels.
__device__ __forceinline__ void insert_tuple(int4 k, int4* table, uint64_t mask, int* err) {
  uint64_t slot = hash_tuple(k.x, k.y, k.z, k.w) & mask;
  const unsigned long long first = (uint64_t)(uint32_t)k.x | ((uint64_t)(uint32_t)k.y << 32);
  const unsigned long long second = (uint64_t)(uint32_t)k.z | ((uint64_t)(uint32_t)k.w << 32);
  for (uint64_t it = 0; it <= mask; ++it) {
    unsigned long long* w = (unsigned long long*)(table + slot);
    if (atomicCAS(w, (unsigned long long)EMPTY64, first) == EMPTY64) {
      w[1] = second;
      return;
    }
    slot = (slot + 1) & mask;
  }
  atomicOr(err, ERR_TABLE);
}

// The three hash sets in one launch: thread i inserts pair i, then 3- and
// 4-hyperedges after the pairs.
// Node signatures of graphs without pair bitmaps (zeroed, 3 n words): each
// hyperedge sets, in every member's word of its size, the bits of the other
// members. One thread per hyperedge of every size.
__global__ void k_signatures(const uint64_t* __restrict__ e2, int64_t m2, const int4* __restrict__ e3,
                             int64_t m3, const int4* __restrict__ e4, int64_t m4, int32_t n,
                             unsigned long long* __restrict__ sig) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m2 + m3 + m4;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    int k;
    unsigned long long* w;
    if (i < m2) {
      v[0] = (int32_t)(e2[i] >> 32);
      v[1] = (int32_t)(e2[i] & 0xFFFFFFFFull);
      k = 2;
      w = sig;
    } else if (i < m2 + m3) {
      const int4 e = e3[i - m2];
      v[0] = e.x;
      v[1] = e.y;
      v[2] = e.z;
      k = 3;
      w = sig + n;
    } else {
      const int4 e = e4[i - m2 - m3];
      v[0] = e.x;
      v[1] = e.y;
      v[2] = e.z;
      v[3] = e.w;
      k = 4;
      w = sig + 2 * (int64_t)n;
    }
    for (int a = 0; a < k; ++a) {
      unsigned long long bits = 0;
      for (int b = 0; b < k; ++b)
        if (b != a) bits |= sig_bit(v[b]);
      atomicOr(&w[v[a]], bits);
    }
  }
}

__global__ void k_insert_all(const uint64_t* __restrict__ e2, int64_t m2, const int4* __restrict__ e3,
                             int64_t m3, const int4* __restrict__ e4, int64_t m4, uint64_t* h2,
                             uint64_t mask2, int4* h3, uint64_t mask3, int4* h4, uint64_t mask4,
                             int* err) {
  const int64_t total = m2 + m3 + m4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < m2)
      insert_pair(e2[i], h2, mask2, err);
    else if (i < m2 + m3)
      insert_tuple(e3[i - m2], h3, mask3, err);
    else
      insert_tuple(e4[i - m2 - m3], h4, mask4, err);
  }
}

// Triple incidence lists by counting and placement: counts of 3-hyperedges
// per node, then each 3-hyperedge placed at its members' cursors. The order
// within a list is that of the atomic cursors; every user of the lists
// (candidate generation, features, contributions) only enumerates them.
__global__ void k_deg3(const int4* __restrict__ e3, int64_t m, uint64_t* __restrict__ deg) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 e = e3[t];
    atomicAdd((unsigned long long*)&deg[e.x], 1ull);
    atomicAdd((unsigned long long*)&deg[e.y], 1ull);
    atomicAdd((unsigned long long*)&deg[e.z], 1ull);
  }
}

__global__ void k_place3(const int4* __restrict__ e3, int64_t m, const int64_t* __restrict__ off,
                         uint32_t* __restrict__ cursor, int32_t* __restrict__ inc) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 e = e3[t];
    inc[off[e.x] + atomicAdd(&cursor[e.x], 1u)] = (int32_t)t;
    inc[off[e.y] + atomicAdd(&cursor[e.y], 1u)] = (int32_t)t;
    inc[off[e.z] + atomicAdd(&cursor[e.z], 1u)] = (int32_t)t;
  }
}

// Pair CSR of a graph without bitmaps, from E_2 in ascending (u, v) order. Row
// x is [its pairs {u, x}, u < x, ascending] ++ [its pairs {x, v}, x < v,
// ascending]; the second part is a contiguous run of E_2. Step 1, per pair p =
// (u, v): both degrees (into the zeroed off2, scanned in place afterwards), the
// count of v's first-part entries (into the zeroed rev), where u's run of
// E_2 starts, and the key (v << 32) | p for the stable sort of the first
// parts by v (p < 2^31).
__global__ void k_pair_counts(const uint64_t* __restrict__ e2, int64_t m,
                              unsigned long long* __restrict__ deg,
                              unsigned long long* __restrict__ rev, int64_t* __restrict__ first,
                              uint64_t* __restrict__ keys) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t uv = e2[p], u = uv >> 32, v = uv & 0xFFFFFFFFull;
    atomicAdd(&deg[u], 1ull);
    atomicAdd(&deg[v], 1ull);
    atomicAdd(&rev[v], 1ull);
    if (p == 0 || (e2[p - 1] >> 32) != u) first[u] = p;
    keys[p] = (v << 32) | (uint64_t)p;
  }
}

// Step 2: v at u's position rev(u) + (p - first[u]); that position is where
// v lies in N2(u).
__global__ void k_place_second(const uint64_t* __restrict__ e2, int64_t m,
                               const int64_t* __restrict__ off2, const uint64_t* __restrict__ rs,
                               const int64_t* __restrict__ first, int32_t* __restrict__ adj2,
                               int2* __restrict__ pos) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t uv = e2[p];
    const int64_t u = (int64_t)(uv >> 32);
    const int32_t at = (int32_t)(rs[u + 1] - rs[u] + (uint64_t)(p - first[u]));
    adj2[off2[u] + at] = (int32_t)(uv & 0xFFFFFFFFull);
    pos[p].x = at;
  }
}

// Step 3: the keys sorted stably by v; v's run starts at rs[v] (exclusive
// prefix of rev) and holds its pairs in E_2 order, i.e. its first-part
// entries u ascending, so the entry at sorted index i lies at i - rs[v] in
// N2(v).
__global__ void k_place_first(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ e2,
                              int64_t m, const int64_t* __restrict__ off2,
                              const uint64_t* __restrict__ rs, int32_t* __restrict__ adj2,
                              int2* __restrict__ pos) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    const int64_t v = (int64_t)(k >> 32), p = (int64_t)(k & 0xFFFFFFFFull);
    const int32_t at = (int32_t)((uint64_t)i - rs[v]);
    adj2[off2[v] + at] = (int32_t)(e2[p] >> 32);
    pos[p].y = at;
  }
}

// Pair positions read off the bitmap rows: the position of v in u's row is
// the number of u's neighbours below v, a popcount of the row's words below v
// (graph-local columns), so no CSR is needed and this runs beside its chain.
__global__ void k_pairpos_bits(const uint32_t* __restrict__ bits, int32_t bw, int32_t block,
                               uint64_t inv, const uint64_t* __restrict__ e2, int64_t m,
                               int2* __restrict__ pos) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = (int32_t)(e2[p] >> 32), v = (int32_t)(e2[p] & 0xFFFFFFFFull);
    const int32_t base = block ? (int32_t)__umul64hi((uint64_t)(uint32_t)u, inv) * block : 0;
    int32_t r[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t* row = bits + (size_t)(k == 0 ? u : v) * bw;
      const int32_t c = (k == 0 ? v : u) - base;
      int32_t cnt = 0;
      for (int32_t w = 0; w < (c >> 5); ++w) cnt += __popc(__ldg(row + w));
      if (c & 31) cnt += __popc(__ldg(row + (c >> 5)) & ((1u << (c & 31)) - 1u));
      r[k] = cnt;
    }
    pos[p] = make_int2(r[0], r[1]);
  }
}

// Pair degrees from the bitmap rows, one warp per node, and the largest
// (one atomic per warp into the zeroed *mx).
__global__ void k_bits_degree(const uint32_t* __restrict__ bits, int32_t n, int32_t bw,
                              uint64_t* __restrict__ deg, int* __restrict__ mx) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  uint32_t most = 0;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const uint32_t* row = bits + (size_t)v * bw;
    uint32_t c = 0;
    for (int w = lane; w < bw; w += 32) c += __popc(__ldg(row + w));
#pragma unroll
    for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if (lane == 0) deg[v] = c;
    most = max(most, c);
  }
  if (lane == 0 && most) atomicMax(mx, (int)most);
}

// Sorted pair neighbours from the bitmap rows (the set bits of row v in
// ascending column order, offset by the first id of v's graph): one warp per
// node, 32 words per round, each lane writing its word's ids at its prefix.
__global__ void k_bits_adjacency(const uint32_t* __restrict__ bits, int32_t n, int32_t bw,
                                 int32_t block, uint64_t inv, const int64_t* __restrict__ off,
                                 int32_t* __restrict__ adj) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const uint32_t* row = bits + (size_t)v * bw;
    const int32_t base = block ? (int32_t)__umul64hi((uint64_t)v, inv) * block : 0;
    int64_t pos = off[v];
    for (int w0 = 0; w0 < bw; w0 += 32) {
      const int w = w0 + lane;
      uint32_t word = w < bw ? __ldg(row + w) : 0u;
      const uint32_t c = __popc(word);
      uint32_t incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      int64_t p = pos + (incl - c);
      while (word) {
        const int j = __ffs(word) - 1;
        word &= word - 1;
        adj[p++] = base + w * 32 + j;
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// E_2 from the pair rows (graphs with bitmaps): row u's ids above u are its
// pairs (u, v), in ascending order, so the rows in order give E_2 sorted and
// without repeats. Counts per row (one warp per row), then the pairs.
__global__ void k_upper_counts(const uint32_t* __restrict__ bits, int32_t n, int32_t bw,
                               int32_t block, uint64_t inv, uint64_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    const int32_t ul = bit_col((int32_t)u, (int32_t)u, block, inv);
    const uint32_t* row = bits + (size_t)u * bw;
    uint32_t c = 0;
    for (int32_t w = lane; w < bw; w += 32) {
      const int32_t tw = ul >> 5;
      const uint32_t above = w < tw ? 0u : w > tw ? ~0u : ((ul & 31) == 31 ? 0u : (~0u << ((ul & 31) + 1)));
      c += __popc(__ldg(row + w) & above);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[u] = c;
  }
}

__global__ void k_upper_emit(const uint32_t* __restrict__ bits, int32_t n, int32_t bw,
                             int32_t block, uint64_t inv, const uint64_t* __restrict__ off,
                             uint64_t* __restrict__ e2) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    const int32_t ul = bit_col((int32_t)u, (int32_t)u, block, inv);
    const int32_t base = (int32_t)u - ul;
    const uint32_t* row = bits + (size_t)u * bw;
    uint64_t pos = off[u];
    for (int32_t w0 = 0; w0 < bw; w0 += 32) {
      const int32_t w = w0 + lane, tw = ul >> 5;
      const uint32_t above = w < tw ? 0u : w > tw ? ~0u : ((ul & 31) == 31 ? 0u : (~0u << ((ul & 31) + 1)));
      uint32_t word = w < bw ? (__ldg(row + w) & above) : 0u;
      const uint32_t c = __popc(word);
      uint32_t incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      uint64_t p = pos + (incl - c);
      while (word) {
        const int j = __ffs(word) - 1;
        word &= word - 1;
        e2[p++] = ((uint64_t)u << 32) | (uint32_t)(base + w * 32 + j);
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

// Largest pair degree: a thread's maximum over its nodes, then one atomic per
// warp.
// The largest pair degree: one atomic per block (same-address atomics
// serialise in L2).
__global__ void __launch_bounds__(256) k_max_degree(const int64_t* __restrict__ off, int32_t n,
                                                    int* out) {
  __shared__ int wmax[8];
  int mx = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, (int)(off[v + 1] - off[v]));
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0;
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (threadIdx.x == 0 && mx > 0) atomicMax(out, mx);
  }
}

__global__ void k_edges_out(const uint64_t* __restrict__ e2, const int4* __restrict__ e34,
                            int64_t m, int s, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (s == 2) {
      out[2 * i] = (int32_t)(e2[i] >> 32);
      out[2 * i + 1] = (int32_t)(e2[i] & 0xFFFFFFFFull);
    } else {
      int4 e = e34[i];
      out[s * i] = e.x;
      out[s * i + 1] = e.y;
      out[s * i + 2] = e.z;
      if (s == 4) out[s * i + 3] = e.w;
    }
  }
}

// Slots of an open-addressing table for m keys: the power of two >= 2m (load
// <= 1/2). HM_TABLE_CAP=c (a test hook) forces c slots (rounded up to a
// power of two, at least 16) whatever m: a table smaller than its key set
// fills up, every insertion and probe still ends after one pass over the
// slots, and hm_build returns HM_ETABLEFULL.
uint64_t table_capacity(int64_t m) {
  uint64_t c = 16;
  if (const char* env = std::getenv("HM_TABLE_CAP")) {
    const long long want = std::atoll(env);
    while ((long long)c < want && c < (1ull << 40)) c <<= 1;
    return c;
  }
  while (c < (uint64_t)(2 * m)) c <<= 1;
  return c;
}

// Dense pair bitmaps: up to 32 MB for one graph; up to 1 GB for a union of
// graphs (block-diagonal rows of one block each), whose alternative is hash
// probes into tables far larger than L2.
bool use_bitmap(int64_t n, int64_t row_ids, bool union_of_graphs) {
  const char* env = std::getenv("HM_PAIR_BITMAP");
  if (env && env[0] == '0') return false;
  const int64_t bytes = n * ((row_ids + 127) / 128) * 16;
  if (env && env[0] == '1') return bytes <= (1ll << 31);
  return bytes <= (union_of_graphs ? (1ll << 30) : (32ll << 20));
}

// exact triple rows cost n * n * ceil(n/32) words: kept for one graph up to
// 64 MB (n <= ~800); HM_TRIPLE_ROWS=0 disables them
bool use_tri3(int64_t n, int32_t block) {
  if (block) return false;
  const char* env = std::getenv("HM_TRIPLE_ROWS");
  if (env && env[0] == '0') return false;
  const int64_t bytes = n * n * ((n + 127) / 128) * 16;
  if (env && env[0] == '1') return bytes <= (1ll << 31);
  return bytes <= (64ll << 20);
}

template <class T>
T* keep(hm_graph* g, T* p) {
  if (p) g->owned.push_back((void*)p);
  return p;
}

}  // namespace

void build_graph(hm_graph* g, const int32_t* d_members, const int64_t* d_offsets, int64_t m,
                 int32_t n, int kmax, cudaStream_t s, int32_t block) {
  keep_pool_memory();
  g->n = n;
  g->kmax = kmax;
  g->block = block;
  g->m_in = m;
  HM_CUDA(cudaGetDevice(&g->device));
  const int b = bits_for((int64_t)n - 1);
  g->bits = b;

  TraceSpan span_norm("ingest_normalize", s);
  // counters of the normalisation pass, the error word and two more words
  // (maximum degree, error word of the structures), zeroed at once
  DBuf<unsigned long long> counters(17, s);
  HM_CUDA(cudaMemsetAsync(counters.p, 0, 17 * sizeof(unsigned long long), s));
  unsigned long long* cnt = counters.p;
  int* err_p = reinterpret_cast<int*>(counters.p + 16);
  const bool bitmaps = use_bitmap(n, block ? block : n, block != 0);
  const bool tri_rows = bitmaps && kmax >= 3 && use_tri3(n, block);
  size_t words = 0, tw = 0;
  auto al = [](size_t bytes) { return (bytes + 255) & ~(size_t)255; };
  size_t bb = 0;
  if (bitmaps) {
    // rows padded to a multiple of four words: 16-byte aligned row loads
    g->bwords = (((block ? block : n) + 127) / 128) * 4;
    words = (size_t)n * g->bwords;
    if (tri_rows) tw = (size_t)n * n * g->bwords;
    bb = al(words * 4);
  }
  const size_t bits_bytes = bitmaps ? 3 * bb + al(tw * 4) : 0;
  // One pass normalises and counts: the bitmaps (kept by the graph) and the
  // sort keys of every hyperedge that could be kept (m per size, temporary)
  // exist before it, so no counting pass has to size them first.
  BitsOut bo{};
  if (bitmaps) {
    unsigned char* bits = keep(g, dalloc<unsigned char>(bits_bytes, s));
    HM_CUDA(cudaMemsetAsync(bits, 0, bits_bytes, s));
    g->bits2 = reinterpret_cast<uint32_t*>(bits);
    g->bits3 = reinterpret_cast<uint32_t*>(bits + bb);
    g->bits4 = reinterpret_cast<uint32_t*>(bits + 2 * bb);
    if (tw) g->tri3 = reinterpret_cast<uint32_t*>(bits + 3 * bb);
    const hm::DevGraph gv = g->view();
    bo = BitsOut{g->bits2, g->bits3, g->bits4, g->tri3, g->bwords, gv.block, n, gv.block_inv};
  }
  const size_t u2 = bitmaps ? 0 : (size_t)m, u3 = kmax >= 3 ? (size_t)m : 0,
               u4 = kmax >= 4 ? (size_t)m : 0;
  DBuf<uint64_t> keybuf(u2 + 2 * u3 + 2 * u4, s);
  uint64_t* c2 = keybuf.p;
  uint64_t* c3hi = c2 + u2;
  uint64_t* c3lo = c3hi + u3;
  uint64_t* c4hi = c3lo + u3;
  uint64_t* c4lo = c4hi + u4;
  if (m > 0) {
    if (bitmaps)
      k_normalize<2><<<norm_grid(m), NORM_THREADS, 0, s>>>(d_members, d_offsets, m, n, kmax, b,
                                                          cnt, err_p, c2, c3hi, c3lo, c4hi, c4lo,
                                                          bo);
    else
      k_normalize<1><<<norm_grid(m), NORM_THREADS, 0, s>>>(d_members, d_offsets, m, n, kmax, b,
                                                          cnt, err_p, c2, c3hi, c3lo, c4hi, c4lo,
                                                          bo);
    HM_KCHECK();
  }
  span_norm.end();
  uint64_t* pin = pinned_words();
  HM_CUDA(cudaMemcpyAsync(pin, counters.p, 17 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  unsigned long long hc[8];
  for (int i = 0; i < 8; ++i) hc[i] = pin[i];
  int herr = (int)(uint32_t)pin[16];
  HM_CHECK(!(herr & ERR_OFFSETS), HM_EINVAL, "offsets are negative or not non-decreasing");
  HM_CHECK(!(herr & ERR_RANGE), HM_EINVAL, "a member lies outside [0, num_nodes)");
  g->counts[0] = n;
  g->counts[1] = m;
  g->counts[kmax + 1] = (int64_t)hc[kmax + 1];

  TraceSpan span_sort("ingest_sort_unique", s);
  // Two allocations for this phase: one the graph keeps (E_2 / E_3 / E_4,
  // sized for the hyperedges before dedup) and one of temporaries with its
  // zeroed part first (kept counts, sort scratch, pair-row counts).
  const size_t h2n = hc[2], h3n = kmax >= 3 ? hc[3] : 0, h4n = kmax >= 4 ? hc[4] : 0;
  const size_t b2 = al(h2n * 8), b3 = al(h3n * 16);
  unsigned char* owned = keep(g, dalloc<unsigned char>(b2 + b3 + h4n * 16 + 256, s));
  g->e2 = reinterpret_cast<uint64_t*>(owned);
  if (h3n) g->e3 = reinterpret_cast<int4*>(owned + b2);
  if (h4n) g->e4 = reinterpret_cast<int4*>(owned + b2 + b3);
  // Sort keys: every size without bitmaps; with bitmaps only the 3- and
  // 4-hyperedges (pairs are read off the pair rows, sorted and without repeats
  // by construction). E_2, E_3, E_4 come out in ascending order in their final
  // layout; their sizes land in kept[] (one synchronisation).
  SortJob jobs[3];
  int nj = 0;
  // kept_base: where the counts will live (the sizing pass only needs which
  // words exist)
  auto make_jobs = [&](uint64_t* kept_base) {
    nj = 0;
    auto add = [&](uint64_t* lo, uint64_t* hi, int64_t count, int size, int unpack, void* out) {
      SortJob& J = jobs[nj];
      J = SortJob{};
      J.a = lo;
      J.b = hi;
      J.b_is_key = hi != nullptr;
      J.n = count;
      const int bits = size * b, lo_bits = bits > 64 ? 64 : bits, hi_bits = bits - lo_bits;
      for (int sh = 0; sh < lo_bits; sh += 8) {
        J.arr[J.passes] = 0;
        J.shift[J.passes++] = (int8_t)sh;
      }
      for (int sh = 0; sh < hi_bits; sh += 8) {
        J.arr[J.passes] = 1;
        J.shift[J.passes++] = (int8_t)sh;
      }
      J.unique = 1;
      J.unpack = unpack;
      J.member_bits = b;
      J.out = out;
      // the count, 32 bits, into the low half of a zeroed 64-bit slot
      J.d_kept = reinterpret_cast<uint32_t*>(kept_base + (size - 2));
      ++nj;
    };
    if (!bitmaps) add(c2, nullptr, (int64_t)h2n, 2, SortJob::PAIR, g->e2);
    if (kmax >= 3) add(c3lo, c3hi, (int64_t)h3n, 3, SortJob::TRIPLE, g->e3);
    if (kmax >= 4) add(c4lo, c4hi, (int64_t)h4n, 4, SortJob::QUAD, g->e4);
  };
  size_t sort_zero = 0, sort_bytes = 0;
  {
    uint64_t sizing[1];  // never dereferenced: only non-null matters
    make_jobs(sizing);
    if (nj) sort_bytes = sort_batch_scratch(jobs, nj, &sort_zero);
  }
  const size_t o_sort = 256, o_rc = o_sort + al(sort_bytes);
  DBuf<unsigned char> tmp(o_rc + ((size_t)n + 1) * 8, s);
  uint64_t* kept = reinterpret_cast<uint64_t*>(tmp.p);
  uint64_t* rc2 = reinterpret_cast<uint64_t*>(tmp.p + o_rc);
  HM_CUDA(cudaMemsetAsync(tmp.p, 0, o_sort + sort_zero, s));
  make_jobs(kept);
  if (bitmaps) {
    // pair rows -> E_2 (f[0]), sorts (s)
    Fork f(s, 1);
    const hm::DevGraph gv = g->view();
    k_upper_counts<<<grid1d((int64_t)n * 32), T256, 0, f[0]>>>(g->bits2, n, g->bwords, gv.block,
                                                               gv.block_inv, rc2);
    HM_KCHECK();
    ScanJob sj{rc2, n, kept};
    scan_batch_inplace(&sj, 1, f[0]);
    k_upper_emit<<<grid1d((int64_t)n * 32), T256, 0, f[0]>>>(g->bits2, n, g->bwords, gv.block,
                                                             gv.block_inv, rc2, g->e2);
    HM_KCHECK();
    if (nj) sort_batch(jobs, nj, s, tmp.p + o_sort, true);
    f.join();
  } else if (nj) {
    sort_batch(jobs, nj, s, tmp.p + o_sort, true);
  }
  span_sort.end();
  uint64_t* hk = pin + 32;
  HM_CUDA(cudaMemcpyAsync(hk, kept, 3 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  const int64_t m2 = (int64_t)hk[0], m3 = kmax >= 3 ? (int64_t)hk[1] : 0,
                m4 = kmax >= 4 ? (int64_t)hk[2] : 0;
  g->counts[2] = m2;
  if (kmax >= 3) g->counts[3] = m3;
  if (kmax >= 4) g->counts[4] = m4;
  tmp.release();
  keybuf.release();

  TraceSpan span_tables("ingest_structures", s);
  // Outputs and temporaries on `s`; then three independent chains run
  // concurrently: hash sets (s), pair CSR + pair positions (f[0]), triple
  // incidence CSR (f[1]).
  const uint64_t cap2 = table_capacity(m2), cap3 = m3 ? table_capacity(m3) : 0,
                 cap4 = m4 ? table_capacity(m4) : 0;
  g->h2_mask = cap2 - 1;
  g->h3_mask = cap3 ? cap3 - 1 : 0;
  g->h4_mask = cap4 ? cap4 - 1 : 0;
  // One allocation for the graph's structures, laid out so that two memsets
  // initialise them: the hash tables (empty = all ones), then the regions that
  // start at zero (triple offsets, triple cursors), then the rest (with the
  // pair degrees of the bitmap CSR).
  uint32_t* cursor3 = nullptr;
  uint64_t* pdeg = nullptr;
  {
    auto al = [](size_t bytes) { return (bytes + 255) & ~(size_t)255; };
    size_t o = 0;
    const size_t o_h2 = o;
    o += al(cap2 * 8);
    const size_t o_h3 = o;
    o += al(cap3 * 16);
    const size_t o_h4 = o;
    o += al(cap4 * 16);
    const size_t ff_end = o;
    const size_t o_off3 = o;
    o += al(((size_t)n + 1) * 8);
    const size_t o_cur3 = o;
    o += al(((size_t)n + 1) * 4);
    const size_t o_sig = o;
    if (!bitmaps) o += al((size_t)3 * n * 8);
    const size_t o_off2 = o;  // pair degrees are counted into it (no bitmaps)
    o += al(((size_t)n + 1) * 8);
    const size_t zero_end = o;
    const size_t o_adj2 = o;
    o += al((size_t)2 * m2 * 4);
    const size_t o_pp = o;
    o += al((size_t)m2 * 8);
    const size_t o_inc3 = o;
    o += al((size_t)3 * m3 * 4);
    const size_t o_pdeg = o;
    if (bitmaps) o += al((size_t)n * 8);
    unsigned char* arena = keep(g, dalloc<unsigned char>(o, s));
    cursor3 = reinterpret_cast<uint32_t*>(arena + o_cur3);
    if (!bitmaps) g->sig = reinterpret_cast<uint64_t*>(arena + o_sig);
    if (bitmaps) pdeg = reinterpret_cast<uint64_t*>(arena + o_pdeg);
    g->h2 = reinterpret_cast<uint64_t*>(arena + o_h2);
    if (m3) g->h3 = reinterpret_cast<int4*>(arena + o_h3);
    if (m4) g->h4 = reinterpret_cast<int4*>(arena + o_h4);
    g->off3 = reinterpret_cast<int64_t*>(arena + o_off3);
    g->off2 = reinterpret_cast<int64_t*>(arena + o_off2);
    g->adj2 = reinterpret_cast<int32_t*>(arena + o_adj2);
    if (m2) g->pairpos = reinterpret_cast<int2*>(arena + o_pp);
    if (m3) g->inc3 = reinterpret_cast<int32_t*>(arena + o_inc3);
    HM_CUDA(cudaMemsetAsync(arena, 0xFF, ff_end, s));
    HM_CUDA(cudaMemsetAsync(arena + ff_end, 0, zero_end - ff_end, s));
  }
  // temporaries of the chains (without bitmaps): per node the count of its
  // pairs to lower ids, scanned (zeroed, n + 1) and where its run of E_2
  // starts (n); per pair a sort key. The maximum pair degree goes to the
  // zeroed counter word beside the error word.
  HM_CHECK(m2 < (1ll << 31), HM_EUNSUPPORTED, "2^31 or more distinct pairs");
  const size_t csr_words = bitmaps ? 0 : ((size_t)n + 1) + (size_t)n + (size_t)m2;
  DBuf<uint64_t> csr_buf(csr_words, s);
  uint64_t* rs = csr_buf.p;
  int64_t* first = bitmaps ? nullptr : reinterpret_cast<int64_t*>(csr_buf.p + n + 1);
  uint64_t* pkeys = bitmaps ? nullptr : csr_buf.p + 2 * (size_t)n + 1;
  if (!bitmaps) HM_CUDA(cudaMemsetAsync(rs, 0, ((size_t)n + 1) * 8, s));
  int* mx_p = reinterpret_cast<int*>(counters.p + 15);

  {
    Fork f(s, 2);
    // hash sets (load <= 0.5), all sizes in one launch
    if (m2 + m3 + m4) {
      k_insert_all<<<grid1d(m2 + m3 + m4), T256, 0, s>>>(g->e2, m2, g->e3, m3, g->e4, m4, g->h2,
                                                         g->h2_mask, g->h3, g->h3_mask, g->h4,
                                                         g->h4_mask, err_p);
      HM_KCHECK();
      if (g->sig) {
        k_signatures<<<grid1d(m2 + m3 + m4), T256, 0, s>>>(
            g->e2, m2, g->e3, m3, g->e4, m4, n, reinterpret_cast<unsigned long long*>(g->sig));
        HM_KCHECK();
      }
    }
    // CSR of pair neighbours, sorted, and the position of each pair in it:
    // read off the pair bitmap where there is one, else a stable sort
    if (bitmaps) {
      const hm::DevGraph gv = g->view();
      k_bits_degree<<<grid1d((int64_t)n * 32), T256, 0, f[0]>>>(g->bits2, n, g->bwords,
                                                                 pdeg, mx_p);
      HM_KCHECK();
      scan_exclusive_u64(pdeg, reinterpret_cast<uint64_t*>(g->off2), n, f[0]);
      k_bits_adjacency<<<grid1d((int64_t)n * 32), T256, 0, f[0]>>>(
          g->bits2, n, g->bwords, gv.block, gv.block_inv, g->off2, g->adj2);
      HM_KCHECK();
    } else if (m2) {
      // degrees and counts, offsets (both scans in one launch), the rows'
      // second parts straight from E_2, the first parts after a stable sort
      // of one key per pair by its larger node; pair positions fall out of
      // the placement
      k_pair_counts<<<grid1d(m2), T256, 0, f[0]>>>(
          g->e2, m2, reinterpret_cast<unsigned long long*>(g->off2),
          reinterpret_cast<unsigned long long*>(rs), first, pkeys);
      HM_KCHECK();
      ScanJob sj[2] = {{reinterpret_cast<uint64_t*>(g->off2), n, nullptr}, {rs, n, nullptr}};
      scan_batch_inplace(sj, 2, f[0]);
      k_place_second<<<grid1d(m2), T256, 0, f[0]>>>(g->e2, m2, g->off2, rs, first, g->adj2,
                                                    g->pairpos);
      HM_KCHECK();
      radix_sort_u64(pkeys, nullptr, m2, b, f[0], 32);
      k_place_first<<<grid1d(m2), T256, 0, f[0]>>>(pkeys, g->e2, m2, g->off2, rs, g->adj2,
                                                   g->pairpos);
      HM_KCHECK();
    }
    if (m2 && bitmaps) {  // positions from the rows, beside the hash inserts
      const hm::DevGraph gv = g->view();
      k_pairpos_bits<<<grid1d(m2), T256, 0, s>>>(g->bits2, g->bwords, gv.block, gv.block_inv,
                                                  g->e2, m2, g->pairpos);
      HM_KCHECK();
    }
    if (!bitmaps) {  // with bitmaps k_bits_degree took the maximum
      k_max_degree<<<grid1d(n), T256, 0, f[0]>>>(g->off2, n, mx_p);
      HM_KCHECK();
    }
    // triple incidence lists: counts (into off3, zeroed), offsets, placement
    if (m3) {
      k_deg3<<<grid1d(m3), T256, 0, f[1]>>>(g->e3, m3, reinterpret_cast<uint64_t*>(g->off3));
      HM_KCHECK();
      ScanJob oj{reinterpret_cast<uint64_t*>(g->off3), n, nullptr};
      scan_batch_inplace(&oj, 1, f[1]);
      k_place3<<<grid1d(m3), T256, 0, f[1]>>>(g->e3, m3, g->off3, cursor3, g->inc3);
      HM_KCHECK();
    }
    f.join();
  }
  span_tables.end();
  // the census work spaces of max_order, ready before the final
  // synchronisation (a census then starts without one)
  PendingSpaces pend;
  spaces_enqueue(g, census_spaces(g, kmax), s, pend);
  uint64_t* tail = pin + 40;  // max degree, error word (adjacent counter words)
  unsigned* timeouts = reinterpret_cast<unsigned*>(pin + 80);
  try {
    HM_CUDA(cudaMemcpyAsync(tail, counters.p + 15, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    wait_timeouts_async(timeouts, s);
    HM_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    for (uint64_t* p : pend.made) cudaFreeAsync(p, s);
    throw;
  }
  g->max_d2 = (int)(uint32_t)tail[0];
  herr = (int)(uint32_t)tail[1];
  spaces_finish(pend);
  choose_variants(g, kmax);
  wait_timeouts_check(*timeouts, s);
  HM_CHECK(!(herr & ERR_TABLE), HM_ETABLEFULL, "hash insertion exceeded its probe bound");
}

// Freed memory stays in the device pool for the next graph instead of going
// back to the system (a process-local setting of this device's default pool).
void keep_pool_memory() {
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep_all = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep_all);
  }
  done[dev] = true;
}

void free_graph(hm_graph* g) {
  if (!g) return;
  // work that reads the graph may still be queued on any stream
  cudaDeviceSynchronize();
  for (void* p : g->owned) cudaFreeAsync(p, 0);  // includes the work spaces
  delete g;
}

}  // namespace hm

extern "C" {

const char* hm_last_error(void) { return hm::g_last_error.c_str(); }

const char* hm_version(void) { return "hm 0.1 (sm_103a)"; }

hm_status hm_build(const int32_t* d_members, const int64_t* d_offsets, int64_t num_hyperedges,
                   int32_t num_nodes, int max_order, void* stream, hm_graph** out) {
  hm_graph* g = nullptr;
  hm_status st = hm::guarded([&] {
    HM_CHECK(out != nullptr, HM_EINVAL, "out is NULL");
    *out = nullptr;
    HM_CHECK(max_order == 3 || max_order == 4, HM_EINVAL, "max_order must be 3 or 4");
    HM_CHECK(num_nodes >= 1, HM_EINVAL, "num_nodes must be >= 1");
    HM_CHECK(num_hyperedges >= 0 && num_hyperedges < (1ll << 31), HM_EINVAL,
             "num_hyperedges must be in [0, 2^31)");
    HM_CHECK(num_hyperedges == 0 || (d_members && d_offsets), HM_EINVAL,
             "members/offsets are NULL");
    g = new hm_graph;
    hm::build_graph(g, d_members, d_offsets, num_hyperedges, num_nodes, max_order,
                    (cudaStream_t)stream);
    *out = g;
  });
  if (st != HM_OK && g) {
    std::string msg = hm_last_error();
    hm::free_graph(g);
    hm::set_last_error(msg);
  }
  return st;
}

hm_status hm_graph_info(const hm_graph* g, int64_t* counts) {
  return hm::guarded([&] {
    HM_CHECK(g && counts, HM_EINVAL, "NULL argument");
    for (int i = 0; i < 8; ++i) counts[i] = g->counts[i];
  });
}

hm_status hm_graph_edges(const hm_graph* g, int s, int32_t* d_out, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g, HM_EINVAL, "NULL graph");
    HM_CHECK(s >= 2 && s <= g->kmax, HM_EINVAL, "size must be in [2, max_order]");
    int64_t m = g->counts[s];
    if (m == 0) return;
    HM_CHECK(d_out, HM_EINVAL, "NULL output");
    cudaStream_t st = (cudaStream_t)stream;
    hm::k_edges_out<<<hm::grid1d(m), 256, 0, st>>>(g->e2, s == 3 ? g->e3 : g->e4, m, s, d_out);
    HM_KCHECK();
  });
}

void hm_free(hm_graph* g) { hm::free_graph(g); }

}  // extern "C"
