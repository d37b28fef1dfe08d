// Alg. 4 at order 5 (Sec. 6.4: the sampler opens motifs of five nodes, which
// exact counting cannot reach).
//
// A 5-node pattern is a 26-bit mask over the subsets of its five sorted
// positions with 2..5 members (by size, then lexicographic: bits 0-9 the
// pairs 01..34, 10-19 the triples 012..234, 20-24 the quads 0123..1234, 25
// the five). There is no class table (2^26 masks): a class is its canonical
// mask, the minimum over the 120 relabelings, and counts go to a direct
// 2^26-entry histogram.
//
// Draw t of stratum s is hyperedge mulhi64(v, |E_s|) of E_s (ascending), v
// the 64-bit Philox4x32-10 value of counter (t, s, "SAMP"), as at order 4.
// The sets counted for a drawn e are the 5-node V' containing e with H[V']
// connected and largest hyperedges of |e| members. All hyperedges inside such
// a V' have at most |e| members, so V' is connected in the projection P_s of
// the hyperedges of size 2..s; one warp per draw enumerates those supersets
// of e by ESU with e as the seed (each connected superset once: ESU on the
// graph with e contracted to one root), then fills each in against the
// hypergraph, keeps it if it passes the rule and is connected, and counts
// its canonical mask. Phase A (a warp per draw) writes each draw's root
// extension; phase B takes one warp per (draw, first node added), so that a
// draw at a hub spreads over many warps. Extension lists live in fixed-size
// slots of scratch: a list at depth c holds at most c times the largest
// projection degree.
#include <algorithm>
#include <vector>

#include "hm_internal.cuh"

namespace hm {
namespace {

constexpr uint32_t TAG_SAMPLE5 = 0x53414D50u;  // "SAMP", as at order 4
constexpr int O5_WARPS = 8;                     // warps per block
constexpr uint32_t NOT_COUNTED = 0xFFFFFFFFu;

// subset tables of five positions (host-built, copied to shared memory)
struct Sub5Tables {
  uint8_t perm[120][26];  // image of subset b under relabeling p
  uint8_t members[26];    // node bitmask of subset b
  uint8_t size[26];
};

Sub5Tables make_tables() {
  Sub5Tables t{};
  int index_of[32];
  for (int i = 0; i < 32; ++i) index_of[i] = -1;
  int b = 0;
  // combinations of each size, lexicographic
  for (int sz = 2; sz <= 5; ++sz) {
    int c[5];
    for (int i = 0; i < sz; ++i) c[i] = i;
    while (true) {
      uint32_t m = 0;
      for (int i = 0; i < sz; ++i) m |= 1u << c[i];
      t.members[b] = (uint8_t)m;
      t.size[b] = (uint8_t)sz;
      index_of[m] = b;
      ++b;
      int i = sz - 1;
      while (i >= 0 && c[i] == 5 - sz + i) --i;
      if (i < 0) break;
      ++c[i];
      for (int j = i + 1; j < sz; ++j) c[j] = c[j - 1] + 1;
    }
  }
  int perm[5] = {0, 1, 2, 3, 4};
  int p = 0;
  do {
    for (int q = 0; q < 26; ++q) {
      uint32_t img = 0;
      for (int i = 0; i < 5; ++i)
        if ((t.members[q] >> i) & 1u) img |= 1u << perm[i];
      t.perm[p][q] = (uint8_t)index_of[img];
    }
    ++p;
  } while (std::next_permutation(perm, perm + 5));
  return t;
}

// 5-member hyperedges: packed sorted keys, b bits per member, most
// significant first (as 128-bit hi:lo)
struct Quint {
  uint64_t hi, lo;
};

__device__ __forceinline__ Quint pack5(const int32_t* v, int b) {
  unsigned __int128 k = 0;
  for (int i = 0; i < 5; ++i) k = (k << b) | (unsigned __int128)(uint32_t)v[i];
  return Quint{(uint64_t)(k >> 64), (uint64_t)k};
}

__device__ __forceinline__ void unpack5(uint64_t hi, uint64_t lo, int b, int32_t* v) {
  unsigned __int128 k = ((unsigned __int128)hi << 64) | lo;
  const unsigned __int128 mask = ((unsigned __int128)1 << b) - 1;
  for (int i = 4; i >= 0; --i) {
    v[i] = (int32_t)(uint32_t)(k & mask);
    k >>= b;
  }
}

__device__ __forceinline__ uint64_t hash_quint(uint64_t hi, uint64_t lo) {
  return mix64(hi ^ mix64(lo + 0x9E3779B97F4A7C15ull));
}

struct Five {
  const int32_t* e5;  // [m5][5] ascending
  int64_t m5;
  const ulonglong2* h5;  // slots (hi, lo), empty hi = ~0
  uint64_t h5_mask;
  int bits;
  // memo of raw mask -> canonical mask (MEMO_DISCONNECTED, or MEMO_UNKNOWN
  // before the first time a mask is met); every writer of an entry writes
  // the same value
  uint32_t* memo;
};
constexpr uint32_t MEMO_UNKNOWN = 0xFFFFFFFFu, MEMO_DISCONNECTED = 0xFFFFFFFEu;

__device__ __forceinline__ bool has_quint(const Five& F, const int32_t* v) {
  if (F.m5 == 0) return false;
  const Quint k = pack5(v, F.bits);
  uint64_t slot = hash_quint(k.hi, k.lo) & F.h5_mask;
  for (uint64_t it = 0; it <= F.h5_mask; ++it) {
    const ulonglong2 s = F.h5[slot];
    if (s.x == k.hi && s.y == k.lo) return true;
    if (s.x == EMPTY64) return false;
    slot = (slot + 1) & F.h5_mask;
  }
  return false;
}

// hyperedges with exactly five distinct members, as packed keys
__global__ void k_quint_keys(const int32_t* __restrict__ mem, const int64_t* __restrict__ off,
                             int64_t m, int b, uint32_t* __restrict__ flag,
                             uint64_t* __restrict__ hi, uint64_t* __restrict__ lo) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[6];
    int nd = 0;
    bool over = false;
    for (int64_t p = off[e]; p < off[e + 1] && !over; ++p) {
      const int32_t x = mem[p];
      int i = 0;
      while (i < nd && v[i] < x) ++i;
      if (i < nd && v[i] == x) continue;
      if (nd == 5) {
        over = true;  // a sixth distinct member
        break;
      }
      for (int j = nd; j > i; --j) v[j] = v[j - 1];
      v[i] = x;
      ++nd;
    }
    const bool five = !over && nd == 5;
    flag[e] = five ? 1u : 0u;
    if (five) {
      const Quint k = pack5(v, b);
      hi[e] = k.hi;
      lo[e] = k.lo;
    } else {
      hi[e] = ~0ull;  // sorts last
      lo[e] = ~0ull;
    }
  }
}

__global__ void k_gather_u64(const uint64_t* __restrict__ src, const uint64_t* __restrict__ idx,
                             int64_t n, uint64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = src[idx[i]];
}

__global__ void k_iota(int64_t n, uint64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint64_t)i;
}

// keep[j] = sorted key j is a quint and differs from key j - 1
__global__ void k_quint_keep(const uint64_t* __restrict__ hi, const uint64_t* __restrict__ lo,
                             int64_t n, uint64_t* __restrict__ keep) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const bool real = hi[j] != ~0ull;
    keep[j] = (real && (j == 0 || hi[j] != hi[j - 1] || lo[j] != lo[j - 1])) ? 1u : 0u;
  }
}

__global__ void k_quint_emit(const uint64_t* __restrict__ hi, const uint64_t* __restrict__ lo,
                             const uint64_t* __restrict__ keep, const uint64_t* __restrict__ pos,
                             int64_t n, int b, int32_t* __restrict__ e5, ulonglong2* __restrict__ h5,
                             uint64_t h5_mask) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[j]) continue;
    const uint64_t q = pos[j];
    unpack5(hi[j], lo[j], b, e5 + 5 * q);
    uint64_t slot = hash_quint(hi[j], lo[j]) & h5_mask;
    for (uint64_t it = 0; it <= h5_mask; ++it) {
      if (atomicCAS((unsigned long long*)&h5[slot].x, (unsigned long long)EMPTY64,
                    (unsigned long long)hi[j]) == EMPTY64) {
        h5[slot].y = lo[j];
        break;
      }
      slot = (slot + 1) & h5_mask;
    }
  }
}

// pairs of E_2, E_3 (and E_4) as 2-member hyperedges: the projection of the
// hyperedges of size 2..s
__global__ void k_proj_pairs(const DevGraph g, int s, int32_t* __restrict__ out) {
  const int64_t n3 = s >= 3 ? g.m3 : 0, n4 = s >= 4 ? g.m4 : 0;
  const int64_t total = g.m2 + 3 * n3 + 6 * n4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t a, b;
    if (i < g.m2) {
      a = (int32_t)(g.e2[i] >> 32);
      b = (int32_t)(g.e2[i] & 0xFFFFFFFFull);
    } else if (i < g.m2 + 3 * n3) {
      const int64_t j = i - g.m2;
      const int4 t = g.e3[j / 3];
      const int r = (int)(j % 3);
      a = r == 2 ? t.y : t.x;
      b = r == 0 ? t.y : t.z;
    } else {
      const int64_t j = i - g.m2 - 3 * n3;
      const int4 t = g.e4[j / 6];
      const int r = (int)(j % 6);  // 01 02 03 12 13 23
      const int32_t m[4] = {t.x, t.y, t.z, t.w};
      const int ia = r < 3 ? 0 : (r < 5 ? 1 : 2);
      const int ib = r < 3 ? r + 1 : (r < 5 ? r - 1 : 3);
      a = m[ia];
      b = m[ib];
    }
    out[2 * i] = a;
    out[2 * i + 1] = b;
  }
}

__global__ void k_even(int64_t n, int64_t* __restrict__ off) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x)
    off[i] = 2 * i;
}

// Fill-in of a 5-node set drawn from stratum s: its canonical mask, or
// NOT_COUNTED when it holds a hyperedge larger than s or is disconnected.
__device__ uint32_t evaluate5(const DevGraph& g, const Five& F, const Sub5Tables& T, int s,
                              int32_t a0, int32_t a1, int32_t a2, int32_t a3, int32_t a4) {
  int32_t v[5] = {a0, a1, a2, a3, a4};
  // sort (insertion; five elements)
  for (int i = 1; i < 5; ++i) {
    const int32_t x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) {
      v[j + 1] = v[j];
      --j;
    }
    v[j + 1] = x;
  }
  uint32_t mask = 0;
  if (s < 5 && has_quint(F, v)) return NOT_COUNTED;
  for (int q = 20; q < 25; ++q) {  // quads
    const uint8_t mb = T.members[q];
    int32_t w[4];
    int c = 0;
    for (int i = 0; i < 5; ++i)
      if ((mb >> i) & 1u) w[c++] = v[i];
    if (has_quad(g, w[0], w[1], w[2], w[3])) {
      if (s < 4) return NOT_COUNTED;
      mask |= 1u << q;
    }
  }
  for (int q = 10; q < 20; ++q) {  // triples
    const uint8_t mb = T.members[q];
    int32_t w[3];
    int c = 0;
    for (int i = 0; i < 5; ++i)
      if ((mb >> i) & 1u) w[c++] = v[i];
    if (has_triple(g, w[0], w[1], w[2])) {
      if (s < 3) return NOT_COUNTED;
      mask |= 1u << q;
    }
  }
  for (int q = 0; q < 10; ++q) {  // pairs
    const uint8_t mb = T.members[q];
    int32_t w[2];
    int c = 0;
    for (int i = 0; i < 5; ++i)
      if ((mb >> i) & 1u) w[c++] = v[i];
    if (has_pair(g, w[0], w[1])) mask |= 1u << q;
  }
  if (s == 5) mask |= 1u << 25;  // the drawn hyperedge itself
  const uint32_t known = F.memo[mask];
  if (known == MEMO_DISCONNECTED) return NOT_COUNTED;
  if (known != MEMO_UNKNOWN) return known;
  // connectivity over the five positions
  int parent[5] = {0, 1, 2, 3, 4};
  for (int q = 0; q < 26; ++q) {
    if (!((mask >> q) & 1u)) continue;
    const uint8_t mb = T.members[q];
    int first = -1;
    for (int i = 0; i < 5; ++i) {
      if (!((mb >> i) & 1u)) continue;
      if (first < 0) {
        first = i;
      } else {
        int x = i, y = first;
        while (parent[x] != x) x = parent[x];
        while (parent[y] != y) y = parent[y];
        parent[x] = y;
      }
    }
  }
  int r0 = 0;
  while (parent[r0] != r0) r0 = parent[r0];
  for (int i = 1; i < 5; ++i) {
    int x = i;
    while (parent[x] != x) x = parent[x];
    if (x != r0) {
      F.memo[mask] = MEMO_DISCONNECTED;
      return NOT_COUNTED;
    }
  }
  // canonical form: the smallest image over the 120 relabelings
  uint32_t best = mask;
  for (int p = 0; p < 120; ++p) {
    uint32_t r = 0, rest = mask;
    while (rest) {
      const int q = __ffs(rest) - 1;
      rest &= rest - 1;
      r |= 1u << T.perm[p][q];
    }
    best = min(best, r);
  }
  F.memo[mask] = best;
  return best;
}

__device__ __forceinline__ void count5(uint32_t key, unsigned long long* hist) {
  const unsigned peers = __match_any_sync(__activemask(), key);
  if (key != NOT_COUNTED && (threadIdx.x & 31) == __ffs(peers) - 1)
    atomicAdd(&hist[key], (unsigned long long)__popc(peers));
}

// Appends the members of a warp-wide predicate to list (warp-uniform *len).
__device__ __forceinline__ void warp_append(bool take, int32_t x, int32_t* list, int32_t& len) {
  const unsigned bal = __ballot_sync(0xffffffffu, take);
  const int lane = threadIdx.x & 31;
  if (take) list[len + __popc(bal & ((1u << lane) - 1u))] = x;
  len += __popc(bal);
}

// u adjacent (in P) to any of the nodes sub[0..c)
__device__ __forceinline__ bool adj_any(const DevGraph& P, const int32_t* sub, int c, int32_t u) {
  for (int i = 0; i < c; ++i)
    if (u == sub[i] || has_pair(P, u, sub[i])) return true;
  return false;
}

// ESU extension: dst = src[from..n) followed by the neighbours u of w (in P)
// outside sub[0..c) and not adjacent to any of them. Returns the length.
__device__ int32_t extend(const DevGraph& P, const int32_t* src, int32_t n, int32_t from,
                          int32_t w, const int32_t* sub, int c, int32_t* dst) {
  const int lane = threadIdx.x & 31;
  int32_t len = 0;
  for (int32_t i = from + lane; i < n; i += 32) dst[i - from] = src[i];
  len = n - from;
  const int64_t o = P.off2[w];
  const int32_t d = (int32_t)(P.off2[w + 1] - o);
  for (int32_t i0 = 0; i0 < d; i0 += 32) {
    const int32_t i = i0 + lane;
    int32_t u = 0;
    bool take = false;
    if (i < d) {
      u = P.adj2[o + i];
      take = !adj_any(P, sub, c, u);
    }
    warp_append(take, u, dst, len);
  }
  __syncwarp();
  return len;
}

__device__ __forceinline__ void load_tables(Sub5Tables& T, const Sub5Tables* __restrict__ Tg) {
  for (int i = threadIdx.x; i < (int)sizeof(Sub5Tables); i += blockDim.x)
    reinterpret_cast<uint8_t*>(&T)[i] = reinterpret_cast<const uint8_t*>(Tg)[i];
  __syncthreads();
}

// members of draw t of stratum S
template <int S>
__device__ __forceinline__ void drawn(const DevGraph& g, const Five& F, uint64_t seed, int64_t t,
                                      int64_t len_s, int32_t* sub) {
  const uint64_t idx =
      __umul64hi(philox_draw64(seed, (uint64_t)t, (uint32_t)S, TAG_SAMPLE5), (uint64_t)len_s);
  if (S == 2) {
    const uint64_t p = g.e2[idx];
    sub[0] = (int32_t)(p >> 32);
    sub[1] = (int32_t)(p & 0xFFFFFFFFull);
  } else if (S == 3) {
    const int4 h = g.e3[idx];
    sub[0] = h.x;
    sub[1] = h.y;
    sub[2] = h.z;
  } else if (S == 4) {
    const int4 h = g.e4[idx];
    sub[0] = h.x;
    sub[1] = h.y;
    sub[2] = h.z;
    sub[3] = h.w;
  } else {
    for (int i = 0; i < 5; ++i) sub[i] = F.e5[5 * idx + i];
  }
}

// Evaluates V4 + {x} for every x of L[0, n) (lanes in parallel).
__device__ __forceinline__ void finish(const DevGraph& g, const Five& F, const Sub5Tables& T,
                                       int S, const int32_t* L, int32_t n, const int32_t* v4,
                                       unsigned long long* hist) {
  const int lane = threadIdx.x & 31;
  for (int32_t i = lane; i - lane < n; i += 32) {
    uint32_t key = NOT_COUNTED;
    if (i < n) key = evaluate5(g, F, T, S, v4[0], v4[1], v4[2], v4[3], L[i]);
    count5(key, hist);
  }
}

// Phase A, one warp per draw: stratum 5 draws are evaluated; stratum 4
// draws enumerate their root extension at once; strata 2 and 3 write their
// root extension L0 (the seed's projection neighbours outside it, each once,
// from its first member in order) to slot t of `roots` (cap0 entries) and
// its length to n0[t].
template <int S>
__global__ void __launch_bounds__(O5_WARPS * 32)
    k_roots5(const DevGraph g, const DevGraph P, const Five F, const Sub5Tables* __restrict__ Tg,
             uint64_t seed, int64_t t0, int64_t draws, int64_t len_s, int64_t cap0,
             int32_t* __restrict__ roots, int32_t* __restrict__ n0, unsigned long long* hist) {
  __shared__ Sub5Tables T;
  load_tables(T, Tg);
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t d = gw; d < draws; d += nw) {
    int32_t sub[5];
    drawn<S>(g, F, seed, t0 + d, len_s, sub);
    if (S == 5) {
      const uint32_t key =
          lane == 0 ? evaluate5(g, F, T, 5, sub[0], sub[1], sub[2], sub[3], sub[4]) : NOT_COUNTED;
      count5(key, hist);
      continue;
    }
    int32_t* L0 = roots + d * cap0;
    int32_t n = 0;
    for (int m = 0; m < S; ++m) {
      const int64_t o = P.off2[sub[m]];
      const int32_t dg = (int32_t)(P.off2[sub[m] + 1] - o);
      for (int32_t i0 = 0; i0 < dg; i0 += 32) {
        const int32_t i = i0 + lane;
        int32_t u = 0;
        bool take = false;
        if (i < dg) {
          u = P.adj2[o + i];
          take = true;
          for (int j = 0; j < S; ++j) take &= u != sub[j];
          for (int j = 0; j < m; ++j) take &= !has_pair(P, u, sub[j]);
        }
        warp_append(take, u, L0, n);
      }
    }
    __syncwarp();
    if (S == 4) {
      finish(g, F, T, 4, L0, n, sub, hist);
    } else if (lane == 0) {
      n0[d] = n;
    }
  }
}

// Phase B, one warp per item (draw d, position i of its root extension): the
// first node added is w = L0[i]; the ESU subtree under it is enumerated
// here (strata 2 and 3).
template <int S>
__global__ void __launch_bounds__(O5_WARPS * 32)
    k_items5(const DevGraph g, const DevGraph P, const Five F, const Sub5Tables* __restrict__ Tg,
             uint64_t seed, int64_t t0, int64_t draws, int64_t len_s, int64_t cap0, int64_t cap,
             const int32_t* __restrict__ roots, const int32_t* __restrict__ n0,
             const uint64_t* __restrict__ item0, uint64_t items, int32_t* __restrict__ arena,
             unsigned long long* hist) {
  __shared__ Sub5Tables T;
  load_tables(T, Tg);
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* L1 = arena + gw * 2 * cap;
  int32_t* L2 = L1 + cap;
  for (uint64_t it = (uint64_t)gw; it < items; it += (uint64_t)nw) {
    int64_t lo = 0, hi = draws;  // the draw: last d with item0[d] <= it
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (item0[mid] <= it) lo = mid;
      else hi = mid;
    }
    const int64_t d = lo;
    const int32_t i = (int32_t)(it - item0[d]);
    const int32_t* L0 = roots + d * cap0;
    const int32_t nd0 = n0[d];
    int32_t sub[5];
    drawn<S>(g, F, seed, t0 + d, len_s, sub);
    const int32_t w = L0[i];
    const int32_t n1 = extend(P, L0, nd0, i + 1, w, sub, S, L1);
    sub[S] = w;
    if (S == 3) {
      finish(g, F, T, 3, L1, n1, sub, hist);
    } else {  // S == 2
      for (int32_t j = 0; j < n1; ++j) {
        const int32_t w2 = L1[j];
        const int32_t n2 = extend(P, L1, n1, j + 1, w2, sub, 3, L2);
        sub[3] = w2;
        finish(g, F, T, 2, L2, n2, sub, hist);
      }
    }
  }
}

// nonzero histogram entries in ascending key order: per-chunk counts, then writes
constexpr int64_t H5_SIZE = 1ll << 26;
constexpr int64_t H5_CHUNK = 4096;

__global__ void k_h5_count(const unsigned long long* __restrict__ hist,
                           uint64_t* __restrict__ cnt) {
  __shared__ unsigned int c;
  for (int64_t ch = blockIdx.x; ch < H5_SIZE / H5_CHUNK; ch += gridDim.x) {
    if (threadIdx.x == 0) c = 0;
    __syncthreads();
    unsigned int mine = 0;
    for (int64_t i = ch * H5_CHUNK + threadIdx.x; i < (ch + 1) * H5_CHUNK; i += blockDim.x)
      mine += hist[i] ? 1u : 0u;
    atomicAdd(&c, mine);
    __syncthreads();
    if (threadIdx.x == 0) cnt[ch] = c;
    __syncthreads();
  }
}

struct EstArgs5 {
  double S[6];
  double E[6];
  uint8_t size[26];
};

__global__ void k_h5_emit(const unsigned long long* __restrict__ hist,
                          const uint64_t* __restrict__ pos, int64_t capacity, EstArgs5 A,
                          uint32_t* __restrict__ masks, uint64_t* __restrict__ raw,
                          double* __restrict__ est) {
  // one warp per chunk, in order: ballots place the chunk's entries
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t ch = gw; ch < H5_SIZE / H5_CHUNK; ch += nw) {
    uint64_t q = pos[ch];
    for (int64_t i0 = ch * H5_CHUNK; i0 < (ch + 1) * H5_CHUNK; i0 += 32) {
      const int64_t i = i0 + lane;
      const unsigned long long v = hist[i];
      const unsigned bal = __ballot_sync(0xffffffffu, v != 0);
      if (v) {
        const uint64_t at = q + __popc(bal & ((1u << lane) - 1u));
        if ((int64_t)at < capacity) {
          const uint32_t m = (uint32_t)i;
          int mc = 0, cm = 0;
          for (int b = 0; b < 26; ++b) {
            if (!((m >> b) & 1u)) continue;
            if (A.size[b] > mc) {
              mc = A.size[b];
              cm = 1;
            } else if (A.size[b] == mc) {
              ++cm;
            }
          }
          masks[at] = m;
          raw[at] = v;
          // (n_c |E_m|) / (S_m countmax_c), in IEEE double in this order
          est[at] = A.S[mc] > 0.0 ? __ddiv_rn(__dmul_rn((double)v, A.E[mc]),
                                              __dmul_rn(A.S[mc], (double)cm))
                                  : 0.0;
        }
      }
      q += __popc(bal);
    }
  }
}

__global__ void k_widen32(const int32_t* __restrict__ in, int64_t n, uint64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint64_t)(uint32_t)in[i];
}

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

}  // namespace

int64_t count_sampled5(const int32_t* d_members, const int64_t* d_offsets, int64_t m, int32_t n,
                       const uint64_t* S, uint64_t seed, uint32_t* d_masks, uint64_t* d_raw,
                       double* d_est, int64_t capacity, cudaStream_t s) {
  hm_graph* g = new hm_graph;
  hm_graph* proj[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t nclasses = 0;
  try {
    build_graph(g, d_members, d_offsets, m, n, 4, s);
    const int b = g->bits;
    HM_CHECK(5 * b <= 125, HM_EUNSUPPORTED, "order 5 needs node ids below 2^25");
    // E_5 and its hash set
    DBuf<int32_t> e5;
    DBuf<ulonglong2> h5;
    int64_t m5 = 0;
    uint64_t h5_mask = 0;
    if (m > 0) {
      DBuf<uint32_t> flag(m, s);
      DBuf<uint64_t> hi(m, s), lo(m, s), idx(m, s), hi2(m, s), pos(m, s), keep(m + 1, s),
          kpos(m + 1, s), hs(m, s), ls(m, s);
      k_quint_keys<<<grid_n(m), 256, 0, s>>>(d_members, d_offsets, m, b, flag.p, hi.p, lo.p);
      HM_KCHECK();
      k_iota<<<grid_n(m), 256, 0, s>>>(m, idx.p);
      HM_KCHECK();
      radix_sort_u64(lo.p, idx.p, m, 64, s);  // by the low word, with the hyperedge index
      k_gather_u64<<<grid_n(m), 256, 0, s>>>(hi.p, idx.p, m, hi2.p);
      HM_KCHECK();
      k_iota<<<grid_n(m), 256, 0, s>>>(m, pos.p);
      HM_KCHECK();
      radix_sort_u64(hi2.p, pos.p, m, 64, s);  // stable by the high word
      k_gather_u64<<<grid_n(m), 256, 0, s>>>(lo.p, pos.p, m, ls.p);  // lo in final order
      HM_KCHECK();
      k_quint_keep<<<grid_n(m), 256, 0, s>>>(hi2.p, ls.p, m, keep.p);
      HM_KCHECK();
      scan_exclusive_u64(keep.p, kpos.p, m, s);
      uint64_t um5 = 0;
      HM_CUDA(cudaMemcpyAsync(&um5, kpos.p + m, sizeof um5, cudaMemcpyDeviceToHost, s));
      HM_CUDA(cudaStreamSynchronize(s));
      m5 = (int64_t)um5;
      if (m5 > 0) {
        uint64_t cap5 = 16;
        while (cap5 < 2 * (uint64_t)m5) cap5 <<= 1;
        h5_mask = cap5 - 1;
        e5.alloc(5 * m5, s);
        h5.alloc(cap5, s);
        HM_CUDA(cudaMemsetAsync(h5.p, 0xFF, cap5 * sizeof(ulonglong2), s));
        k_quint_emit<<<grid_n(m), 256, 0, s>>>(hi2.p, ls.p, keep.p, kpos.p, m, b, e5.p, h5.p,
                                               h5_mask);
        HM_KCHECK();
      }
    }
    DBuf<uint32_t> memo(H5_SIZE, s);
    HM_CUDA(cudaMemsetAsync(memo.p, 0xFF, H5_SIZE * sizeof(uint32_t), s));
    const Five F{e5.p, m5, h5.p, h5_mask, b, memo.p};
    const int64_t lens[6] = {0, 0, g->counts[2], g->counts[3], g->counts[4], m5};
    for (int st = 2; st <= 5; ++st)
      HM_CHECK(lens[st] == 0 || S[st] > 0, HM_EINVAL,
               "a non-empty stratum has no samples (S_s == 0 with |E_s| > 0)");
    // the projections of hyperedges of size 2..s, for the strata 3 and 4
    for (int st = 3; st <= 4; ++st) {
      if (S[st] == 0 || lens[st] == 0) continue;
      const int64_t np = g->counts[2] + 3 * g->counts[3] + (st == 4 ? 6 * g->counts[4] : 0);
      HM_CHECK(np < (1ll << 31), HM_EINVAL, "projection too large");
      DBuf<int32_t> pm(2 * np, s);
      DBuf<int64_t> po(np + 1, s);
      if (np) {
        k_proj_pairs<<<grid_n(np), 256, 0, s>>>(g->view(), st, pm.p);
        HM_KCHECK();
      }
      k_even<<<grid_n(np + 1), 256, 0, s>>>(np, po.p);
      HM_KCHECK();
      proj[st] = new hm_graph;
      build_graph(proj[st], pm.p, po.p, np, n, 3, s);
    }
    // the histogram over all 2^26 masks
    DBuf<unsigned long long> hist(H5_SIZE, s);
    HM_CUDA(cudaMemsetAsync(hist.p, 0, H5_SIZE * sizeof(unsigned long long), s));
    static const Sub5Tables host_tables = make_tables();
    DBuf<Sub5Tables> tables(1, s);
    HM_CUDA(cudaMemcpyAsync(tables.p, &host_tables, sizeof(Sub5Tables), cudaMemcpyHostToDevice, s));
    int sms = 0, dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int st = 2; st <= 5; ++st) {
      if (S[st] == 0 || lens[st] == 0) continue;
      const hm_graph* P = st == 2 ? g : (st == 5 ? g : proj[st]);
      const int64_t maxdeg = std::max(1, P->max_d2);
      // lists at depth c hold at most c * maxdeg entries (c <= 4)
      const int64_t cap0 = (int64_t)st * maxdeg + 32, cap = 4 * maxdeg + 32;
      const DevGraph gv = g->view(), pv = P->view();
      // draws in batches whose root lists take at most ~256 MB
      const int64_t per = std::max<int64_t>(1, std::min<int64_t>((int64_t)S[st],
                                                                 (64ll << 20) / cap0));
      for (int64_t t0 = 0; t0 < (int64_t)S[st]; t0 += per) {
        const int64_t nd = std::min<int64_t>(per, (int64_t)S[st] - t0);
        const int64_t rblocks =
            std::max<int64_t>(1, std::min<int64_t>((nd + O5_WARPS - 1) / O5_WARPS, (int64_t)sms * 8));
        DBuf<int32_t> roots(st <= 4 ? (size_t)(nd * cap0) : 1, s), n0(nd + 1, s);
        switch (st) {
          case 2:
            k_roots5<2><<<(unsigned)rblocks, O5_WARPS * 32, 0, s>>>(
                gv, pv, F, tables.p, seed, t0, nd, lens[st], cap0, roots.p, n0.p, hist.p);
            break;
          case 3:
            k_roots5<3><<<(unsigned)rblocks, O5_WARPS * 32, 0, s>>>(
                gv, pv, F, tables.p, seed, t0, nd, lens[st], cap0, roots.p, n0.p, hist.p);
            break;
          case 4:
            k_roots5<4><<<(unsigned)rblocks, O5_WARPS * 32, 0, s>>>(
                gv, pv, F, tables.p, seed, t0, nd, lens[st], cap0, roots.p, n0.p, hist.p);
            break;
          default:
            k_roots5<5><<<(unsigned)rblocks, O5_WARPS * 32, 0, s>>>(
                gv, pv, F, tables.p, seed, t0, nd, lens[st], cap0, roots.p, n0.p, hist.p);
            break;
        }
        HM_KCHECK();
        if (st >= 4) continue;
        // items (draw, first added node): prefix of the root list lengths
        DBuf<uint64_t> n64(nd + 1, s), item0(nd + 1, s);
        k_widen32<<<grid_n(nd), 256, 0, s>>>(n0.p, nd, n64.p);
        HM_KCHECK();
        scan_exclusive_u64(n64.p, item0.p, nd, s);
        uint64_t items = 0;
        HM_CUDA(cudaMemcpyAsync(&items, item0.p + nd, sizeof items, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        if (items == 0) continue;
        const int64_t iblocks = std::max<int64_t>(
            1, std::min<int64_t>(((int64_t)items + O5_WARPS - 1) / O5_WARPS, (int64_t)sms * 8));
        DBuf<int32_t> arena((size_t)(iblocks * O5_WARPS * 2 * cap), s);
        if (st == 2)
          k_items5<2><<<(unsigned)iblocks, O5_WARPS * 32, 0, s>>>(
              gv, pv, F, tables.p, seed, t0, nd, lens[st], cap0, cap, roots.p, n0.p, item0.p,
              items, arena.p, hist.p);
        else
          k_items5<3><<<(unsigned)iblocks, O5_WARPS * 32, 0, s>>>(
              gv, pv, F, tables.p, seed, t0, nd, lens[st], cap0, cap, roots.p, n0.p, item0.p,
              items, arena.p, hist.p);
        HM_KCHECK();
      }
    }
    // the classes met, ascending, with their estimates
    const int64_t nch = H5_SIZE / H5_CHUNK;
    DBuf<uint64_t> cnt(nch + 1, s), pos(nch + 1, s);
    k_h5_count<<<(unsigned)std::min<int64_t>(nch, (int64_t)sms * 8), 256, 0, s>>>(hist.p, cnt.p);
    HM_KCHECK();
    scan_exclusive_u64(cnt.p, pos.p, nch, s);
    uint64_t total = 0;
    HM_CUDA(cudaMemcpyAsync(&total, pos.p + nch, sizeof total, cudaMemcpyDeviceToHost, s));
    EstArgs5 A{};
    for (int st = 2; st <= 5; ++st) {
      A.S[st] = (double)S[st];
      A.E[st] = (double)lens[st];
    }
    for (int q = 0; q < 26; ++q) A.size[q] = host_tables.size[q];
    if (capacity > 0) {
      k_h5_emit<<<(unsigned)std::min<int64_t>((nch + 7) / 8, (int64_t)sms * 8), 256, 0, s>>>(
          hist.p, pos.p, capacity, A, d_masks, d_raw, d_est);
      HM_KCHECK();
    }
    unsigned timeouts = 0;
    wait_timeouts_async(&timeouts, s);
    HM_CUDA(cudaStreamSynchronize(s));
    wait_timeouts_check(timeouts, s);
    nclasses = (int64_t)total;
  } catch (...) {
    free_graph(g);
    for (auto* p : proj)
      if (p) free_graph(p);
    throw;
  }
  free_graph(g);
  for (auto* p : proj)
    if (p) free_graph(p);
  return nclasses;
}

}  // namespace hm

extern "C" hm_status hm_count_sampled5(const int32_t* d_members, const int64_t* d_offsets,
                                       int64_t num_hyperedges, int32_t num_nodes,
                                       const uint64_t* samples_per_size, uint64_t total_samples,
                                       uint64_t seed, uint32_t* d_masks, uint64_t* d_raw,
                                       double* d_est, int64_t capacity, int64_t* h_num_classes,
                                       void* stream) {
  return hm::guarded([&] {
    HM_CHECK(num_nodes >= 1, HM_EINVAL, "num_nodes must be >= 1");
    HM_CHECK(num_hyperedges >= 0 && num_hyperedges < (1ll << 31), HM_EINVAL,
             "num_hyperedges must be in [0, 2^31)");
    HM_CHECK(num_hyperedges == 0 || (d_members && d_offsets), HM_EINVAL, "NULL hyperedges");
    HM_CHECK(capacity >= 0 && (capacity == 0 || (d_masks && d_raw && d_est)), HM_EINVAL,
             "NULL output buffers");
    uint64_t S[6] = {0, 0, 0, 0, 0, 0};
    if (samples_per_size) {
      for (int st = 2; st <= 5; ++st) S[st] = samples_per_size[st];
    } else {
      S[2] = total_samples / 8;
      S[3] = 3 * total_samples / 8;
      S[4] = total_samples / 4;
      S[5] = total_samples - S[2] - S[3] - S[4];
    }
    const int64_t nc = hm::count_sampled5(d_members, d_offsets, num_hyperedges, num_nodes, S,
                                          seed, d_masks, d_raw, d_est, capacity,
                                          (cudaStream_t)stream);
    if (h_num_classes) *h_num_classes = nc;
  });
}
