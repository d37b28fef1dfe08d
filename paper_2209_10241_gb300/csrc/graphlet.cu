// Pairs-only 4-node sets by graphlet identities (dense graphs with pair
// bitmaps): the alternative to enumerating the S and P families.
//
// A connected 4-node set without a 3- or 4-hyperedge inside has one of the six
// connected simple-graph patterns on its pairs (star, path, paw, 4-cycle,
// diamond, 4-clique). For every 4-node set, the pattern of its pairs is counted
// from sums over the pair graph G: with d = degree, t(e) = triangles through
// pair e, t(v) = triangles at v, T = triangles, K4 = 4-cliques, and c(x, z) =
// common neighbours of a node pair,
//   S3 = sum_v C(d(v), 3)                       3-stars
//   P3 = sum_{uv in E} (d(u)-1)(d(v)-1) - 3T    3-edge paths
//   TT = sum_v t(v) (d(v) - 2)                  tailed triangles
//   D  = sum_e C(t(e), 2)                       diamonds
//   C4 = 1/2 sum_{x<z} C(c(x, z), 2)            4-cycles
// (all not necessarily induced), and the induced counts follow:
//   k4 = K4, diamond = D - 6 K4, c4 = C4 - D + 3 K4, paw = TT - 4 D + 12 K4,
//   star = S3 - paw - 2 diamond - 4 k4,
//   path = P3 - 2 paw - 4 c4 - 6 diamond - 12 k4.
// The sets that do hold a 3- or 4-hyperedge are exactly the ones the TX and Q
// families enumerate; those launches subtract each such set from the class of
// its pair pattern, so the histogram ends with the pairs-only counts. All sums
// are exact integers (uint64, subtraction modulo 2^64 with a non-negative
// result).
#include <atomic>
#include <cstdio>
#include <cstdlib>

#include "families.cuh"
#include "hm_internal.cuh"

namespace hm {
namespace {

using namespace fam;

constexpr int NAGG = 8;  // S3, P3raw, 3T, TT, D, K4, 2 C4, spare

__device__ __forceinline__ int32_t degree(const DevGraph& g, int32_t v) {
  return (int32_t)(g.off2[v + 1] - g.off2[v]);
}

constexpr int GL_WARPS = 8;      // warps per block of the pair kernel
constexpr int SPARSE_WARPS = 8;  // warps per block of the hash-probe pair kernel
constexpr int GL_MAXW = 512;     // row words kept in shared memory (n <= 16384)
constexpr int GL_LIST = 1024;    // common neighbours listed per round (32 words)

// 4-cliques of pair (u, v) over the listed common neighbours w > v: lanes take
// the listed w in turn and count the common neighbours z > w of u, v and w.
__device__ __forceinline__ uint64_t k4_of_list(const DevGraph& g, int32_t base, const uint32_t* cw,
                                               const int16_t* list, int count) {
  const int lane = threadIdx.x & 31;
  const int32_t bw = g.bwords;
  uint64_t k4 = 0;
  for (int i = lane; i < count; i += 32) {
    const int32_t wl = list[i];
    const uint32_t* Bw = brow(g.bits2, bw, base + wl);
    for (int32_t x = wl >> 5; x < bw; ++x) k4 += __popc(cw[x] & __ldg(Bw + x) & above(x, wl));
  }
  return k4;
}

// Per-pair sums (d(u)-1)(d(v)-1), t(e), C(t(e), 2) and the 4-cliques, added
// to slots 1, 2, 4 and 5 of the pair's graph. Lane 0 of a warp keeps them in
// registers while its pairs stay in one graph; at the end of the kernel the
// block merges its warps' runs, so that each block issues one atomic per slot
// and graph instead of one per pair (thousands of same-address atomics
// otherwise serialise in L2).
struct PairSums {
  int32_t gi = -1;
  uint64_t v[4] = {0, 0, 0, 0};
};

__device__ __forceinline__ void pair_sums_flush(unsigned long long* agg, const PairSums& P) {
  if (P.gi < 0) return;
  unsigned long long* A = agg + (int64_t)P.gi * NAGG;
  if (P.v[0]) atomicAdd(&A[1], (unsigned long long)P.v[0]);
  if (P.v[1]) atomicAdd(&A[2], (unsigned long long)P.v[1]);
  if (P.v[2]) atomicAdd(&A[4], (unsigned long long)P.v[2]);
  if (P.v[3]) atomicAdd(&A[5], (unsigned long long)P.v[3]);
}

__device__ __forceinline__ void pair_sums_add(PairSums& P, unsigned long long* agg, int32_t gi,
                                              uint64_t du, uint64_t dv, uint64_t t, uint64_t k4) {
  if (gi != P.gi) {
    pair_sums_flush(agg, P);
    P = PairSums{};
    P.gi = gi;
  }
  P.v[0] += (du - 1) * (dv - 1);
  P.v[1] += t;
  P.v[2] += t * (t - (t > 0 ? 1 : 0)) / 2;
  P.v[3] += k4;
}

// Called by every thread of the block after the pair loop; the leader of each
// of the block's NG lane groups holds the group's run.
template <int NG>
__device__ __forceinline__ void pair_sums_groups(const PairSums& P, int grp, bool leader,
                                                 unsigned long long* agg) {
  __shared__ int32_t gi_s[NG];
  __shared__ uint64_t v_s[NG][4];
  if (leader) {
    gi_s[grp] = P.gi;
#pragma unroll
    for (int i = 0; i < 4; ++i) v_s[grp][i] = P.v[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    PairSums R;
    for (int w = 0; w < NG; ++w) {
      if (gi_s[w] < 0) continue;
      if (gi_s[w] != R.gi) {
        pair_sums_flush(agg, R);
        R = PairSums{};
        R.gi = gi_s[w];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) R.v[i] += v_s[w][i];
    }
    pair_sums_flush(agg, R);
  }
}

// The same with one group per warp (blockDim.x = 32 * NW), lane 0 leading.
template <int NW>
__device__ __forceinline__ void pair_sums_block(const PairSums& P, unsigned long long* agg) {
  pair_sums_groups<NW>(P, threadIdx.x >> 5, (threadIdx.x & 31) == 0, agg);
}

// Rows of at most 16 words: one half-warp per pair, lanes over words. t(e)
// is the popcount of the rows' AND; the common neighbours w > v (at most
// 16 x 32) are listed in shared memory and shared out over the 16 lanes for
// the 4-cliques, as in k_graphlet_edges, with half the lanes of a warp per
// pair.
constexpr int GLH_LIST = 16 * 32;
__global__ void __launch_bounds__(GL_WARPS * 32, 4)
    k_graphlet_edges16(const DevGraph g, uint32_t* __restrict__ tnode,
                       unsigned long long* __restrict__ agg) {
  __shared__ uint32_t cw_s[GL_WARPS * 2][16];
  __shared__ int16_t wl_s[GL_WARPS * 2][GLH_LIST];
  const int32_t bw = g.bwords;
  const int lane = threadIdx.x & 31, sub = lane >> 4, sl = lane & 15;
  const int grp = (threadIdx.x >> 5) * 2 + sub;
  const unsigned mask = 0xFFFFu << (sub * 16);
  uint32_t* cw = cw_s[grp];
  int16_t* list = wl_s[grp];
  const int64_t groups = ((int64_t)gridDim.x * blockDim.x) >> 4;
  PairSums P;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4; p < g.m2; p += groups) {
    const int32_t u = (int32_t)(g.e2[p] >> 32), v = (int32_t)(g.e2[p] & 0xFFFFFFFFull);
    const int32_t base = graph_base(g, u), vl = v - base;
    uint32_t c = 0;
    if (sl < bw) {
      c = __ldg(brow(g.bits2, bw, u) + sl) & __ldg(brow(g.bits2, bw, v) + sl);
      cw[sl] = c;
    }
    uint32_t t = __popc(c);
    uint32_t word = sl < bw ? (c & above(sl, vl)) : 0u;
    const uint32_t cc = __popc(word);
    uint32_t incl = cc;
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
      const uint32_t y = __shfl_up_sync(mask, incl, d, 16);
      if (sl >= d) incl += y;
    }
    int pos = (int)(incl - cc);
    while (word) {
      const int j = __ffs(word) - 1;
      word &= word - 1;
      list[pos++] = (int16_t)(sl * 32 + j);
    }
    const int count = (int)__shfl_sync(mask, incl, 15, 16);
    __syncwarp(mask);
    uint64_t k4 = 0;
    for (int i = sl; i < count; i += 16) {
      const int32_t wl = list[i];
      const uint32_t* Bw = brow(g.bits2, bw, base + wl);
      for (int32_t x = wl >> 5; x < bw; ++x) k4 += __popc(cw[x] & __ldg(Bw + x) & above(x, wl));
    }
#pragma unroll
    for (int o = 8; o; o >>= 1) {
      t += __shfl_xor_sync(mask, t, o, 16);
      k4 += __shfl_xor_sync(mask, k4, o, 16);
    }
    if (sl == 0) {
      atomicAdd(&tnode[u], t);
      atomicAdd(&tnode[v], t);
      pair_sums_add(P, agg, graph_of(g, u), (uint64_t)degree(g, u), (uint64_t)degree(g, v), t, k4);
    }
    __syncwarp(mask);
  }
  pair_sums_groups<GL_WARPS * 2>(P, grp, sl == 0, agg);
}

// One warp per pair (u < v): t(e) = popcount of the rows' AND (lanes over
// words, kept in shared memory), the 4-cliques whose two smallest nodes are
// u < v (common neighbours w > v listed in shared memory and shared out over
// the lanes), then the per-pair sums and t(e) added at both ends. Rows longer
// than GL_MAXW words take the lanes over words directly.
__global__ void __launch_bounds__(GL_WARPS * 32, 4)
    k_graphlet_edges(const DevGraph g, uint32_t* __restrict__ tnode,
                     unsigned long long* __restrict__ agg) {
  __shared__ uint32_t cw_s[GL_WARPS][GL_MAXW];
  __shared__ int16_t wl_s[GL_WARPS][GL_LIST];
  const int32_t bw = g.bwords;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* cw = cw_s[wid];
  int16_t* list = wl_s[wid];
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  PairSums P;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < g.m2; p += warps) {
    const int32_t u = (int32_t)(g.e2[p] >> 32), v = (int32_t)(g.e2[p] & 0xFFFFFFFFull);
    const int32_t base = graph_base(g, u), vl = v - base;
    const uint32_t* Bu = brow(g.bits2, bw, u);
    const uint32_t* Bv = brow(g.bits2, bw, v);
    uint32_t t = 0;
    uint64_t k4 = 0;
    if (bw <= GL_MAXW) {
      for (int32_t w = lane; w < bw; w += 32) {
        const uint32_t c = __ldg(Bu + w) & __ldg(Bv + w);
        cw[w] = c;
        t += __popc(c);
      }
      __syncwarp();
      int count = 0;
      for (int32_t w0 = 0; w0 < bw; w0 += 32) {
        const int32_t w = w0 + lane;
        uint32_t word = w < bw ? (cw[w] & above(w, vl)) : 0u;
        const uint32_t c = __popc(word);
        uint32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += y;
        }
        const int round = (int)__shfl_sync(0xffffffffu, incl, 31);
        if (count + round > GL_LIST) {  // list full: count its cliques first
          k4 += k4_of_list(g, base, cw, list, count);
          __syncwarp();
          count = 0;
        }
        int pos = count + (int)(incl - c);
        while (word) {
          const int j = __ffs(word) - 1;
          word &= word - 1;
          list[pos++] = (int16_t)(w * 32 + j);
        }
        count += round;
        __syncwarp();
      }
      k4 += k4_of_list(g, base, cw, list, count);
      __syncwarp();
    } else {
      for (int32_t w = lane; w < bw; w += 32) {
        const uint32_t c = __ldg(Bu + w) & __ldg(Bv + w);
        t += __popc(c);
        uint32_t ws = c & above(w, vl);
        while (ws) {
          const int j = __ffs(ws) - 1;
          ws &= ws - 1;
          const int32_t wl = w * 32 + j;
          const uint32_t* Bw = brow(g.bits2, bw, base + wl);
          for (int32_t x = w; x < bw; ++x)
            k4 += __popc(__ldg(Bu + x) & __ldg(Bv + x) & __ldg(Bw + x) & above(x, wl));
        }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      t += __shfl_xor_sync(0xffffffffu, t, o);
      k4 += __shfl_xor_sync(0xffffffffu, k4, o);
    }
    if (lane == 0) {
      atomicAdd(&tnode[u], t);
      atomicAdd(&tnode[v], t);
      pair_sums_add(P, agg, graph_of(g, u), (uint64_t)degree(g, u), (uint64_t)degree(g, v), t, k4);
    }
  }
  pair_sums_block<GL_WARPS>(P, agg);
}

// Node pairs x < z of one graph: one warp per row x (grid-stride), lanes over
// the z > x of x's graph; C(c(x, z), 2) summed per warp.
__global__ void k_graphlet_pairs(const DevGraph g, int32_t nodes_per_graph,
                                 unsigned long long* __restrict__ agg) {
  const int32_t bw = g.bwords;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < g.n; x += warps) {
    const int64_t gi = x / nodes_per_graph;
    const int64_t end = min((int64_t)g.n, (gi + 1) * nodes_per_graph);
    const uint32_t* Bx = brow(g.bits2, bw, (int32_t)x);
    uint64_t acc = 0;
    for (int64_t z = x + 1 + lane; z < end; z += 32) {
      const uint32_t* Bz = brow(g.bits2, bw, (int32_t)z);
      uint64_t c = 0;
      for (int32_t w4 = 0; w4 < bw; w4 += 4) {
        uint32_t a4[4], b4[4];
        ld4(Bx + w4, a4);
        ld4(Bz + w4, b4);
        c += __popc(a4[0] & b4[0]) + __popc(a4[1] & b4[1]) + __popc(a4[2] & b4[2]) +
             __popc(a4[3] & b4[3]);
      }
      acc += c * (c - (c > 0 ? 1 : 0)) / 2;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc) atomicAdd(&agg[gi * NAGG + 6], (unsigned long long)acc);
  }
}

// Graphs without pair bitmaps: the pair sums from the triangles and 4-cliques,
// each found once at its lowest-ranked node u (rank = (degree, id), as in the
// 4-cycle pass) among u's neighbours of higher rank, out(u): a triangle is a
// pair of out(u) that is itself a pair, a 4-clique a triple of out(u) whose
// three pairs are pairs. Ranked this way out(u) is short (at most
// sqrt(2 m2)), so this probes far fewer pairs than intersecting the two
// neighbour lists of every pair. A triangle adds 1 to t(e) of its three
// pairs (a counter per slot of the pair hash set, tslot) and 2 to tnode of
// its three nodes; every pair (u, v), v in out(u), adds (d(u) - 1)(d(v) - 1)
// once; k_graphlet_tslots then sums C(t(e), 2) over the slots.
//   d(u) <= GLT_SMALL: a lane per node, out(u) in shared memory, and the
//   pairs of the warp's 32 nodes spread over its lanes;
//   larger: the whole warp per node, out(u) in the warp's global list
//   (capacity = the largest degree); 4-cliques from adjacency rows of out(u)
//   in shared memory when |out(u)| <= GLT_ROWS, else by probing each
//   triangle's later members of out(u).
// rank order of the sparse passes: (degree, id)
__device__ __forceinline__ bool lower_rank(int32_t dz, int32_t z, int32_t dx, int32_t x) {
  return dz < dx || (dz == dx && z < x);
}

constexpr int GLT_SMALL = 8;
constexpr int GLT_ROWS = 128;
constexpr int GLT_WORDS = GLT_ROWS / 32;

__device__ __forceinline__ int64_t pair_slot(const DevGraph& g, int32_t a, int32_t b) {
  const uint64_t key = pair_key(a, b);
  uint64_t slot = hash_pair(key) & g.h2_mask;
  for (uint64_t it = 0; it <= g.h2_mask; ++it) {
    const uint64_t v = __ldg(g.h2 + slot);
    if (v == key) return (int64_t)slot;
    if (v == EMPTY64) return -1;
    slot = (slot + 1) & g.h2_mask;
  }
  return -1;
}

__device__ __forceinline__ void pair_sums_put(PairSums& P, unsigned long long* agg, int32_t gi,
                                              int i, uint64_t x) {
  if (gi != P.gi) {
    pair_sums_flush(agg, P);
    P = PairSums{};
    P.gi = gi;
  }
  P.v[i] += x;
}

// Triangle {u, v, w} found at u; s_vw is the slot of the pair (v, w).
__device__ __forceinline__ void triangle_at(const DevGraph& g, uint32_t* tslot, uint32_t* tnode,
                                            int32_t u, int32_t v, int32_t w, int64_t s_vw) {
  atomicAdd(&tslot[s_vw], 1u);
  const int64_t s_uv = pair_slot(g, u, v), s_uw = pair_slot(g, u, w);
  if (s_uv >= 0) atomicAdd(&tslot[s_uv], 1u);
  if (s_uw >= 0) atomicAdd(&tslot[s_uw], 1u);
  atomicAdd(&tnode[u], 2u);
  atomicAdd(&tnode[v], 2u);
  atomicAdd(&tnode[w], 2u);
}

__global__ void __launch_bounds__(SPARSE_WARPS * 32)
    k_graphlet_tri(const DevGraph g, int32_t* __restrict__ lists, int64_t cap,
                   uint32_t* __restrict__ tslot, uint32_t* __restrict__ tnode,
                   unsigned long long* __restrict__ agg) {
  __shared__ int32_t out_s[SPARSE_WARPS][32][GLT_SMALL];
  __shared__ uint32_t adj_s[SPARSE_WARPS][32][GLT_SMALL];
  __shared__ uint32_t pre_s[SPARSE_WARPS][32];
  __shared__ uint32_t row_s[SPARSE_WARPS][GLT_ROWS][GLT_WORDS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* list = lists + gw * cap;
  int32_t(*outl)[GLT_SMALL] = out_s[wid];
  uint32_t(*adjm)[GLT_SMALL] = adj_s[wid];
  uint32_t* pre = pre_s[wid];
  uint32_t(*row)[GLT_WORDS] = row_s[wid];
  PairSums P;
  for (int64_t c0 = gw * 32; c0 < g.n; c0 += warps * 32) {
    const int64_t ul = c0 + lane;
    const int32_t u = (int32_t)ul;
    int32_t du = 0;
    int64_t ou = 0;
    if (ul < g.n) {
      ou = g.off2[u];
      du = (int32_t)(g.off2[u + 1] - ou);
    }
    const bool small = du <= GLT_SMALL;
    int k = 0;
    if (small) {
      const int32_t gu = du ? graph_of(g, u) : 0;
      for (int i = 0; i < du; ++i) {
        const int32_t y = g.adj2[ou + i];
        const int32_t dy = degree(g, y);
        if (lower_rank(du, u, dy, y)) {
          pair_sums_put(P, agg, gu, 0, (uint64_t)(du - 1) * (uint64_t)(dy - 1));
          outl[lane][k] = y;
          adjm[lane][k] = 0u;
          ++k;
        }
      }
    }
    // the pairs of the small nodes' out-lists, spread over the lanes
    const uint32_t np = (uint32_t)(k * (k - 1) / 2);
    uint32_t incl = np;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    pre[lane] = incl - np;
    const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    for (uint32_t p = lane; p < tot; p += 32) {
      int lo = 0, hi = 32;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= p) lo = mid;
        else hi = mid;
      }
      uint32_t i, j;
      fam::unrank2(p - pre[lo], i, j);
      const int32_t v = outl[lo][i], w = outl[lo][j];
      const int64_t s_vw = pair_slot(g, v, w);
      if (s_vw < 0) continue;
      const int32_t uo = (int32_t)(c0 + lo);
      triangle_at(g, tslot, tnode, uo, v, w, s_vw);
      pair_sums_put(P, agg, graph_of(g, uo), 1, 3);
      atomicOr(&adjm[lo][i], 1u << j);
      atomicOr(&adjm[lo][j], 1u << i);
    }
    __syncwarp();
    if (k >= 3) {  // 4-cliques at a small node: i < j < l, all three pairs present
      uint64_t k4 = 0;
      for (int i = 0; i < k; ++i) {
        uint32_t mi = adjm[lane][i] & ~((2u << i) - 1u);
        while (mi) {
          const int j = __ffs(mi) - 1;
          mi &= mi - 1;
          k4 += __popc(adjm[lane][i] & adjm[lane][j] & ~((2u << j) - 1u));
        }
      }
      if (k4) pair_sums_put(P, agg, graph_of(g, u), 3, k4);
    }
    __syncwarp();
    // the other nodes, one at a time with the whole warp
    unsigned bigs = __ballot_sync(0xffffffffu, !small);
    while (bigs) {
      const int src = __ffs(bigs) - 1;
      bigs &= bigs - 1;
      const int32_t x = (int32_t)(c0 + src);
      const int32_t dx = __shfl_sync(0xffffffffu, du, src);
      const int64_t ox = __shfl_sync(0xffffffffu, ou, src);
      const int32_t gx = graph_of(g, x);
      int kx = 0;
      for (int32_t i0 = 0; i0 < dx; i0 += 32) {
        const int32_t i = i0 + lane;
        int32_t y = 0;
        bool higher = false;
        if (i < dx) {
          y = g.adj2[ox + i];
          const int32_t dy = degree(g, y);
          higher = lower_rank(dx, x, dy, y);
          if (higher) pair_sums_put(P, agg, gx, 0, (uint64_t)(dx - 1) * (uint64_t)(dy - 1));
        }
        const unsigned b = __ballot_sync(0xffffffffu, higher);
        if (higher) list[kx + __popc(b & lt)] = y;
        kx += __popc(b);
      }
      const bool rows = kx <= GLT_ROWS;
      if (rows)
        for (int r = lane; r < kx * GLT_WORDS; r += 32) row[r / GLT_WORDS][r % GLT_WORDS] = 0u;
      __syncwarp();
      const uint64_t npx = (uint64_t)kx * (uint64_t)(kx - 1) / 2;
      for (uint64_t p = lane; p < npx; p += 32) {
        uint32_t i, j;
        fam::unrank2(p, i, j);
        const int32_t v = list[i], w = list[j];
        const int64_t s_vw = pair_slot(g, v, w);
        if (s_vw < 0) continue;
        triangle_at(g, tslot, tnode, x, v, w, s_vw);
        pair_sums_put(P, agg, gx, 1, 3);
        if (rows) {
          atomicOr(&row[i][j >> 5], 1u << (j & 31));
          atomicOr(&row[j][i >> 5], 1u << (i & 31));
        } else {
          uint64_t k4 = 0;
          for (int l = (int)j + 1; l < kx; ++l) {
            const int32_t z = list[l];
            if (has_pair(g, v, z) && has_pair(g, w, z)) ++k4;
          }
          if (k4) pair_sums_put(P, agg, gx, 3, k4);
        }
      }
      __syncwarp();
      if (rows && kx >= 3) {
        uint64_t k4 = 0;
        for (uint64_t p = lane; p < npx; p += 32) {
          uint32_t i, j;
          fam::unrank2(p, i, j);
          if (!((row[i][j >> 5] >> (j & 31)) & 1u)) continue;
          for (uint32_t wd = j >> 5; wd < GLT_WORDS; ++wd) {
            uint32_t m = row[i][wd] & row[j][wd];
            if (wd == (j >> 5)) m &= ~((2u << (j & 31)) - 1u);
            k4 += __popc(m);
          }
        }
        if (k4) pair_sums_put(P, agg, gx, 3, k4);
      }
      __syncwarp();
    }
  }
  pair_sums_groups<SPARSE_WARPS * 32>(P, threadIdx.x, true, agg);
}

// C(t(e), 2) over the slots of the pair hash set, into the pair's graph.
__global__ void k_graphlet_tslots(const DevGraph g, const uint32_t* __restrict__ tslot,
                                  unsigned long long* __restrict__ agg) {
  PairSums P;
  const uint64_t slots = g.h2_mask + 1;
  for (uint64_t sl = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; sl < slots;
       sl += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t t = tslot[sl];
    if (t < 2) continue;
    const int32_t a = (int32_t)(__ldg(g.h2 + sl) >> 32);
    pair_sums_put(P, agg, graph_of(g, a), 2, t * (t - 1) / 2);
  }
  pair_sums_flush(agg, P);
}

// 4-cycles of graphs without pair bitmaps, each at its highest-ranked node x
// (rank = (degree, id)): the nodes z of lower rank reached by paths x - y - z
// through a y of lower rank are counted, and every two such paths to one z
// close a 4-cycle x - y - z - y'. Each pass adds 2 C4 to the graph's sum, as
// the bitmap kernel does. The paths from x number at most ub(x) = the sum of
// d(y) over its lower-ranked neighbours y, and the work sits in few nodes (on
// a communication-shaped graph 1 % of the nodes hold 84 % of 2.2e8 paths, the
// largest 3.6e5), so:
//   ub <= warp bound: one warp per node counts in a shared-memory hash;
//   above: the node owns ub slots of one path space (a prefix sum of the
//   bounds, computed at build time) and a table of 2 ub slots in global
//   memory; blocks take equal pieces of the path space and insert their
//   paths' endpoints into the owners' tables, then one pass adds C(c, 2)
//   over the tables. (HM_C4_SORT=1 instead writes each path as a key
//   (x << bits) | z into its slot, unused slots a sentinel, sorts the keys
//   and adds C(c, 2) per run of c equal keys.)
constexpr int C4_WARPS = 4;
constexpr int C4_WARP_SLOTS = 512;
constexpr uint32_t C4_WARP_UB = C4_WARP_SLOTS / 2;
constexpr uint64_t C4_SENTINEL = ~0ull;

// HM_C4_SORT=1 counts the heavy nodes' 4-cycles by sorting their path keys
// instead of per-node tables (the tests cover both tiers).
bool c4_sort_tier() {
  const char* e = std::getenv("HM_C4_SORT");
  return e && e[0] == '1';
}

// The warp tier's bound: C4_WARP_UB, or lower by HM_C4_UB (tests send small
// graphs' nodes to the heavy tier with it).
uint32_t c4_warp_bound() {
  uint32_t w = C4_WARP_UB;
  if (const char* e = std::getenv("HM_C4_UB")) {
    unsigned a = 0;
    if (std::sscanf(e, "%u", &a) == 1) w = std::min<uint32_t>(a, C4_WARP_UB);
  }
  return w;
}


// Counts z in a table of 2^lg slots (keys -1 = empty). Every table holds
// fewer distinct keys than slots, so a probe always ends; the bound on the
// loop only makes that visible.
__device__ __forceinline__ void c4_insert(int32_t* keys, uint32_t* cnt, int lg, int32_t z) {
  const uint32_t mask = (1u << lg) - 1u;
  uint32_t sl = ((uint32_t)z * 0x9E3779B1u) >> (32 - lg);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int32_t k = atomicCAS(&keys[sl], -1, z);
    if (k == -1 || k == z) {
      atomicAdd(&cnt[sl], 1u);
      return;
    }
    sl = (sl + 1) & mask;
  }
}

__device__ __forceinline__ int c4_lg(uint32_t ub) {
  int lg = 5;
  while ((1u << lg) < 2 * ub) ++lg;
  return lg;
}

// Running sum of one thread for graph gcur; one atomic per graph change.
struct C4Sum {
  int64_t gcur = -1;
  uint64_t s = 0;
  __device__ void add(unsigned long long* agg, int64_t gi, uint64_t v) {
    if (gi != gcur) {
      flush(agg);
      gcur = gi;
      s = 0;
    }
    s += v;
  }
  __device__ void flush(unsigned long long* agg) {
    if (gcur >= 0 && s) atomicAdd(&agg[gcur * NAGG + 6], (unsigned long long)(2 * s));
  }
};

// End of a kernel: every thread's C4Sum into agg with one atomic per block and
// graph run. A warp whose lanes all hold one graph (or nothing) is summed by
// shuffles; the warps' sums meet in shared memory and thread 0 adds runs of
// one graph. A warp that straddles graphs flushes lane by lane. All threads
// of the block (NW warps) call it.
template <int NW>
__device__ __forceinline__ void c4_flush_block(C4Sum& acc, unsigned long long* agg) {
  __shared__ int64_t g_s[NW];
  __shared__ unsigned long long v_s[NW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool has = acc.gcur >= 0 && acc.s != 0;
  const unsigned any = __ballot_sync(0xffffffffu, has);
  const int64_t gref = any ? __shfl_sync(0xffffffffu, acc.gcur, __ffs(any) - 1) : -1;
  if (__all_sync(0xffffffffu, !has || acc.gcur == gref)) {
    unsigned long long v = has ? acc.s : 0ull;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
      g_s[wid] = gref;
      v_s[wid] = v;
    }
  } else {
    acc.flush(agg);
    if (lane == 0) g_s[wid] = -1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t gc = -1;
    unsigned long long sum = 0;
    for (int w = 0; w < NW; ++w) {
      if (g_s[w] < 0 || v_s[w] == 0) continue;
      if (g_s[w] != gc) {
        if (gc >= 0 && sum) atomicAdd(&agg[gc * NAGG + 6], 2 * sum);
        gc = g_s[w];
        sum = 0;
      }
      sum += v_s[w];
    }
    if (gc >= 0 && sum) atomicAdd(&agg[gc * NAGG + 6], 2 * sum);
  }
}

// Path bound of x over its lower-ranked neighbours, summed over the warp
// (every lane gets it).
__device__ __forceinline__ uint64_t c4_bound(const DevGraph& g, int32_t x, int64_t ox, int32_t dx) {
  const int lane = threadIdx.x & 31;
  uint64_t ub = 0;
  for (int32_t i = lane; i < dx; i += 32) {
    const int32_t y = g.adj2[ox + i];
    const int32_t dy = degree(g, y);
    if (lower_rank(dy, y, dx, x)) ub += (uint64_t)dy;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) ub += __shfl_xor_sync(0xffffffffu, ub, o);
  return ub;
}

// Per node: its bound when above the warp tier's bound (its slots of the
// heavy tier), else 0; and into light, its bound when in [2, warp_ub], else
// 0. One warp per node.
__global__ void k_c4_bound(const DevGraph g, uint32_t warp_ub, uint64_t* __restrict__ out,
                           uint16_t* __restrict__ light) {
  // a warp takes 32 consecutive nodes: those of degree <= 8 a lane each, the
  // others in turn with the whole warp
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c0 = gw * 32; c0 < g.n; c0 += warps * 32) {
    const int64_t xl = c0 + lane;
    int64_t ox = 0;
    int32_t dx = 0;
    if (xl < g.n) {
      ox = g.off2[xl];
      dx = (int32_t)(g.off2[xl + 1] - ox);
    }
    const bool small = dx <= 8;
    if (small && xl < g.n) {
      const int32_t x = (int32_t)xl;
      uint64_t ub = 0;
      for (int32_t i = 0; i < dx; ++i) {
        const int32_t y = g.adj2[ox + i];
        const int32_t dy = degree(g, y);
        if (lower_rank(dy, y, dx, x)) ub += (uint64_t)dy;
      }
      out[x] = ub > warp_ub ? ub : 0;
      light[x] = (ub >= 2 && ub <= warp_ub) ? (uint16_t)ub : (uint16_t)0;
    }
    unsigned bigs = __ballot_sync(0xffffffffu, !small);
    while (bigs) {
      const int src = __ffs(bigs) - 1;
      bigs &= bigs - 1;
      const int32_t x = (int32_t)(c0 + src);
      const uint64_t ub = c4_bound(g, x, __shfl_sync(0xffffffffu, ox, src),
                                   __shfl_sync(0xffffffffu, dx, src));
      if (lane == 0) {
        out[x] = ub > warp_ub ? ub : 0;
        light[x] = (ub >= 2 && ub <= warp_ub) ? (uint16_t)ub : (uint16_t)0;
      }
    }
  }
}

// Warp tier: the nodes with a bound ub in [2, warp_ub] (light[x] = ub, else
// 0), one warp per node. A warp reads the bounds of 32 consecutive nodes and
// takes its active ones in turn. It stages x's lower-ranked neighbours y (at
// most ub of them, each with d(y) >= 1) with the exclusive prefix of their
// degrees, then its lanes take the ub paths in turn (lane l the paths l,
// l + 32, ...), each finding its y by binary search in the prefix, so that a
// lane's work is ub / 32 paths whatever the degrees.
__global__ void __launch_bounds__(C4_WARPS * 32)
    k_c4_warp(const DevGraph g, const uint16_t* __restrict__ light, int32_t nodes_per_graph,
              unsigned long long* __restrict__ agg) {
  __shared__ int32_t keys_s[C4_WARPS][C4_WARP_SLOTS];
  __shared__ uint32_t cnt_s[C4_WARPS][C4_WARP_SLOTS];
  __shared__ int64_t off_s[C4_WARPS][C4_WARP_UB];
  __shared__ uint32_t pre_s[C4_WARPS][C4_WARP_UB];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* keys = keys_s[wid];
  uint32_t* cnt = cnt_s[wid];
  int64_t* soff = off_s[wid];
  uint32_t* spre = pre_s[wid];
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  C4Sum acc;
  for (int64_t c0 = gw * 32; c0 < g.n; c0 += warps * 32) {
   const uint32_t mine = c0 + lane < g.n ? light[c0 + lane] : 0u;
   unsigned act = __ballot_sync(0xffffffffu, mine != 0);
   while (act) {
    const int src = __ffs(act) - 1;
    act &= act - 1;
    const int32_t x = (int32_t)(c0 + src);
    const uint32_t ub = __shfl_sync(0xffffffffu, mine, src);
    const int64_t ox = g.off2[x];
    const int32_t dx = (int32_t)(g.off2[x + 1] - ox);
    const int lg = c4_lg(ub);
    for (int i = lane; i < (1 << lg); i += 32) {
      keys[i] = -1;
      cnt[i] = 0;
    }
    uint32_t m = 0, run = 0;  // staged neighbours, their degree sum (warp-uniform)
    for (int32_t i0 = 0; i0 < dx; i0 += 32) {
      const int32_t i = i0 + lane;
      uint32_t v = 0;
      int64_t oy = 0;
      if (i < dx) {
        const int32_t y = g.adj2[ox + i];
        oy = g.off2[y];
        const int32_t dy = (int32_t)(g.off2[y + 1] - oy);
        if (lower_rank(dy, y, dx, x)) v = (uint32_t)dy;
      }
      const unsigned b = __ballot_sync(0xffffffffu, v != 0);
      uint32_t incl = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += u;
      }
      if (v) {
        const uint32_t at = m + __popc(b & ((1u << lane) - 1u));
        soff[at] = oy;
        spre[at] = run + incl - v;
      }
      m += __popc(b);
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    for (uint32_t sl = lane; sl < run; sl += 32) {
      uint32_t lo = 0, hi = m;
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (spre[mid] <= sl) lo = mid;
        else hi = mid;
      }
      const int32_t z = g.adj2[soff[lo] + (sl - spre[lo])];
      if (z != x && lower_rank(degree(g, z), z, dx, x)) c4_insert(keys, cnt, lg, z);
    }
    __syncwarp();
    uint64_t sum = 0;
    for (int i = lane; i < (1 << lg); i += 32) {
      const uint64_t c = keys[i] >= 0 ? cnt[i] : 0u;
      sum += c * (c - (c > 0 ? 1 : 0)) / 2;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) acc.add(agg, x / nodes_per_graph, sum);
    __syncwarp();
   }
  }
  c4_flush_block<C4_WARPS>(acc, agg);
}

// Sort tier, emission: one block per node with slots [ws[x], ws[x+1]). The
// lower-ranked neighbours y are staged in shared memory (C4E_CAP per round)
// with an exclusive prefix of their degrees; the block's threads then walk
// the round's slots in order, each finding its y by binary search in the
// prefix, so that neighbour lists are read and keys written in consecutive
// runs. A slot holds the key of its path x - y - z when z is kept, else the
// sentinel. The slots of a round sum the same degrees as c4_bound, so the
// node's slots are exactly [ws[x], ws[x+1]).
constexpr int C4E_THREADS = 512;
constexpr int C4E_CAP = 1024;  // neighbours per round (2 per thread)

__global__ void __launch_bounds__(C4E_THREADS)
    k_c4_emit(const DevGraph g, int bits, const uint64_t* __restrict__ ws,
              uint64_t* __restrict__ keys) {
  __shared__ int64_t s_off[C4E_CAP];
  __shared__ uint32_t s_pre[C4E_CAP];
  __shared__ uint32_t s_wsum[C4E_THREADS / 32];
  __shared__ int32_t s_heavy[C4E_THREADS];
  __shared__ int s_nheavy;
  __shared__ uint32_t s_total;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t c0 = (int64_t)blockIdx.x * C4E_THREADS; c0 < g.n;
       c0 += (int64_t)gridDim.x * C4E_THREADS) {
    if (threadIdx.x == 0) s_nheavy = 0;
    __syncthreads();
    const int64_t xi = c0 + threadIdx.x;
    if (xi < g.n && ws[xi + 1] != ws[xi]) s_heavy[atomicAdd(&s_nheavy, 1)] = (int32_t)xi;
    __syncthreads();
    const int nh = s_nheavy;
    for (int hh = 0; hh < nh; ++hh) {
      const int32_t x = s_heavy[hh];
      const int64_t ox = g.off2[x];
      const int32_t dx = (int32_t)(g.off2[x + 1] - ox);
      uint64_t base = ws[x];
      const uint64_t hi = (uint64_t)x << bits;
      for (int32_t r0 = 0; r0 < dx; r0 += C4E_CAP) {
        const int32_t cnt = min(C4E_CAP, dx - r0);
        uint32_t v[2];
        int64_t o[2];
        uint32_t tsum = 0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int32_t j = threadIdx.x * 2 + q;
          v[q] = 0;
          o[q] = 0;
          if (j < cnt) {
            const int32_t y = g.adj2[ox + r0 + j];
            const int64_t oy = g.off2[y];
            const int32_t dy = (int32_t)(g.off2[y + 1] - oy);
            if (lower_rank(dy, y, dx, x)) {
              v[q] = (uint32_t)dy;
              o[q] = oy;
            }
          }
          tsum += v[q];
        }
        // exclusive prefix of the per-thread sums over the block
        uint32_t incl = tsum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += u;
        }
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
          uint32_t w = lane < C4E_THREADS / 32 ? s_wsum[lane] : 0u;
          uint32_t wi = w;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += u;
          }
          if (lane < C4E_THREADS / 32) s_wsum[lane] = wi - w;
          if (lane == 31) s_total = wi;
        }
        __syncthreads();
        uint32_t ex = s_wsum[wid] + incl - tsum;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int32_t j = threadIdx.x * 2 + q;
          if (j < cnt) {
            s_pre[j] = ex;
            s_off[j] = o[q];
          }
          ex += v[q];
        }
        __syncthreads();
        const uint32_t total = s_total;
        for (uint32_t sl = threadIdx.x; sl < total; sl += C4E_THREADS) {
          // the last staged neighbour whose range starts at or before sl (a
          // neighbour without slots shares its start with the next one)
          int lo = 0, hi2 = cnt;
          while (hi2 - lo > 1) {
            const int mid = (lo + hi2) >> 1;
            if (s_pre[mid] <= sl) lo = mid;
            else hi2 = mid;
          }
          const int32_t z = g.adj2[s_off[lo] + (sl - s_pre[lo])];
          const bool keep = z != x && lower_rank(degree(g, z), z, dx, x);
          keys[base + sl] = keep ? (hi | (uint64_t)(uint32_t)z) : C4_SENTINEL;
        }
        base += total;
        __syncthreads();  // the next round overwrites the staged neighbours
      }
    }
  }
}

// Table tier (the default for heavy nodes). Node x's paths own the slots
// [ws[x], ws[x+1]) of one path space, which is cut into pieces of C4T_PIECE
// consecutive slots, one block per piece, so that a node with many paths is
// spread over many blocks and every block has the same work. For each node
// its piece overlaps, the block stages x's lower-ranked neighbours (rounds of
// C4E_CAP, degree prefix as in k_c4_emit), walks the overlapped slots and
// puts each kept endpoint z into x's open-addressing table of 2 (ws[x+1] -
// ws[x]) slots at [2 ws[x], 2 ws[x+1]) (slot = (z << 32) | count, empty = all
// ones; a match adds 1 to the count word, which never carries into z). A
// table holds at most ws[x+1] - ws[x] keys in twice as many slots, so every
// probe ends. The 4-cycle sum Σ_z C(count_z, 2) is taken on the way: a match
// adds the count it found (the pairs its path closes with the earlier paths
// to z), so no pass over the tables follows.
constexpr uint32_t C4T_PIECE = 4096;

// The node x with ws[x] <= pos < ws[x + 1] (ws is nondecreasing, ws[0] = 0 <=
// pos < ws[n]), by a 32-way search of one warp; every lane returns it.
__device__ __forceinline__ int64_t c4_owner(const uint64_t* __restrict__ ws, int64_t n,
                                            uint64_t pos) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = n;  // ws[lo] <= pos < ws[hi]
  while (hi - lo > 1) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t idx = min(lo + lane * step, hi);
    const unsigned ok = __ballot_sync(0xffffffffu, ws[idx] <= pos);  // lane 0 always
    const int l = 31 - __clz(ok);
    const int64_t nlo = lo + l * step;
    hi = min(nlo + step, hi);
    lo = nlo;
  }
  return lo;
}

__global__ void __launch_bounds__(C4E_THREADS)
    k_c4_table(const DevGraph g, const uint64_t* __restrict__ ws, uint64_t total,
               unsigned long long* __restrict__ table, int32_t nodes_per_graph,
               unsigned long long* __restrict__ agg) {
  C4Sum acc;  // each repeat of an endpoint z adds its count so far: Σ_z C(count_z, 2)
  __shared__ int64_t s_off[C4E_CAP];
  __shared__ uint32_t s_pre[C4E_CAP];
  __shared__ uint32_t s_wsum[C4E_THREADS / 32];
  __shared__ uint32_t s_total;
  __shared__ int64_t s_x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint64_t p0 = (uint64_t)blockIdx.x * C4T_PIECE; p0 < total;
       p0 += (uint64_t)gridDim.x * C4T_PIECE) {
    const uint64_t p1 = min(p0 + (uint64_t)C4T_PIECE, total);
    uint64_t pos = p0;
    while (pos < p1) {
      if (wid == 0) {
        const int64_t xo = c4_owner(ws, g.n, pos);
        if (lane == 0) s_x = xo;
      }
      __syncthreads();
      const int32_t x = (int32_t)s_x;
      const uint64_t wx = ws[x], wx1 = ws[x + 1];
      const uint64_t a = pos - wx, e = min(p1, wx1) - wx;  // x's local slots [a, e)
      const int64_t ox = g.off2[x];
      const int32_t dx = (int32_t)(g.off2[x + 1] - ox);
      const uint64_t tb = 2 * wx, tcap = 2 * (wx1 - wx);
      uint64_t base = 0;  // local slot of the round's first path
      for (int32_t r0 = 0; r0 < dx && base < e; r0 += C4E_CAP) {
        const int32_t cnt = min(C4E_CAP, dx - r0);
        uint32_t v[2];
        int64_t o[2];
        uint32_t tsum = 0;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int32_t j = threadIdx.x * 2 + q;
          v[q] = 0;
          o[q] = 0;
          if (j < cnt) {
            const int32_t y = g.adj2[ox + r0 + j];
            const int64_t oy = g.off2[y];
            const int32_t dy = (int32_t)(g.off2[y + 1] - oy);
            if (lower_rank(dy, y, dx, x)) {
              v[q] = (uint32_t)dy;
              o[q] = oy;
            }
          }
          tsum += v[q];
        }
        uint32_t incl = tsum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += u;
        }
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
          uint32_t w = lane < C4E_THREADS / 32 ? s_wsum[lane] : 0u;
          uint32_t wi = w;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += u;
          }
          if (lane < C4E_THREADS / 32) s_wsum[lane] = wi - w;
          if (lane == 31) s_total = wi;
        }
        __syncthreads();
        uint32_t ex = s_wsum[wid] + incl - tsum;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int32_t j = threadIdx.x * 2 + q;
          if (j < cnt) {
            s_pre[j] = ex;
            s_off[j] = o[q];
          }
          ex += v[q];
        }
        __syncthreads();
        const uint64_t rt = s_total;
        // the round's slots [base, base + rt) cut to [a, e)
        const uint64_t lo_s = a > base ? a - base : 0;
        const uint64_t hi_s = min(e, base + rt) > base ? min(e, base + rt) - base : 0;
        for (uint64_t sl = lo_s + threadIdx.x; sl < hi_s; sl += C4E_THREADS) {
          int lo = 0, hi2 = cnt;
          while (hi2 - lo > 1) {
            const int mid = (lo + hi2) >> 1;
            if (s_pre[mid] <= (uint32_t)sl) lo = mid;
            else hi2 = mid;
          }
          const int32_t z = g.adj2[s_off[lo] + ((uint32_t)sl - s_pre[lo])];
          if (z == x || !lower_rank(degree(g, z), z, dx, x)) continue;
          const unsigned long long key = (unsigned long long)(uint32_t)z << 32;
          uint64_t slot = __umul64hi(mix64((uint64_t)(uint32_t)z), tcap);
          for (uint64_t it = 0; it < tcap; ++it) {
            unsigned long long* p = table + tb + slot;
            const unsigned long long prev = atomicCAS(p, ~0ull, key | 1ull);
            if (prev == ~0ull) break;
            if ((prev >> 32) == (uint32_t)z) {
              const unsigned long long old = atomicAdd(p, 1ull);
              acc.add(agg, (int64_t)z / nodes_per_graph, old & 0xFFFFFFFFull);
              break;
            }
            if (++slot == tcap) slot = 0;
          }
        }
        base += rt;
        __syncthreads();  // the next round overwrites the staged neighbours
      }
      pos = wx + e;
    }
  }
  c4_flush_block<C4E_THREADS / 32>(acc, agg);
}


// Sort tier, counting: each run of c equal keys (c paths from x to one z)
// closes C(c, 2) 4-cycles at x.
__global__ void k_c4_runs(const uint64_t* __restrict__ keys, uint64_t nkeys, int bits,
                          int32_t nodes_per_graph, unsigned long long* __restrict__ agg) {
  C4Sum acc;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nkeys;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    if (k == C4_SENTINEL || (i > 0 && keys[i - 1] == k)) continue;
    uint64_t c = 1;
    while (i + c < nkeys && keys[i + c] == k) ++c;
    if (c > 1) acc.add(agg, (int64_t)(k >> bits) / nodes_per_graph, c * (c - 1) / 2);
  }
  // one flush per warp when its lanes share a graph
  const int lane = threadIdx.x & 31;
  const int64_t g0 = __shfl_sync(0xffffffffu, acc.gcur, 0);
  if (__all_sync(0xffffffffu, acc.gcur == g0 || acc.gcur < 0 || acc.s == 0)) {
    uint64_t s = acc.s;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && g0 >= 0 && s) atomicAdd(&agg[g0 * NAGG + 6], (unsigned long long)(2 * s));
  } else {
    acc.flush(agg);
  }
}

struct PatternClasses {
  int cls[6];  // star, path, paw, c4, diamond, k4
};

// One block per graph: the per-node sums C(d, 3) and t(v) (d - 2), then the
// induced pattern counts into the graph's histogram row.
// Per-node sums S3 and TT of large graphs over the whole grid, into slots 0
// and 3 (one atomic pair per warp when its lanes share a graph).
__global__ void k_graphlet_nodes(const DevGraph g, int32_t nodes_per_graph,
                                 const uint32_t* __restrict__ tnode,
                                 unsigned long long* __restrict__ agg) {
  int64_t gcur = -1;
  uint64_t s3 = 0, tt = 0;
  auto flush = [&]() {
    if (gcur < 0) return;
    if (s3) atomicAdd(&agg[gcur * NAGG + 0], (unsigned long long)s3);
    if (tt) atomicAdd(&agg[gcur * NAGG + 3], (unsigned long long)tt);
  };
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gi = v / nodes_per_graph;
    if (gi != gcur) {
      flush();
      gcur = gi;
      s3 = tt = 0;
    }
    const uint64_t d = (uint64_t)degree(g, (int32_t)v), tv = tnode[v] / 2;
    if (d >= 3) s3 += choose3(d);
    if (d >= 2) tt += tv * (d - 2);
  }
  const int64_t g0 = __shfl_sync(0xffffffffu, gcur, 0);
  if (__all_sync(0xffffffffu, gcur == g0 || gcur < 0 || (s3 == 0 && tt == 0))) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      tt += __shfl_xor_sync(0xffffffffu, tt, o);
    }
    if ((threadIdx.x & 31) == 0) {
      gcur = g0;
      flush();
    }
  } else {
    flush();
  }
}

// One block per graph: the per-node sums S3 and TT (or, with `node_sums`,
// slots 0 and 3 that k_graphlet_nodes filled), then the induced counts.
__global__ void k_graphlet_finish(const DevGraph g, int32_t nodes_per_graph,
                                  const uint32_t* __restrict__ tnode,
                                  const unsigned long long* __restrict__ agg, int ncls,
                                  const PatternClasses P, int node_sums,
                                  unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long part[2][8];
  const int64_t gi = blockIdx.x;
  const int64_t v0 = gi * nodes_per_graph, v1 = min((int64_t)g.n, v0 + nodes_per_graph);
  uint64_t s3 = 0, tt = 0;
  for (int64_t v = v0 + threadIdx.x; v < v1 && !node_sums; v += blockDim.x) {
    const uint64_t d = (uint64_t)degree(g, (int32_t)v), tv = tnode[v] / 2;
    if (d >= 3) s3 += choose3(d);
    if (d >= 2) tt += tv * (d - 2);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    tt += __shfl_xor_sync(0xffffffffu, tt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    part[0][threadIdx.x >> 5] = s3;
    part[1][threadIdx.x >> 5] = tt;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const unsigned long long* A = agg + gi * NAGG;
  uint64_t S3 = 0, TT = 0;
  if (node_sums) {
    S3 = A[0];
    TT = A[3];
  } else {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      S3 += part[0][w];
      TT += part[1][w];
    }
  }
  const uint64_t T = A[2] / 3, P3 = A[1] - 3 * T, D = A[4], K4 = A[5], C4 = A[6] / 2;
  const uint64_t k4 = K4, dia = D - 6 * K4, c4 = C4 - D + 3 * K4, paw = TT - 4 * D + 12 * K4;
  const uint64_t star = S3 - paw - 2 * dia - 4 * k4;
  const uint64_t path = P3 - 2 * paw - 4 * c4 - 6 * dia - 12 * k4;
  const uint64_t val[6] = {star, path, paw, c4, dia, k4};
  unsigned long long* row = hist + gi * ncls;
#pragma unroll
  for (int k = 0; k < 6; ++k)
    if (val[k]) atomicAdd(&row[P.cls[k]], (unsigned long long)val[k]);
}

unsigned grid_n(uint64_t n) {
  uint64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)b;
}

}  // namespace

// Pair masks (k = 4 layout: bits 0-5 = pairs 01 02 03 12 13 23) of the six
// connected patterns, in the order star, path, paw, 4-cycle, diamond, 4-clique.
static const uint32_t kPatternMask[6] = {7u, 41u, 15u, 45u, 31u, 63u};

constexpr int SPARSE_EDGE_BLOCKS = 152 * 8;

void graphlet_prepare(const hm_graph* g, GraphletScratch& G, cudaStream_t s) {
  G.ngraphs = g->block ? (g->n + g->block - 1) / g->block : 1;
  G.per = g->block ? g->block : g->n;
  const size_t tb = ((size_t)g->n * 4 + 255) & ~(size_t)255;
  const size_t ab = ((size_t)G.ngraphs * NAGG * 8 + 255) & ~(size_t)255;
  // graphs without pair bitmaps: a triangle counter per slot of the pair hash set
  const size_t sb = g->bits2 || !g->counts[2] ? 0 : ((size_t)(g->h2_mask + 1) * 4 + 255) & ~(size_t)255;
  size_t zero = tb + ab + sb, extra = 0;
  size_t keyb = 0;
  if (!g->bits2) {
    // the sort tier's path keys, then the per-warp pair lists
    G.cap = std::max<int64_t>(1, g->max_d2);
    HM_CHECK(g->C4.ready, HM_EINVAL, "4-cycle paths not sized");
    // path keys for the sort (HM_C4_SORT=1), else a table of 2 slots per path
    keyb = ((size_t)g->C4.total * (c4_sort_tier() ? 8 : 16) + 255) & ~(size_t)255;
    extra = keyb + (size_t)SPARSE_EDGE_BLOCKS * SPARSE_WARPS * G.cap * 4;
  }
  G.buf.alloc(zero + extra, s);
  G.tnode = reinterpret_cast<uint32_t*>(G.buf.p);
  G.agg = reinterpret_cast<unsigned long long*>(G.buf.p + tb);
  G.tslot = sb ? reinterpret_cast<uint32_t*>(G.buf.p + tb + ab) : nullptr;
  if (!g->bits2) {
    G.c4_keys = g->C4.total ? reinterpret_cast<uint64_t*>(G.buf.p + zero) : nullptr;
    G.lists = reinterpret_cast<int32_t*>(G.buf.p + zero + keyb);
  }
  HM_CUDA(cudaMemsetAsync(G.buf.p, 0, zero, s));
}

void c4_bounds(hm_graph* g, uint64_t* out, cudaStream_t s) {
  g->c4_warp_ub = c4_warp_bound();
  if (!g->c4_light) {
    g->c4_light = dalloc<uint16_t>((size_t)g->n, s);
    g->owned.push_back(g->c4_light);
  }
  const uint64_t want = ((uint64_t)g->n + 255) / 256;  // 32 nodes per warp
  k_c4_bound<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, 152 * 8)), 256, 0, s>>>(
      g->view(), g->c4_warp_ub, out, g->c4_light);
  HM_KCHECK();
}

void graphlet_edges(const hm_graph* g, GraphletScratch& G, cudaStream_t s) {
  if (g->counts[2] == 0) return;
  TraceSpan span("census_gl_edges", s);
  if (!g->bits2) {
    // 32 nodes per warp
    const uint64_t want = ((uint64_t)g->n + SPARSE_WARPS * 32 - 1) / (SPARSE_WARPS * 32);
    const unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, SPARSE_EDGE_BLOCKS));
    k_graphlet_tri<<<blocks, SPARSE_WARPS * 32, 0, s>>>(g->view(), G.lists, G.cap, G.tslot,
                                                       G.tnode, G.agg);
    HM_KCHECK();
    k_graphlet_tslots<<<grid_n(g->h2_mask + 1), 256, 0, s>>>(g->view(), G.tslot, G.agg);
    HM_KCHECK();
    span.end();
    return;
  }
  // HM_GL_WIDE=1 keeps a warp per pair on short rows too (tests cover both)
  const char* wide = std::getenv("HM_GL_WIDE");
  if (g->bwords <= 16 && !(wide && wide[0] == '1'))
    k_graphlet_edges16<<<grid_n((uint64_t)g->counts[2] * 16), GL_WARPS * 32, 0, s>>>(
        g->view(), G.tnode, G.agg);
  else
    k_graphlet_edges<<<grid_n((uint64_t)g->counts[2] * 32), GL_WARPS * 32, 0, s>>>(
        g->view(), G.tnode, G.agg);
  HM_KCHECK();
  span.end();
}

void graphlet_pairs(const hm_graph* g, GraphletScratch& G, cudaStream_t s) {
  if (!g->bits2) {
    // warp tier over all nodes, then the heavy tier over the heavy nodes (a
    // trace span per stage)
    const uint64_t want = ((uint64_t)g->n + C4_WARPS * 32 - 1) / (C4_WARPS * 32);
    const unsigned wblocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, 152 * 7));
    TraceSpan sw("census_c4_warp", s);
    k_c4_warp<<<wblocks, C4_WARPS * 32, 0, s>>>(g->view(), g->c4_light, G.per, G.agg);
    HM_KCHECK();
    sw.end();
    const uint64_t nk = g->C4.total;
    if (nk && !c4_sort_tier()) {
      TraceSpan st("census_c4_table", s);
      unsigned long long* tab = reinterpret_cast<unsigned long long*>(G.c4_keys);
      HM_CUDA(cudaMemsetAsync(tab, 0xFF, 2 * nk * sizeof(uint64_t), s));
      const uint64_t pieces = (nk + C4T_PIECE - 1) / C4T_PIECE;
      k_c4_table<<<(unsigned)std::min<uint64_t>(pieces, 1u << 30), C4E_THREADS, 0, s>>>(
          g->view(), g->C4.ws, nk, tab, G.per, G.agg);
      HM_KCHECK();
      st.end();
    } else if (nk) {
      const uint64_t eb = std::min<uint64_t>(((uint64_t)g->n + C4E_THREADS - 1) / C4E_THREADS,
                                             152 * 4);
      TraceSpan se("census_c4_emit", s);
      k_c4_emit<<<(unsigned)std::max<uint64_t>(1, eb), C4E_THREADS, 0, s>>>(g->view(), g->bits,
                                                                           g->C4.ws, G.c4_keys);
      HM_KCHECK();
      se.end();
      TraceSpan ss("census_c4_sort", s);
      radix_sort_u64(G.c4_keys, nullptr, (int64_t)nk, 2 * g->bits, s);
      ss.end();
      const uint64_t rb = std::min<uint64_t>((nk + 255) / 256, 152 * 8);
      TraceSpan sr("census_c4_runs", s);
      k_c4_runs<<<(unsigned)rb, 256, 0, s>>>(G.c4_keys, nk, g->bits, G.per, G.agg);
      HM_KCHECK();
      sr.end();
    }
    return;
  }
  TraceSpan span("census_gl_pairs", s);
  k_graphlet_pairs<<<grid_n((uint64_t)g->n * 32), 256, 0, s>>>(g->view(), G.per, G.agg);
  HM_KCHECK();
  span.end();
}

void graphlet_finish(const hm_graph* g, GraphletScratch& G, unsigned long long* hist,
                     cudaStream_t s) {
  const ClassTables& T = class_tables(4);
  PatternClasses P{};
  for (int k = 0; k < 6; ++k) {
    const uint8_t c = T.lut[kPatternMask[k]];
    HM_CHECK(c != 0xFF, HM_EINVAL, "pattern mask is not connected");
    P.cls[k] = c;
  }
  TraceSpan span("census_gl_finish", s);
  // graphs above 16K nodes: the per-node sums over the whole grid first
  // (HM_GL_NODE_SUMS=1 forces it, for the tests)
  const char* ns_env = std::getenv("HM_GL_NODE_SUMS");
  const int node_sums = (G.per > 16384 || (ns_env && ns_env[0] == '1')) ? 1 : 0;
  if (node_sums) {
    k_graphlet_nodes<<<grid_n((uint64_t)g->n), 256, 0, s>>>(g->view(), G.per, G.tnode, G.agg);
    HM_KCHECK();
  }
  k_graphlet_finish<<<(unsigned)G.ngraphs, 256, 0, s>>>(g->view(), G.per, G.tnode, G.agg, T.ncls,
                                                        P, node_sums, hist);
  HM_KCHECK();
  span.end();
}

// Work of the graphlet variant, in bitmap-word operations: every node pair of
// a graph plus every pair of the graph (the 4-clique search adds at most that
// again for the triangles of dense graphs).
double graphlet_cost(const hm_graph* g) {
  const int ngraphs = g->block ? (g->n + g->block - 1) / g->block : 1;
  const double per = g->block ? g->block : g->n;
  return (per * (per - 1) / 2 * ngraphs + 2.0 * (double)g->counts[2]) * (double)g->bwords;
}

}  // namespace hm
