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

// Called by every thread of the block (blockDim.x = 32 * NW) after the pair
// loop; lane 0 of each warp holds its run.
template <int NW>
__device__ __forceinline__ void pair_sums_block(const PairSums& P, unsigned long long* agg) {
  __shared__ int32_t gi_s[NW];
  __shared__ uint64_t v_s[NW][4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    gi_s[wid] = P.gi;
#pragma unroll
    for (int i = 0; i < 4; ++i) v_s[wid][i] = P.v[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    PairSums R;
    for (int w = 0; w < NW; ++w) {
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

// One warp per pair (u < v): t(e) = popcount of the rows' AND (lanes over
// words, kept in shared memory), the 4-cliques whose two smallest nodes are
// u < v (common neighbours w > v listed in shared memory and shared out over
// the lanes), then the per-pair sums and t(e) added at both ends. Rows longer
// than GL_MAXW words take the lanes over words directly.
__global__ void __launch_bounds__(GL_WARPS * 32)
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

// Graphs without pair bitmaps. One warp per pair (u < v): t(e) by hash probes
// of the shorter adjacency list against the other endpoint; the common
// neighbours w > v, in ascending order, go to the warp's list (capacity = the
// largest pair degree) and every pair of them that is itself a pair closes a
// 4-clique with u and v.
__global__ void __launch_bounds__(SPARSE_WARPS * 32)
    k_graphlet_edges_sparse(const DevGraph g, int32_t* __restrict__ lists, int64_t cap,
                                        uint32_t* __restrict__ tnode,
                                        unsigned long long* __restrict__ agg) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* list = lists + gw * cap;
  PairSums P;
  for (int64_t p = gw; p < g.m2; p += warps) {
    const int32_t u = (int32_t)(g.e2[p] >> 32), v = (int32_t)(g.e2[p] & 0xFFFFFFFFull);
    const int32_t du = degree(g, u), dv = degree(g, v);
    const int32_t a = du <= dv ? u : v, b = du <= dv ? v : u, da = du <= dv ? du : dv;
    const int64_t oa = g.off2[a];
    uint32_t t = 0;
    int count = 0;
    for (int32_t i0 = 0; i0 < da; i0 += 32) {
      const int32_t i = i0 + lane;
      const int32_t w = i < da ? g.adj2[oa + i] : -1;
      const bool common = w >= 0 && w != b && has_pair(g, b, w);
      t += common ? 1u : 0u;
      const bool keep = common && w > v;
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) list[count + __popc(bal & lt)] = w;
      count += __popc(bal);
    }
    __syncwarp();
    uint64_t k4 = 0;
    for (int i = lane; i < count; i += 32) {
      const int32_t wi = list[i];
      for (int j = i + 1; j < count; ++j) k4 += has_pair(g, wi, list[j]) ? 1u : 0u;
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      t += __shfl_xor_sync(0xffffffffu, t, o);
      k4 += __shfl_xor_sync(0xffffffffu, k4, o);
    }
    if (lane == 0) {
      atomicAdd(&tnode[u], t);
      atomicAdd(&tnode[v], t);
      pair_sums_add(P, agg, graph_of(g, u), (uint64_t)du, (uint64_t)dv, t, k4);
    }
  }
  pair_sums_block<SPARSE_WARPS>(P, agg);
}

// 4-cycles of graphs without pair bitmaps, each at its highest-ranked node x
// (rank = (degree, id)): the nodes z of lower rank reached by paths x - y - z
// through a y of lower rank are counted (per-block dense counters, with the
// list of the counters touched); every two such paths to one z close a
// 4-cycle x - y - z - y'. Adds 2 C4 to the graph's sum, as the bitmap kernel
// does.
__global__ void k_graphlet_c4_sparse(const DevGraph g, int32_t nodes_per_graph,
                                     uint32_t* __restrict__ acc_all, int32_t* __restrict__ touched_all,
                                     unsigned long long* __restrict__ agg) {
  __shared__ int tcount;
  __shared__ unsigned long long part[32];
  uint32_t* acc = acc_all + (size_t)blockIdx.x * g.n;
  int32_t* touched = touched_all + (size_t)blockIdx.x * g.n;
  // thread 0: the block's running sum for graph gcur, one atomic per graph
  int64_t gcur = -1;
  uint64_t scur = 0;
  for (int64_t x = blockIdx.x; x < g.n; x += gridDim.x) {
    const int32_t dx = degree(g, (int32_t)x);
    if (threadIdx.x == 0) tcount = 0;
    __syncthreads();
    const int64_t ox = g.off2[x];
    for (int32_t i = threadIdx.x; i < dx; i += blockDim.x) {
      const int32_t y = g.adj2[ox + i];
      const int32_t dy = degree(g, y);
      if (!(dy < dx || (dy == dx && y < x))) continue;
      const int64_t oy = g.off2[y];
      for (int32_t k = 0; k < dy; ++k) {
        const int32_t z = g.adj2[oy + k];
        if (z == x) continue;
        const int32_t dz = degree(g, z);
        if (!(dz < dx || (dz == dx && z < x))) continue;
        if (atomicAdd(&acc[z], 1u) == 0u) touched[atomicAdd(&tcount, 1)] = z;
      }
    }
    __syncthreads();
    uint64_t sum = 0;
    const int tc = tcount;
    for (int i = threadIdx.x; i < tc; i += blockDim.x) {
      const int32_t z = touched[i];
      const uint64_t c = acc[z];
      sum += c * (c - 1) / 2;
      acc[z] = 0;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
      const int64_t gi = x / nodes_per_graph;
      if (gi != gcur) {
        if (scur) atomicAdd(&agg[gcur * NAGG + 6], (unsigned long long)(2 * scur));
        gcur = gi;
        scur = 0;
      }
      scur += s;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && scur) atomicAdd(&agg[gcur * NAGG + 6], (unsigned long long)(2 * scur));
}

struct PatternClasses {
  int cls[6];  // star, path, paw, c4, diamond, k4
};

// One block per graph: the per-node sums C(d, 3) and t(v) (d - 2), then the
// induced pattern counts into the graph's histogram row.
__global__ void k_graphlet_finish(const DevGraph g, int32_t nodes_per_graph,
                                  const uint32_t* __restrict__ tnode,
                                  const unsigned long long* __restrict__ agg, int ncls,
                                  const PatternClasses P, unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long part[2][8];
  const int64_t gi = blockIdx.x;
  const int64_t v0 = gi * nodes_per_graph, v1 = min((int64_t)g.n, v0 + nodes_per_graph);
  uint64_t s3 = 0, tt = 0;
  for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
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
  uint64_t S3 = 0, TT = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    S3 += part[0][w];
    TT += part[1][w];
  }
  const unsigned long long* A = agg + gi * NAGG;
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

constexpr int SPARSE_C4_BLOCKS = 152;
constexpr int SPARSE_EDGE_BLOCKS = 152 * 8;

void graphlet_prepare(const hm_graph* g, GraphletScratch& G, cudaStream_t s) {
  G.ngraphs = g->block ? (g->n + g->block - 1) / g->block : 1;
  G.per = g->block ? g->block : g->n;
  const size_t tb = ((size_t)g->n * 4 + 255) & ~(size_t)255;
  const size_t ab = ((size_t)G.ngraphs * NAGG * 8 + 255) & ~(size_t)255;
  size_t zero = tb + ab, extra = 0;
  if (!g->bits2) {
    // 4-cycle counters (zero) and touched lists per block; pair lists per warp
    G.cap = std::max<int64_t>(1, g->max_d2);
    zero += (size_t)SPARSE_C4_BLOCKS * g->n * 4;
    extra = (size_t)SPARSE_C4_BLOCKS * g->n * 4 + (size_t)SPARSE_EDGE_BLOCKS * SPARSE_WARPS * G.cap * 4;
  }
  G.buf.alloc(zero + extra, s);
  G.tnode = reinterpret_cast<uint32_t*>(G.buf.p);
  G.agg = reinterpret_cast<unsigned long long*>(G.buf.p + tb);
  if (!g->bits2) {
    G.acc = reinterpret_cast<uint32_t*>(G.buf.p + tb + ab);
    G.touched = reinterpret_cast<int32_t*>(G.buf.p + zero);
    G.lists = G.touched + (size_t)SPARSE_C4_BLOCKS * g->n;
  }
  HM_CUDA(cudaMemsetAsync(G.buf.p, 0, zero, s));
}

void graphlet_edges(const hm_graph* g, GraphletScratch& G, cudaStream_t s) {
  if (g->counts[2] == 0) return;
  TraceSpan span("census_gl_edges", s);
  if (!g->bits2) {
    const uint64_t want = ((uint64_t)g->counts[2] * 32 + 255) / 256;
    const unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, SPARSE_EDGE_BLOCKS));
    k_graphlet_edges_sparse<<<blocks, SPARSE_WARPS * 32, 0, s>>>(g->view(), G.lists, G.cap, G.tnode, G.agg);
    HM_KCHECK();
    span.end();
    return;
  }
  k_graphlet_edges<<<grid_n((uint64_t)g->counts[2] * 32), GL_WARPS * 32, 0, s>>>(g->view(), G.tnode,
                                                                                 G.agg);
  HM_KCHECK();
  span.end();
}

void graphlet_pairs(const hm_graph* g, GraphletScratch& G, cudaStream_t s) {
  TraceSpan span("census_gl_pairs", s);
  if (!g->bits2) {
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(g->n, SPARSE_C4_BLOCKS));
    k_graphlet_c4_sparse<<<blocks, 256, 0, s>>>(g->view(), G.per, G.acc, G.touched, G.agg);
    HM_KCHECK();
    span.end();
    return;
  }
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
  k_graphlet_finish<<<(unsigned)G.ngraphs, 256, 0, s>>>(g->view(), G.per, G.tnode, G.agg, T.ncls,
                                                        P, hist);
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
