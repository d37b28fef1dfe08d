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

// One thread per pair (u < v): t(e) by the rows' AND, the per-edge sums, t at
// both ends, and the 4-cliques whose two smallest nodes are u < v (for each w
// > v adjacent to both, the common neighbours z > w).
__global__ void k_graphlet_edges(const DevGraph g, uint32_t* __restrict__ tnode,
                                 unsigned long long* __restrict__ agg) {
  const int32_t bw = g.bwords;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < g.m2;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = (int32_t)(g.e2[p] >> 32), v = (int32_t)(g.e2[p] & 0xFFFFFFFFull);
    const int32_t base = graph_base(g, u), vl = v - base;
    const uint32_t* Bu = brow(g.bits2, bw, u);
    const uint32_t* Bv = brow(g.bits2, bw, v);
    uint64_t t = 0, k4 = 0;
    for (int32_t w4 = 0; w4 < bw; w4 += 4) {
      uint32_t a4[4], b4[4];
      ld4(Bu + w4, a4);
      ld4(Bv + w4, b4);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t c = a4[k] & b4[k];
        t += __popc(c);
        uint32_t ws = c & above(w4 + k, vl);
        while (ws) {
          const int j = __ffs(ws) - 1;
          ws &= ws - 1;
          const int32_t wl = (w4 + k) * 32 + j;
          const uint32_t* Bw = brow(g.bits2, bw, base + wl);
          for (int32_t x = w4 + k; x < bw; ++x)
            k4 += __popc(__ldg(Bu + x) & __ldg(Bv + x) & __ldg(Bw + x) & above(x, wl));
        }
      }
    }
    const uint64_t du = (uint64_t)degree(g, u), dv = (uint64_t)degree(g, v);
    atomicAdd(&tnode[u], (uint32_t)t);
    atomicAdd(&tnode[v], (uint32_t)t);
    unsigned long long* A = agg + (int64_t)graph_of(g, u) * NAGG;
    atomicAdd(&A[1], (unsigned long long)((du - 1) * (dv - 1)));
    atomicAdd(&A[2], (unsigned long long)t);
    atomicAdd(&A[4], (unsigned long long)(t * (t - (t > 0 ? 1 : 0)) / 2));
    if (k4) atomicAdd(&A[5], (unsigned long long)k4);
  }
}

// Per node: C(d, 3) and t(v) (d - 2). Per node pair x < z of one graph (pairs
// ranked within the graph's block of ids): C(c(x, z), 2).
__global__ void k_graphlet_nodes_pairs(const DevGraph g, int32_t nodes_per_graph, int32_t ngraphs,
                                       const uint32_t* __restrict__ tnode,
                                       unsigned long long* __restrict__ agg) {
  const int32_t bw = g.bwords;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.n; v += stride) {
    const uint64_t d = (uint64_t)degree(g, (int32_t)v);
    const uint64_t tv = tnode[v] / 2;
    unsigned long long* A = agg + (int64_t)graph_of(g, (int32_t)v) * NAGG;
    if (d >= 3) atomicAdd(&A[0], (unsigned long long)choose3(d));
    if (d >= 2 && tv) atomicAdd(&A[3], (unsigned long long)(tv * (d - 2)));
  }
  const uint64_t per = choose2((uint64_t)nodes_per_graph);
  const uint64_t pairs = per * (uint64_t)ngraphs;
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < pairs; p += stride) {
    const uint64_t gi = p / per;
    uint32_t i, j;
    unrank2(p - gi * per, i, j);
    const int32_t x = (int32_t)(gi * nodes_per_graph + i), z = (int32_t)(gi * nodes_per_graph + j);
    if (z >= g.n) continue;
    const uint32_t* Bx = brow(g.bits2, bw, x);
    const uint32_t* Bz = brow(g.bits2, bw, z);
    uint64_t c = 0;
    for (int32_t w4 = 0; w4 < bw; w4 += 4) {
      uint32_t a4[4], b4[4];
      ld4(Bx + w4, a4);
      ld4(Bz + w4, b4);
      c += __popc(a4[0] & b4[0]) + __popc(a4[1] & b4[1]) + __popc(a4[2] & b4[2]) +
           __popc(a4[3] & b4[3]);
    }
    if (c >= 2) atomicAdd(&agg[gi * NAGG + 6], (unsigned long long)choose2(c));
  }
}

struct PatternClasses {
  int cls[6];  // star, path, paw, c4, diamond, k4
};

// Induced pattern counts of each graph into its histogram row.
__global__ void k_graphlet_finish(const unsigned long long* __restrict__ agg, int ngraphs, int ncls,
                                  const PatternClasses P, unsigned long long* __restrict__ hist) {
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < ngraphs; gi += gridDim.x * blockDim.x) {
    const unsigned long long* A = agg + (int64_t)gi * NAGG;
    const uint64_t T = A[2] / 3, S3 = A[0], P3 = A[1] - 3 * T, TT = A[3], D = A[4], K4 = A[5],
                   C4 = A[6] / 2;
    const uint64_t k4 = K4, dia = D - 6 * K4, c4 = C4 - D + 3 * K4, paw = TT - 4 * D + 12 * K4;
    const uint64_t star = S3 - paw - 2 * dia - 4 * k4;
    const uint64_t path = P3 - 2 * paw - 4 * c4 - 6 * dia - 12 * k4;
    const uint64_t v[6] = {star, path, paw, c4, dia, k4};
    unsigned long long* row = hist + (int64_t)gi * ncls;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (v[k]) atomicAdd(&row[P.cls[k]], (unsigned long long)v[k]);
  }
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

void launch_graphlets(const hm_graph* g, unsigned long long* hist, cudaStream_t s) {
  HM_CHECK(g->bits2 != nullptr, HM_EINVAL, "graphlet census needs pair bitmaps");
  const ClassTables& T = class_tables(4);
  PatternClasses P{};
  for (int k = 0; k < 6; ++k) {
    const uint8_t c = T.lut[kPatternMask[k]];
    HM_CHECK(c != 0xFF, HM_EINVAL, "pattern mask is not connected");
    P.cls[k] = c;
  }
  const int ngraphs = g->block ? (g->n + g->block - 1) / g->block : 1;
  const int32_t per = g->block ? g->block : g->n;
  DBuf<unsigned char> scratch((size_t)g->n * 4 + (size_t)ngraphs * NAGG * 8 + 256, s);
  uint32_t* tnode = reinterpret_cast<uint32_t*>(scratch.p);
  unsigned long long* agg = reinterpret_cast<unsigned long long*>(
      scratch.p + (((size_t)g->n * 4 + 255) & ~(size_t)255));
  HM_CUDA(cudaMemsetAsync(scratch.p, 0, scratch.n, s));
  cudaEvent_t ev = nullptr;
  const bool tr = trace_on();
  if (tr) trace_begin(s, &ev);
  const hm::DevGraph gv = g->view();
  if (g->counts[2] > 0) {
    k_graphlet_edges<<<grid_n((uint64_t)g->counts[2]), 256, 0, s>>>(gv, tnode, agg);
    HM_KCHECK();
  }
  const uint64_t pairs = (uint64_t)choose2((uint64_t)per) * (uint64_t)ngraphs;
  k_graphlet_nodes_pairs<<<grid_n(std::max<uint64_t>(pairs, (uint64_t)g->n)), 256, 0, s>>>(
      gv, per, ngraphs, tnode, agg);
  HM_KCHECK();
  k_graphlet_finish<<<(ngraphs + 63) / 64, 64, 0, s>>>(agg, ngraphs, T.ncls, P, hist);
  HM_KCHECK();
  if (tr) trace_end("census_graphlets", s, ev);
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
