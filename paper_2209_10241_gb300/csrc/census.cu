// Exact census of higher-order motifs of order 3 and 4 (problem statement,
// Sec. 3; efficient exact algorithms, Sec. 4.2, Alg. 2 and Alg. 3).
//
// Alg. 2/3 enumerate candidate node sets from the hyperedges (largest size
// first) and drop repeats with a global "visited" set. Here every connected
// k-node set is generated by exactly one (anchor, item) pair of one family,
// decided by a local canonical-generation rule, so no visited set is needed
// and all families run as flat data-parallel index spaces:
//
//   k = 3  T3  anchor: a 3-hyperedge; the set is the hyperedge (Alg. 2 loop 1)
//          W   anchor: node v, items: pairs x < y of pair-neighbours of v; the
//              set {v,x,y} with no 3-hyperedge (Alg. 2 loop 2); kept when v
//              is the smallest node of induced pair-degree 2
//   k = 4  Q   anchor: a 4-hyperedge (Alg. 3 loop 1)
//          TX  anchor: a 3-hyperedge e; items: hyperedges h of size 2 or 3
//              through a member x of e adding one node d (Alg. 3 loop 2); kept
//              when the set has no 4-hyperedge, e is its smallest 3-hyperedge,
//              h its smallest hyperedge containing d and x = min(h ∩ e)
//          S   anchor: node v, items: triples of pair-neighbours of v; sets
//              with pairs only (Alg. 3 loop 3) holding a node of induced
//              degree 3; kept when v is the smallest such node
//          P   anchor: pair (u,v), items: x in N2(u), y in N2(v); pairs-only
//              sets whose induced degrees are all <= 2 (paths and 4-cycles);
//              kept when (u,v) is the smallest pair whose ends have degree 2
// Hyperedge order for "smallest": size, then the sorted member tuple.
//
// Each candidate's induced sub-hypergraph is filled in by probing its
// subsets of size 2..k (Sec. 4.3) and classified by one lookup of the
// labelled mask in the class table; counts are aggregated per warp
// (__match_any_sync) into shared-memory bins and flushed once per block.
#include <cmath>
#include <algorithm>
#include <cstdlib>
#include <initializer_list>
#include <vector>

#include "families.cuh"

namespace hm {
namespace {

using namespace fam;

// Union of graphs (null-model batch): at most this many graphs per launch,
// each with its own histogram row; block bins are then uint32 (the launch
// keeps every block below 2^31 candidates).
constexpr int MAX_GRAPHS = 64;
constexpr int BIN_STRIDE = 176;

template <class F, bool kBatched>
__global__ void __launch_bounds__(CENSUS_THREADS)
    k_census(const DevGraph g, const F fam, const uint64_t* __restrict__ ws, int64_t A,
             uint64_t total, int chunk, const uint8_t* __restrict__ lut_g, int nmask, int ncls,
             int ngraphs, unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long bins[kBatched ? 1 : BIN_STRIDE];
  __shared__ unsigned int gbins[kBatched ? MAX_GRAPHS * BIN_STRIDE : 1];
  __shared__ uint8_t lut[2048];
  for (int i = threadIdx.x; i < nmask; i += blockDim.x) lut[i] = lut_g[i];
  if (kBatched) {
    for (int i = threadIdx.x; i < ngraphs * BIN_STRIDE; i += blockDim.x) gbins[i] = 0;
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x) bins[i] = 0;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const uint64_t nchunks = (total + chunk - 1) / chunk;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t cb = warp * 32; cb < nchunks; cb += nwarps * 32) {
    const uint64_t g0 = (cb + lane) * chunk;
    const uint64_t g1 = min(g0 + chunk, total);
    typename F::State st;
    int64_t a = 0;
    int32_t gid = 0;
    uint64_t r = 0, wa = 0;
    if (!F::kDirect && g0 < total) {
      a = anchor_of(ws, A, g0);
      r = g0 - ws[a];
      wa = ws[a + 1] - ws[a];
      fam.begin(g, a, r, st);
      if (kBatched) gid = graph_of(g, fam.graph_node(g, a));
    }
    for (int it = 0; it < chunk; ++it) {
      const uint64_t gi = g0 + it;
      int key = -1;
      if (gi < g1) {
        uint32_t mask = 0;
        int32_t nd[4];
        bool ok;
        if (F::kDirect) {
          ok = fam.item(g, (int64_t)gi, st, mask, nd);
          if (kBatched) gid = graph_of(g, fam.graph_node(g, (int64_t)gi));
        } else {
          if (r == wa) {
            do {
              ++a;
            } while (ws[a + 1] == ws[a]);
            r = 0;
            wa = ws[a + 1] - ws[a];
            fam.begin(g, a, 0, st);
            if (kBatched) gid = graph_of(g, fam.graph_node(g, a));
          }
          ok = fam.item(g, a, st, mask, nd);
          ++r;
          fam.next(st);
        }
        if (ok) {
          const uint8_t c = lut[mask];
          key = c == 0xFF ? -1 : (kBatched ? gid * BIN_STRIDE : 0) + (int)c;
        }
      }
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      if (key >= 0 && lane == __ffs(peers) - 1) {
        if (kBatched)
          atomicAdd(&gbins[key], (unsigned int)__popc(peers));
        else
          atomicAdd(&bins[key], (unsigned long long)__popc(peers));
      }
    }
  }
  __syncthreads();
  if (kBatched) {
    for (int i = threadIdx.x; i < ngraphs * BIN_STRIDE; i += blockDim.x)
      if (gbins[i]) atomicAdd(&hist[(i / BIN_STRIDE) * ncls + i % BIN_STRIDE], (unsigned long long)gbins[i]);
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x)
      if (bins[i]) atomicAdd(&hist[i], bins[i]);
  }
}

// Bit-sliced families: each item evaluates up to bwords*32 candidates and
// adds its class counts to the block's bins.
constexpr int BITS_CHUNK = 4;
#ifndef HM_BITS_MINBLOCKS
#define HM_BITS_MINBLOCKS 4  // resident blocks per SM the register budget targets
#endif

template <class F, bool kBatched>
__global__ void __launch_bounds__(CENSUS_THREADS, HM_BITS_MINBLOCKS)
    k_census_bits(const DevGraph g, const F fam, const uint64_t* __restrict__ ws, int64_t A,
                  uint64_t total, const uint8_t* __restrict__ lut_g, int nmask, int ncls,
                  int ngraphs, unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long bins[kBatched ? 1 : BIN_STRIDE];
  __shared__ unsigned int gbins[kBatched ? MAX_GRAPHS * BIN_STRIDE : 1];
  __shared__ uint8_t lut[2048];
  for (int i = threadIdx.x; i < nmask; i += blockDim.x) lut[i] = lut_g[i];
  if (kBatched) {
    for (int i = threadIdx.x; i < ngraphs * BIN_STRIDE; i += blockDim.x) gbins[i] = 0;
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x) bins[i] = 0;
  }
  __syncthreads();
  const uint64_t nchunks = (total + BITS_CHUNK - 1) / BITS_CHUNK;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g0 = c * BITS_CHUNK, g1 = min(g0 + BITS_CHUNK, total);
    typename F::State st;
    int64_t a = anchor_of(ws, A, g0);
    uint64_t r = g0 - ws[a], wa = ws[a + 1] - ws[a];
    fam.begin(g, a, r, st);
    int32_t gid = kBatched ? graph_of(g, fam.graph_node(g, a)) : 0;
    for (uint64_t gi = g0; gi < g1; ++gi) {
      if (r == wa) {
        do {
          ++a;
        } while (ws[a + 1] == ws[a]);
        r = 0;
        wa = ws[a + 1] - ws[a];
        fam.begin(g, a, 0, st);
        if (kBatched) gid = graph_of(g, fam.graph_node(g, a));
      }
      if (kBatched)
        fam.item(g, a, st, lut, gbins + gid * BIN_STRIDE);
      else
        fam.item(g, a, st, lut, bins);
      ++r;
      fam.next(st);
    }
  }
  __syncthreads();
  if (kBatched) {
    for (int i = threadIdx.x; i < ngraphs * BIN_STRIDE; i += blockDim.x)
      if (gbins[i]) atomicAdd(&hist[(i / BIN_STRIDE) * ncls + i % BIN_STRIDE], (unsigned long long)gbins[i]);
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x)
      if (bins[i]) atomicAdd(&hist[i], bins[i]);
  }
}

// ---------------------------------------------------------------- work spaces
__global__ void k_ws_nodes(const int64_t* __restrict__ off2, int32_t n, int choose,
                           uint64_t* __restrict__ w) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t d = (uint64_t)(off2[v + 1] - off2[v]);
    w[v] = choose == 2 ? choose2(d) : choose3(d);
  }
}

// bit-sliced spaces: W -> d (d >= 2), S -> C(d, 2) per node; P -> d(u) - 1 per pair (u, v)
__global__ void k_ws_nodes_bits(const int64_t* __restrict__ off2, int32_t n, int choose,
                                uint64_t* __restrict__ w) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t d = (uint64_t)(off2[v + 1] - off2[v]);
    w[v] = choose == 2 ? (d >= 2 ? d : 0) : choose2(d);
  }
}

__global__ void k_ws_pairs_bits(const uint64_t* __restrict__ e2, int64_t m,
                                const int64_t* __restrict__ off2, uint64_t* __restrict__ w) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = (int32_t)(e2[p] >> 32), v = (int32_t)(e2[p] & 0xFFFFFFFFull);
    const uint64_t du = (uint64_t)(off2[u + 1] - off2[u]), dv = (uint64_t)(off2[v + 1] - off2[v]);
    w[p] = dv > 1 ? du - 1 : 0;
  }
}

__global__ void k_ws_pairs(const uint64_t* __restrict__ e2, int64_t m, const int64_t* __restrict__ off2,
                           uint64_t* __restrict__ w) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = (int32_t)(e2[p] >> 32), v = (int32_t)(e2[p] & 0xFFFFFFFFull);
    const uint64_t du = (uint64_t)(off2[u + 1] - off2[u]), dv = (uint64_t)(off2[v + 1] - off2[v]);
    w[p] = (du - 1) * (dv - 1);
  }
}

__global__ void k_ws_triples(const int4* __restrict__ e3, int64_t m, const int64_t* __restrict__ off2,
                             const int64_t* __restrict__ off3, uint64_t* __restrict__ w) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 e = e3[t];
    uint64_t s = 0;
    const int32_t xs[3] = {e.x, e.y, e.z};
#pragma unroll
    for (int j = 0; j < 3; ++j)
      s += (uint64_t)(off2[xs[j] + 1] - off2[xs[j]]) + (uint64_t)(off3[xs[j] + 1] - off3[xs[j]]);
    w[t] = s;
  }
}

unsigned grid1d(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

// Prefix sums of the candidates per anchor for every family in `todo`, with
// one host synchronisation for all of them (the totals size the launches).
void ensure_spaces(hm_graph* g, std::initializer_list<std::pair<hm_graph::Space*, char>> todo,
                   cudaStream_t s) {
  std::vector<std::pair<hm_graph::Space*, char>> need;
  for (auto& t : todo)
    if (!t.first->ready) need.push_back(t);
  if (need.empty()) return;
  DBuf<uint64_t> totals(need.size(), s);
  std::vector<uint64_t*> made;
  try {
    for (size_t i = 0; i < need.size(); ++i) {
      hm_graph::Space& sp = *need[i].first;
      const char fam = need[i].second;
      int64_t A = 0;
      if (fam == 'W' || fam == 'S' || fam == 'w' || fam == 's') A = g->n;
      if (fam == 'P' || fam == 'p') A = g->counts[2];
      if (fam == 'X') A = g->kmax >= 3 ? g->counts[3] : 0;
      DBuf<uint64_t> w(A, s);
      uint64_t* ws = dalloc<uint64_t>((size_t)A + 1, s);
      made.push_back(ws);
      if (A > 0) {
        if (fam == 'W' || fam == 'S')
          k_ws_nodes<<<grid1d(A), 256, 0, s>>>(g->off2, g->n, fam == 'W' ? 2 : 3, w.p);
        else if (fam == 'w' || fam == 's')
          k_ws_nodes_bits<<<grid1d(A), 256, 0, s>>>(g->off2, g->n, fam == 'w' ? 2 : 3, w.p);
        else if (fam == 'P')
          k_ws_pairs<<<grid1d(A), 256, 0, s>>>(g->e2, A, g->off2, w.p);
        else if (fam == 'p')
          k_ws_pairs_bits<<<grid1d(A), 256, 0, s>>>(g->e2, A, g->off2, w.p);
        else
          k_ws_triples<<<grid1d(A), 256, 0, s>>>(g->e3, A, g->off2, g->off3, w.p);
        HM_KCHECK();
      }
      scan_exclusive_u64(w.p, ws, A, s);
      HM_CUDA(cudaMemcpyAsync(totals.p + i, ws + A, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
      sp.anchors = A;
    }
    std::vector<uint64_t> h(need.size());
    HM_CUDA(cudaMemcpyAsync(h.data(), totals.p, h.size() * sizeof(uint64_t),
                            cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    for (size_t i = 0; i < need.size(); ++i) {
      need[i].first->ws = made[i];
      need[i].first->total = h[i];
      need[i].first->ready = true;
    }
  } catch (...) {
    for (uint64_t* p : made) cudaFreeAsync(p, s);
    throw;
  }
}

// Persistent grid: SMs x resident blocks, capped by the work; with a union
// of graphs, enough blocks that no block counts 2^31 candidates.
int grid_for(const void* kernel, uint64_t lanes_needed, uint64_t max_candidates, bool batched) {
  int dev = 0, sms = 0, per_sm = 0;
  HM_CUDA(cudaGetDevice(&dev));
  HM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, CENSUS_THREADS, 0));
  if (per_sm < 1) per_sm = 1;
  const uint64_t need = (lanes_needed + CENSUS_THREADS - 1) / CENSUS_THREADS;
  uint64_t blocks = (uint64_t)sms * per_sm;
  if (batched) {
    const uint64_t floor_blocks = max_candidates / (1ull << 31) + 1;
    if (blocks < floor_blocks) blocks = floor_blocks;
  }
  if (need < blocks) blocks = need;
  if (blocks > (1ull << 30)) blocks = 1ull << 30;
  return (int)(blocks < 1 ? 1 : blocks);
}

int num_graphs(const hm_graph* g) { return g->block ? (g->n + g->block - 1) / g->block : 1; }

template <class F, bool kBatched>
void launch_bits_t(const hm_graph* g, const F& fam, const hm_graph::Space& sp, int order,
                   unsigned long long* hist, cudaStream_t s) {
  const ClassTables& T = class_tables(order);
  const uint8_t* lut = device_lut(order);
  const uint64_t lanes = (sp.total + BITS_CHUNK - 1) / BITS_CHUNK;
  const uint64_t max_cand = sp.total * (uint64_t)g->bwords * 32;
  const int blocks = grid_for((const void*)k_census_bits<F, kBatched>, lanes, max_cand, kBatched);
  cudaEvent_t ev = nullptr;
  const bool tr = trace_on();
  if (tr) trace_begin(s, &ev);
  k_census_bits<F, kBatched><<<blocks, CENSUS_THREADS, 0, s>>>(
      g->view(), fam, sp.ws, sp.anchors, sp.total, lut, (int)T.lut.size(), T.ncls, num_graphs(g),
      hist);
  HM_KCHECK();
  if (tr) trace_end(F::kName, s, ev);
}

template <class F>
void launch_bits(const hm_graph* g, const F& fam, const hm_graph::Space& sp, int order,
                 unsigned long long* hist, cudaStream_t s) {
  if (sp.total == 0) return;
  if (g->block)
    launch_bits_t<F, true>(g, fam, sp, order, hist, s);
  else
    launch_bits_t<F, false>(g, fam, sp, order, hist, s);
}

template <class F, bool kBatched>
void launch_family_t(const hm_graph* g, const F& fam, const hm_graph::Space* sp, uint64_t total,
                     int order, unsigned long long* hist, cudaStream_t s) {
  const ClassTables& T = class_tables(order);
  const uint8_t* lut = device_lut(order);
  // consecutive candidates per lane: up to CHUNK, fewer when the family is
  // too small to fill the GPU that way (every lane of a warp takes the same)
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const uint64_t lanes_wanted = (uint64_t)sms * 2048;
  int chunk = (int)std::min<uint64_t>(CHUNK, (total + lanes_wanted - 1) / lanes_wanted);
  if (chunk < 1) chunk = 1;
  const int blocks = grid_for((const void*)k_census<F, kBatched>, (total + chunk - 1) / chunk,
                              total, kBatched);
  cudaEvent_t ev = nullptr;
  const bool tr = trace_on();
  if (tr) trace_begin(s, &ev);
  k_census<F, kBatched><<<blocks, CENSUS_THREADS, 0, s>>>(
      g->view(), fam, sp ? sp->ws : nullptr, sp ? sp->anchors : 0, total, chunk, lut,
      (int)T.lut.size(), T.ncls, num_graphs(g), hist);
  HM_KCHECK();
  if (tr) trace_end(F::kName, s, ev);
}

template <class F>
void launch_family(const hm_graph* g, const F& fam, const hm_graph::Space* sp, uint64_t total,
                   int order, unsigned long long* hist, cudaStream_t s) {
  if (total == 0) return;
  if (g->block)
    launch_family_t<F, true>(g, fam, sp, total, order, hist, s);
  else
    launch_family_t<F, false>(g, fam, sp, total, order, hist, s);
}

}  // namespace

// Work spaces and launches of the census of one order; shared with the
// null-model batch.
// The bit-sliced variant of a family is used when its estimated cost, items
// x bitmap words scanned x the cost of a word relative to one per-candidate
// evaluation (measured on this GPU: ~0.35 with 4-word loads, where the
// per-candidate kernels run at ~12 % SIMT efficiency), is below the number of
// candidates it replaces. Star and wedge items scan the words above their
// second node (half a row on average), path items the whole row.
// HM_DENSE_FAMILIES=0 / 1 forces the per-candidate / bit-sliced variants (the
// latter whenever bitmaps exist).
bool prefer_bits(const hm_graph* g, const hm_graph::Space& bits, uint64_t candidates,
                 double row_fraction) {
  if (!g->bits2) return false;
  const char* env = std::getenv("HM_DENSE_FAMILIES");
  if (env && env[0] == '0') return false;
  if (env && env[0] == '1') return true;
  const double words = 2.0 + (double)g->bwords * row_fraction;
  return (double)bits.total * words * 0.35 < (double)candidates;
}

void prepare_census(hm_graph* g, int order, cudaStream_t s) {
  if (order == 3) {
    if (g->bits2)
      ensure_spaces(g, {{&g->W, 'W'}, {&g->Wb, 'w'}}, s);
    else
      ensure_spaces(g, {{&g->W, 'W'}}, s);
    if (g->bits2) g->useWb = prefer_bits(g, g->Wb, g->W.total, 0.5);
  } else {
    HM_CHECK(g->max_d2 < (1 << 21), HM_EUNSUPPORTED,
             "a node has 2^21 or more pair neighbours; order-4 star space overflows");
    if (g->bits2)
      ensure_spaces(g, {{&g->S, 'S'}, {&g->P, 'P'}, {&g->TX, 'X'}, {&g->Sb, 's'}, {&g->Pb, 'p'}},
                    s);
    else
      ensure_spaces(g, {{&g->S, 'S'}, {&g->P, 'P'}, {&g->TX, 'X'}}, s);
    if (g->bits2) {
      g->useSb = prefer_bits(g, g->Sb, g->S.total, 0.5);
      g->usePb = prefer_bits(g, g->Pb, g->P.total, 1.0);
    }
  }
}

void launch_census(const hm_graph* g, int order, unsigned long long* hist, cudaStream_t s) {
  if (order == 3) {
    launch_family(g, FamT3{}, nullptr, (uint64_t)g->counts[3], 3, hist, s);
    if (g->useWb && g->tri3)
      launch_bits(g, BitsWT<true>{}, g->Wb, 3, hist, s);
    else if (g->useWb)
      launch_bits(g, BitsWT<false>{}, g->Wb, 3, hist, s);
    else
      launch_family(g, FamW{}, &g->W, g->W.total, 3, hist, s);
  } else {
    launch_family(g, FamQ{}, nullptr, (uint64_t)g->counts[4], 4, hist, s);
    launch_family(g, FamTX{}, &g->TX, g->TX.total, 4, hist, s);
    if (g->useSb && g->tri3)
      launch_bits(g, BitsST<true>{}, g->Sb, 4, hist, s);
    else if (g->useSb)
      launch_bits(g, BitsST<false>{}, g->Sb, 4, hist, s);
    else
      launch_family(g, FamS{}, &g->S, g->S.total, 4, hist, s);
    if (g->usePb && g->tri3)
      launch_bits(g, BitsPT<true>{}, g->Pb, 4, hist, s);
    else if (g->usePb)
      launch_bits(g, BitsPT<false>{}, g->Pb, 4, hist, s);
    else
      launch_family(g, FamP{}, &g->P, g->P.total, 4, hist, s);
  }
}

}  // namespace hm

extern "C" hm_status hm_count_exact(hm_graph* g, int order, uint64_t* d_hist, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g != nullptr, HM_EINVAL, "NULL graph");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= g->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    HM_CHECK(d_hist != nullptr, HM_EINVAL, "NULL histogram");
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CHECK(dev == g->device, HM_EINVAL, "graph was built on another device");
    cudaStream_t s = (cudaStream_t)stream;
    hm::prepare_census(g, order, s);
    HM_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(uint64_t) * hm::class_tables(order).ncls, s));
    hm::launch_census(g, order, (unsigned long long*)d_hist, s);
  });
}

extern "C" hm_status hm_count_exact_host(const int32_t* h_members, const int64_t* h_offsets,
                                         int64_t num_hyperedges, int32_t num_nodes, int order,
                                         uint64_t* h_hist, void* stream) {
  hm_graph* g = nullptr;
  hm_status st = hm::guarded([&] {
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(h_offsets && h_hist, HM_EINVAL, "NULL argument");
    HM_CHECK(num_hyperedges >= 0 && num_hyperedges < (1ll << 31), HM_EINVAL,
             "num_hyperedges must be in [0, 2^31)");
    HM_CHECK(num_nodes >= 1, HM_EINVAL, "num_nodes must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t total = h_offsets[num_hyperedges];
    HM_CHECK(total >= 0 && (total == 0 || h_members), HM_EINVAL, "bad members/offsets");
    hm::DBuf<int32_t> mem(total, s);
    hm::DBuf<int64_t> off(num_hyperedges + 1, s);
    hm::DBuf<unsigned long long> hist(hm::class_tables(order).ncls, s);
    if (total)
      HM_CUDA(cudaMemcpyAsync(mem.p, h_members, total * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyAsync(off.p, h_offsets, (num_hyperedges + 1) * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s));
    g = new hm_graph;
    hm::build_graph(g, mem.p, off.p, num_hyperedges, num_nodes, order, s);
    hm::prepare_census(g, order, s);
    HM_CUDA(cudaMemsetAsync(hist.p, 0, hist.n * sizeof(unsigned long long), s));
    hm::launch_census(g, order, hist.p, s);
    HM_CUDA(cudaMemcpyAsync(h_hist, hist.p, hist.n * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
  });
  if (g) {
    std::string msg = hm_last_error();
    hm::free_graph(g);
    hm::set_last_error(msg);
  }
  return st;
}

extern "C" hm_status hm_work_totals(hm_graph* g, int order, uint64_t* totals, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g && totals, HM_EINVAL, "NULL argument");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= g->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    hm::prepare_census(g, order, (cudaStream_t)stream);
    for (int i = 0; i < 8; ++i) totals[i] = 0;
    if (order == 3) {
      totals[0] = (uint64_t)g->counts[3];
      totals[1] = g->W.total;
      totals[2] = g->Wb.total;
      totals[3] = g->useWb ? 1 : 0;
    } else {
      totals[0] = (uint64_t)g->counts[4];
      totals[1] = g->TX.total;
      totals[2] = g->S.total;
      totals[3] = g->P.total;
      totals[4] = g->Sb.total;
      totals[5] = g->Pb.total;
      totals[6] = g->useSb ? 1 : 0;
      totals[7] = g->usePb ? 1 : 0;
    }
  });
}
