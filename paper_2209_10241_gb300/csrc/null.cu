// Null-model batch: the counting step repeated on randomised hypergraphs
// (motif analysis compares observed counts with a null model, Sec. 1 and
// Sec. 6.3, which samples 10 draws of a configuration model). The null model
// here is stub shuffling: the stubs (members in input order) of a base
// hypergraph are reordered by the keys (v >> 6, i), v the 64-bit Philox value
// for counter (i lo, i hi, model, "NULL"), and cut again into the input sizes.
// Degrees and hyperedge sizes are kept up to the collapse of repeated members
// and duplicate hyperedges that normalisation then applies.
//
// A batch of up to 64 models is counted as ONE disjoint union: model t's node
// v becomes t * block + v (block = the largest base node count), so one
// ingest and one persistent launch per candidate family cover every model,
// whatever their sizes, and the census kernels route each count to the
// histogram row of the anchor's model.
#include <algorithm>

#include "hm_internal.cuh"

namespace hm {
namespace {

constexpr uint32_t TAG_NULL = 0x4E554C4Cu;  // "NULL"
constexpr int GROUP = 64;                   // models per union (6-bit model field)

struct ModelInfo {
  int64_t base_stub0;  // first stub of the model's base in the input members
  int64_t stub0;       // first stub of the model in the union
  int64_t base_edge0;  // first hyperedge of the model's base in the input
  int64_t edge0;       // first hyperedge of the model in the union
  int32_t node0;       // t * block
  uint32_t model_id;   // Philox lane of this model
  int32_t n;           // node count of the model's base
};

__device__ __forceinline__ int model_of_stub(const ModelInfo* __restrict__ mi, int T, int64_t p) {
  int lo = 0, hi = T;  // last t with stub0 <= p
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (mi[mid].stub0 <= p)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int model_of_edge(const ModelInfo* __restrict__ mi, int T, int64_t e) {
  int lo = 0, hi = T;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (mi[mid].edge0 <= e)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// sort key of every stub: model in the top 6 bits, then the top 58 bits of its draw
__global__ void k_stub_keys(const ModelInfo* __restrict__ mi, int T, int64_t total, uint64_t seed,
                            uint64_t* __restrict__ keys, uint64_t* __restrict__ src) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int t = model_of_stub(mi, T, p);
    const uint64_t i = (uint64_t)(p - mi[t].stub0);
    const uint64_t v = philox_draw64(seed, i, mi[t].model_id, TAG_NULL);
    keys[p] = ((uint64_t)t << 58) | (v >> 6);
    src[p] = (uint64_t)(mi[t].base_stub0 + (int64_t)i);
  }
}

// after the stable sort, position p of model t receives the stub src[p]
__global__ void k_union_members(const ModelInfo* __restrict__ mi, int T, int64_t total,
                                const uint64_t* __restrict__ src,
                                const int32_t* __restrict__ members, int32_t* __restrict__ out,
                                int* __restrict__ err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int t = model_of_stub(mi, T, p);
    const int32_t v = members[src[p]];
    if (v < 0 || v >= mi[t].n) {
      atomicOr(err, 1);
      out[p] = mi[t].node0;
    } else {
      out[p] = mi[t].node0 + v;
    }
  }
}

// the model's hyperedges keep their base sizes
__global__ void k_union_offsets(const ModelInfo* __restrict__ mi, int T, int64_t edges,
                                int64_t stubs, const int64_t* __restrict__ offsets,
                                int64_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= edges;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e == edges) {
      out[e] = stubs;
      continue;
    }
    const int t = model_of_edge(mi, T, e);
    const int64_t je = mi[t].base_edge0 + (e - mi[t].edge0);
    out[e] = mi[t].stub0 + (offsets[je] - offsets[mi[t].base_edge0]);
  }
}

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

// ---------------------------------------------------------------- configuration model (MCMC)
// Chodrow's configuration model of hypergraphs (the null model Sec. 6.3
// cites), sampled by pairwise reshuffles: a pair of hyperedges e, f keeps its
// intersection I and re-deals the other |e| + |f| - 2|I| members at random,
// |e| - |I| of them to e and the rest to f. The move returns to the old state
// with the same probability as it left it (I and the re-dealt set are
// preserved), so the chain is symmetric and its stationary distribution is
// uniform over the hyperedge-labelled hypergraphs with the input's degrees
// and sizes and no repeated member in a hyperedge. A round pairs every
// model's hyperedges by a random matching (hyperedges sorted by Philox keys,
// consecutive positions paired, an odd one out stays) and reshuffles every
// pair at once: disjoint moves commute, and a mixture of symmetric moves is
// symmetric. Pairs with more than MCMC_CAP re-dealt members are left as they
// are (that set is preserved by every move, so skipping it is symmetric too).
constexpr uint32_t TAG_MCMC = 0x4D434D43u;  // "MCMC"
constexpr int MCMC_CAP = 255;

// starting state: model t's members are its base's, shifted into its block
__global__ void k_union_copy(const ModelInfo* __restrict__ mi, int T, int64_t total,
                             const int32_t* __restrict__ members, int32_t* __restrict__ out,
                             int* __restrict__ err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int t = model_of_stub(mi, T, p);
    const int32_t v = members[mi[t].base_stub0 + (p - mi[t].stub0)];
    if (v < 0 || v >= mi[t].n) {
      atomicOr(err, 1);
      out[p] = mi[t].node0;
    } else {
      out[p] = mi[t].node0 + v;
    }
  }
}

// matching keys of round r: model in the top 6 bits, then the top 58 bits of
// the draw of hyperedge i of the model (counter ((r << 32) | i, model << 8, "MCMC"))
__global__ void k_match_keys(const ModelInfo* __restrict__ mi, int T, int64_t edges, uint64_t seed,
                             uint32_t round, uint64_t* __restrict__ keys, uint64_t* __restrict__ idx) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < edges;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int t = model_of_edge(mi, T, e);
    const uint64_t i = (uint64_t)(e - mi[t].edge0);
    const uint64_t v = philox_draw64(seed, ((uint64_t)round << 32) | i, mi[t].model_id << 8, TAG_MCMC);
    keys[e] = ((uint64_t)t << 58) | (v >> 6);
    idx[e] = (uint64_t)e;
  }
}

// One pairwise reshuffle per pair k of each model: the hyperedges at sorted
// positions edge0 + 2k and edge0 + 2k + 1. The re-dealt members S (e's
// members outside f, in order, then f's outside e) and their slots are
// listed; draw q of the pair (counter ((r << 32) | k, (model << 8) | (q + 1),
// "MCMC")) picks j = q + mulhi(draw, |S| - q) for step q of a partial
// Fisher-Yates shuffle (q < |e \ f|, and q < |S| - 1), and S then goes back
// into the listed slots in order: e's slots get the first |e \ f|.
__global__ void k_reshuffle(const ModelInfo* __restrict__ mi, int T, int64_t edges, uint64_t seed,
                            uint32_t round, const uint64_t* __restrict__ order,
                            const int64_t* __restrict__ off, int32_t* __restrict__ mem,
                            int* __restrict__ err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < edges;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int t = model_of_edge(mi, T, p);
    const int64_t in_model = p - mi[t].edge0;
    const int64_t m_t = (t + 1 < T ? mi[t + 1].edge0 : edges) - mi[t].edge0;
    if ((in_model & 1) || in_model + 1 >= m_t) continue;
    const int64_t e = (int64_t)order[p], f = (int64_t)order[p + 1];
    const int64_t e0 = off[e], f0 = off[f];
    const int le = (int)(off[e + 1] - e0), lf = (int)(off[f + 1] - f0);
    int32_t S[MCMC_CAP];
    int64_t slot[MCMC_CAP];
    int ns = 0;
    bool skip = false;
    for (int x = 0; x < le; ++x) {
      const int32_t v = mem[e0 + x];
      bool shared = false;
      for (int y = 0; y < lf; ++y) shared |= mem[f0 + y] == v;
      for (int y = 0; y < x; ++y)
        if (mem[e0 + y] == v) atomicOr(err, 2);
      if (shared) continue;
      if (ns == MCMC_CAP) {
        skip = true;
        break;
      }
      S[ns] = v;
      slot[ns++] = e0 + x;
    }
    const int ae = ns;
    for (int y = 0; y < lf && !skip; ++y) {
      const int32_t v = mem[f0 + y];
      bool shared = false;
      for (int x = 0; x < le; ++x) shared |= mem[e0 + x] == v;
      for (int x = 0; x < y; ++x)
        if (mem[f0 + x] == v) atomicOr(err, 2);
      if (shared) continue;
      if (ns == MCMC_CAP) {
        skip = true;
        break;
      }
      S[ns] = v;
      slot[ns++] = f0 + y;
    }
    if (skip || ns < 2 || ae == 0 || ae == ns) continue;
    const uint64_t k = (uint64_t)(in_model >> 1);
    const uint32_t lane = mi[t].model_id << 8;
    for (int q = 0; q < ae && q < ns - 1; ++q) {
      const uint64_t v = philox_draw64(seed, ((uint64_t)round << 32) | k, lane | (uint32_t)(q + 1),
                                       TAG_MCMC);
      const int j = q + (int)__umul64hi(v, (uint64_t)(ns - q));
      const int32_t tmp = S[q];
      S[q] = S[j];
      S[j] = tmp;
    }
    for (int q = 0; q < ns; ++q) mem[slot[q]] = S[q];
  }
}

// err bit 2 when a hyperedge repeats a member
__global__ void k_check_repeats(int64_t edges, const int64_t* __restrict__ off,
                                const int32_t* __restrict__ mem, int* __restrict__ err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < edges;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[e], n = off[e + 1] - b;
    for (int64_t x = 1; x < n; ++x)
      for (int64_t y = 0; y < x; ++y)
        if (mem[b + x] == mem[b + y]) atomicOr(err, 2);
  }
}

// `sweeps` rounds of pairwise reshuffles on the models of a union (members
// umem, offsets uoff, `edges` hyperedges); err bit 2: a repeated member.
void mcmc_rounds(const ModelInfo* dmi, int nt, int64_t edges, uint64_t seed, int sweeps,
                 const int64_t* uoff, int32_t* umem, int* err, cudaStream_t s) {
  if (edges > 0) {
    k_check_repeats<<<grid_n(edges), 256, 0, s>>>(edges, uoff, umem, err);
    HM_KCHECK();
  }
  if (edges < 2 || sweeps <= 0) return;
  DBuf<uint64_t> keys(edges, s), idx(edges, s);
  for (int r = 0; r < sweeps; ++r) {
    k_match_keys<<<grid_n(edges), 256, 0, s>>>(dmi, nt, edges, seed, (uint32_t)r, keys.p, idx.p);
    HM_KCHECK();
    radix_sort_u64(keys.p, idx.p, edges, 64, s);
    k_reshuffle<<<grid_n(edges), 256, 0, s>>>(dmi, nt, edges, seed, (uint32_t)r, idx.p, uoff,
                                               umem, err);
    HM_KCHECK();
  }
}

}  // namespace

void count_null_batch(int num_bases, const int32_t* d_members, const int64_t* d_offsets,
                      const int64_t* h_base_edges, const int32_t* h_num_nodes, int order,
                      int models_per_base, uint64_t seed, uint64_t* d_hists, cudaStream_t s,
                      int sweeps) {
  const ClassTables& T = class_tables(order);
  std::vector<int64_t> stub_at(num_bases + 1);  // first stub of every base (and the end)
  for (int b = 0; b <= num_bases; ++b)
    HM_CUDA(cudaMemcpyAsync(&stub_at[b], d_offsets + h_base_edges[b], sizeof(int64_t),
                            cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  int32_t block = 2;
  for (int b = 0; b < num_bases; ++b) {
    HM_CHECK(h_base_edges[b + 1] >= h_base_edges[b], HM_EINVAL, "base ranges must not decrease");
    HM_CHECK(stub_at[b + 1] >= stub_at[b], HM_EINVAL, "offsets must not decrease");
    HM_CHECK(h_num_nodes[b] >= 1, HM_EINVAL, "every base needs num_nodes >= 1");
    block = std::max(block, h_num_nodes[b]);
  }
  HM_CHECK((int64_t)block * GROUP < (1ll << 31), HM_EINVAL,
           "a base has too many nodes for a 64-model union (block * 64 must be < 2^31)");
  const int total_models = num_bases * models_per_base;
  HM_CUDA(cudaMemsetAsync(d_hists, 0, sizeof(uint64_t) * (size_t)total_models * T.ncls, s));
  for (int g0 = 0; g0 < total_models; g0 += GROUP) {
    const int nt = std::min(GROUP, total_models - g0);
    std::vector<ModelInfo> mi(nt);
    int64_t stubs = 0, edges = 0;
    for (int t = 0; t < nt; ++t) {
      const int gm = g0 + t, b = gm / models_per_base;
      mi[t].base_stub0 = stub_at[b];
      mi[t].stub0 = stubs;
      mi[t].base_edge0 = h_base_edges[b];
      mi[t].edge0 = edges;
      mi[t].node0 = t * block;
      mi[t].model_id = (uint32_t)gm;
      mi[t].n = h_num_nodes[b];
      stubs += stub_at[b + 1] - stub_at[b];
      edges += h_base_edges[b + 1] - h_base_edges[b];
    }
    HM_CHECK(edges < (1ll << 31) && stubs < (1ll << 31), HM_EINVAL,
             "a 64-model union exceeds 2^31 hyperedges or members");
    DBuf<ModelInfo> dmi(nt, s);
    HM_CUDA(cudaMemcpyAsync(dmi.p, mi.data(), nt * sizeof(ModelInfo), cudaMemcpyHostToDevice, s));
    DBuf<int32_t> umem(stubs, s);
    DBuf<int64_t> uoff(edges + 1, s);
    k_union_offsets<<<grid_n(edges + 1), 256, 0, s>>>(dmi.p, nt, edges, stubs, d_offsets, uoff.p);
    HM_KCHECK();
    {
      DBuf<int> err(1, s);
      HM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
      if (stubs && sweeps < 0) {  // stub shuffling
        DBuf<uint64_t> keys(stubs, s), src(stubs, s);
        k_stub_keys<<<grid_n(stubs), 256, 0, s>>>(dmi.p, nt, stubs, seed, keys.p, src.p);
        HM_KCHECK();
        radix_sort_u64(keys.p, src.p, stubs, 64, s);
        k_union_members<<<grid_n(stubs), 256, 0, s>>>(dmi.p, nt, stubs, src.p, d_members, umem.p,
                                                      err.p);
        HM_KCHECK();
      } else if (stubs) {  // configuration model by pairwise reshuffles
        k_union_copy<<<grid_n(stubs), 256, 0, s>>>(dmi.p, nt, stubs, d_members, umem.p, err.p);
        HM_KCHECK();
        mcmc_rounds(dmi.p, nt, edges, seed, sweeps, uoff.p, umem.p, err.p, s);
      }
      int herr = 0;
      unsigned timeouts = 0;
      HM_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof herr, cudaMemcpyDeviceToHost, s));
      wait_timeouts_async(&timeouts, s);
      HM_CUDA(cudaStreamSynchronize(s));
      wait_timeouts_check(timeouts, s);
      HM_CHECK(!(herr & 1), HM_EINVAL, "a member lies outside its base's [0, num_nodes)");
      HM_CHECK(!(herr & 2), HM_EINVAL,
               "the configuration model needs hyperedges without repeated members");
    }
    hm_graph* u = new hm_graph;
    try {
      build_graph(u, umem.p, uoff.p, edges, nt * block, order, s, block);
      umem.release();
      uoff.release();
      prepare_census(u, order, s);
      launch_census(u, order, (unsigned long long*)(d_hists + (size_t)g0 * T.ncls), s);
      HM_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      free_graph(u);
      throw;
    }
    free_graph(u);
  }
}

}  // namespace hm

extern "C" hm_status hm_count_null_batch(int num_bases, const int32_t* d_members,
                                         const int64_t* d_offsets, const int64_t* h_base_edges,
                                         const int32_t* h_num_nodes, int order,
                                         int models_per_base, uint64_t seed, uint64_t* d_hists,
                                         void* stream) {
  return hm::guarded([&] {
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(num_bases >= 1 && models_per_base >= 1, HM_EINVAL,
             "need at least one base and one model per base");
    HM_CHECK((int64_t)num_bases * models_per_base < (1ll << 31), HM_EINVAL, "too many models");
    HM_CHECK(d_offsets && h_base_edges && h_num_nodes && d_hists, HM_EINVAL, "NULL argument");
    hm::count_null_batch(num_bases, d_members, d_offsets, h_base_edges, h_num_nodes, order,
                         models_per_base, seed, d_hists, (cudaStream_t)stream, -1);
  });
}

extern "C" hm_status hm_count_null_batch_mcmc(int num_bases, const int32_t* d_members,
                                              const int64_t* d_offsets,
                                              const int64_t* h_base_edges,
                                              const int32_t* h_num_nodes, int order,
                                              int models_per_base, int sweeps, uint64_t seed,
                                              uint64_t* d_hists, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(num_bases >= 1 && models_per_base >= 1, HM_EINVAL,
             "need at least one base and one model per base");
    HM_CHECK((int64_t)num_bases * models_per_base < (1ll << 24), HM_EINVAL, "too many models");
    HM_CHECK(sweeps >= 0, HM_EINVAL, "sweeps must be >= 0");
    HM_CHECK(d_offsets && h_base_edges && h_num_nodes && d_hists, HM_EINVAL, "NULL argument");
    hm::count_null_batch(num_bases, d_members, d_offsets, h_base_edges, h_num_nodes, order,
                         models_per_base, seed, d_hists, (cudaStream_t)stream, sweeps);
  });
}

extern "C" hm_status hm_configuration_model(const int32_t* d_members, const int64_t* d_offsets,
                                            int64_t num_hyperedges, int32_t num_nodes,
                                            uint32_t model, int sweeps, uint64_t seed,
                                            int32_t* d_out, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(num_hyperedges >= 0 && num_hyperedges < (1ll << 31), HM_EINVAL,
             "num_hyperedges must be in [0, 2^31)");
    HM_CHECK(num_nodes >= 1 && sweeps >= 0 && model < (1u << 24), HM_EINVAL,
             "bad num_nodes, sweeps or model");
    HM_CHECK(num_hyperedges == 0 || (d_members && d_offsets && d_out), HM_EINVAL,
             "NULL argument");
    if (num_hyperedges == 0) return;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t stubs = 0;
    HM_CUDA(cudaMemcpyAsync(&stubs, d_offsets + num_hyperedges, sizeof stubs,
                            cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    HM_CHECK(stubs >= 0 && stubs < (1ll << 31), HM_EINVAL, "members must be < 2^31");
    hm::ModelInfo mi{};
    mi.base_stub0 = 0;
    mi.stub0 = 0;
    mi.base_edge0 = 0;
    mi.edge0 = 0;
    mi.node0 = 0;
    mi.model_id = model;
    mi.n = num_nodes;
    hm::DBuf<hm::ModelInfo> dmi(1, s);
    HM_CUDA(cudaMemcpyAsync(dmi.p, &mi, sizeof mi, cudaMemcpyHostToDevice, s));
    hm::DBuf<int> err(1, s);
    HM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    hm::k_union_copy<<<hm::grid_n(stubs), 256, 0, s>>>(dmi.p, 1, stubs, d_members, d_out, err.p);
    HM_KCHECK();
    hm::mcmc_rounds(dmi.p, 1, num_hyperedges, seed, sweeps, d_offsets, d_out, err.p, s);
    int herr = 0;
    unsigned timeouts = 0;
    HM_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof herr, cudaMemcpyDeviceToHost, s));
    hm::wait_timeouts_async(&timeouts, s);
    HM_CUDA(cudaStreamSynchronize(s));
    hm::wait_timeouts_check(timeouts, s);
    HM_CHECK(!(herr & 1), HM_EINVAL, "a member lies outside [0, num_nodes)");
    HM_CHECK(!(herr & 2), HM_EINVAL,
             "the configuration model needs hyperedges without repeated members");
  });
}
