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

}  // namespace

void count_null_batch(int num_bases, const int32_t* d_members, const int64_t* d_offsets,
                      const int64_t* h_base_edges, const int32_t* h_num_nodes, int order,
                      int models_per_base, uint64_t seed, uint64_t* d_hists, cudaStream_t s) {
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
    {
      DBuf<uint64_t> keys(stubs, s), src(stubs, s);
      DBuf<int> err(1, s);
      HM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
      if (stubs) {
        k_stub_keys<<<grid_n(stubs), 256, 0, s>>>(dmi.p, nt, stubs, seed, keys.p, src.p);
        HM_KCHECK();
        radix_sort_u64(keys.p, src.p, stubs, 64, s);
        k_union_members<<<grid_n(stubs), 256, 0, s>>>(dmi.p, nt, stubs, src.p, d_members, umem.p,
                                                      err.p);
        HM_KCHECK();
      }
      int herr = 0;
      unsigned timeouts = 0;
      HM_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof herr, cudaMemcpyDeviceToHost, s));
      wait_timeouts_async(&timeouts, s);
      HM_CUDA(cudaStreamSynchronize(s));
      wait_timeouts_check(timeouts, s);
      HM_CHECK(herr == 0, HM_EINVAL, "a member lies outside its base's [0, num_nodes)");
    }
    k_union_offsets<<<grid_n(edges + 1), 256, 0, s>>>(dmi.p, nt, edges, stubs, d_offsets, uoff.p);
    HM_KCHECK();
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
                         models_per_base, seed, d_hists, (cudaStream_t)stream);
  });
}
