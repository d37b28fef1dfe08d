// The baseline of Sec. 4.1 (Alg. 1) on the GPU, for the comparison of
// Table 2: project the hypergraph onto a graph (nodes joined when they share
// a hyperedge of any size), enumerate the connected k-node subgraphs of the
// projection, fill each in against the hypergraph (Sec. 4.3) and count the
// connected ones by class. The projection is built as a graph of its own:
// every pair of every hyperedge becomes a 2-member hyperedge of a second
// hm_graph, whose ingest deduplicates the pairs and lays out their rows and
// hash set; its W / S / P index spaces are the baseline's candidates
// (census.cu, launch_baseline, with the families of baseline.cuh).
#include "hm_internal.cuh"

namespace hm {

uint64_t launch_baseline(hm_graph* p, const hm_graph* h, int order, unsigned long long* hist,
                         cudaStream_t s);

namespace {

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

// pairs per hyperedge: C(size, 2)
__global__ void k_pair_counts(const int64_t* __restrict__ off, int64_t m, uint64_t* __restrict__ cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z = (uint64_t)(off[e + 1] - off[e]);
    cnt[e] = z * (z - (z > 0 ? 1 : 0)) / 2;
  }
}

// every pair (positions a < b) of hyperedge e as a 2-member hyperedge, from
// slot pos[e] on; the offsets of the 2-member hyperedges are 2 i
__global__ void k_pair_emit(const int32_t* __restrict__ mem, const int64_t* __restrict__ off,
                            int64_t m, const uint64_t* __restrict__ pos,
                            int32_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[e], z = off[e + 1] - b;
    uint64_t q = pos[e];
    for (int64_t i = 0; i < z; ++i)
      for (int64_t j = i + 1; j < z; ++j, ++q) {
        out[2 * q] = mem[b + i];
        out[2 * q + 1] = mem[b + j];
      }
  }
}

__global__ void k_even_offsets(int64_t n, int64_t* __restrict__ off) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x)
    off[i] = 2 * i;
}

}  // namespace

void count_baseline(const int32_t* d_members, const int64_t* d_offsets, int64_t m, int32_t n,
                    int order, uint64_t* d_hist, uint64_t* info, cudaStream_t s) {
  hm_graph* h = new hm_graph;
  hm_graph* p = nullptr;
  uint64_t cand = 0;
  try {
    build_graph(h, d_members, d_offsets, m, n, order, s);
    uint64_t np = 0;
    {
      DBuf<uint64_t> cnt(m + 1, s), pos(m + 1, s);
      if (m) {
        k_pair_counts<<<grid_n(m), 256, 0, s>>>(d_offsets, m, cnt.p);
        HM_KCHECK();
      }
      scan_exclusive_u64(cnt.p, pos.p, m, s);
      HM_CUDA(cudaMemcpyAsync(&np, pos.p + m, sizeof np, cudaMemcpyDeviceToHost, s));
      HM_CUDA(cudaStreamSynchronize(s));
      HM_CHECK(np < (1ull << 31), HM_EINVAL, "the projection has 2^31 pairs or more");
      DBuf<int32_t> pmem(2 * np, s);
      DBuf<int64_t> poff(np + 1, s);
      if (np) {
        k_pair_emit<<<grid_n(m), 256, 0, s>>>(d_members, d_offsets, m, pos.p, pmem.p);
        HM_KCHECK();
      }
      k_even_offsets<<<grid_n((int64_t)np + 1), 256, 0, s>>>((int64_t)np, poff.p);
      HM_KCHECK();
      p = new hm_graph;
      build_graph(p, pmem.p, poff.p, (int64_t)np, n, order, s);
    }
    HM_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(uint64_t) * class_tables(order).ncls, s));
    cand = launch_baseline(p, h, order, (unsigned long long*)d_hist, s);
    HM_CUDA(cudaStreamSynchronize(s));
    info[0] = cand;
    info[1] = (uint64_t)p->counts[2];
  } catch (...) {
    free_graph(h);
    if (p) free_graph(p);
    throw;
  }
  free_graph(h);
  free_graph(p);
}

}  // namespace hm

extern "C" hm_status hm_count_exact_baseline(const int32_t* d_members, const int64_t* d_offsets,
                                             int64_t num_hyperedges, int32_t num_nodes, int order,
                                             uint64_t* d_hist, uint64_t* h_info,
                                             void* stream) {
  return hm::guarded([&] {
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(num_nodes >= 1, HM_EINVAL, "num_nodes must be >= 1");
    HM_CHECK(num_hyperedges >= 0 && num_hyperedges < (1ll << 31), HM_EINVAL,
             "num_hyperedges must be in [0, 2^31)");
    HM_CHECK(d_hist && (num_hyperedges == 0 || (d_members && d_offsets)), HM_EINVAL,
             "NULL argument");
    uint64_t info[2] = {0, 0};
    hm::count_baseline(d_members, d_offsets, num_hyperedges, num_nodes, order, d_hist, info,
                       (cudaStream_t)stream);
    if (h_info) {
      h_info[0] = info[0];
      h_info[1] = info[1];
    }
  });
}
