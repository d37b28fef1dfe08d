// Per-hyperedge exact contributions and per-hyperedge features: the inputs
// of the learned sampling proposal.
//
// Contributions. Alg. 4 (Sec. 5) counts a k-node set only when the drawn
// hyperedge is one of the set's hyperedges of maximum cardinality, so the
// expected count a draw of hyperedge e adds to class c is n_{e,c} = the number
// of connected k-node sets of class c in which e is a maximum-cardinality
// hyperedge. This census variant walks the same canonical families as the
// exact census (each set once) and credits every maximum-cardinality
// hyperedge of each set: contrib[row(e) * ncls + c] += 1, rows ordered E_2,
// E_3, ..., E_k (ascending within each). Summed over e it gives
// countmax_c * T_c.
//
// Features (12 used of 16 slots, float32) of hyperedge e with members x_i, d2
// = pair degree, t3 = number of 3-hyperedges through a node, L = the number
// of sets a draw of e enumerates (see the sampler):
//   0: 1                      1: |e| / 4
//   2-4: log1p(min, mean, max of d2(x_i))
//   5-7: log1p(min, mean, max of t3(x_i))
//   8: log1p(number of pairs {x_i, x_j} that are hyperedges)
//   9: log1p(enumeration size of a draw of e at this order)
//   10: log1p(sum of d2(x_i))  11: log1p(sum of t3(x_i))  12-15: 0
#include "families.cuh"

namespace hm {
namespace {

using namespace fam;

// members (positions in the candidate) of every mask bit, k = 3 and k = 4
__constant__ int8_t c_sub3[4][4] = {{0, 1, -1, -1}, {0, 2, -1, -1}, {1, 2, -1, -1}, {0, 1, 2, -1}};
__constant__ int8_t c_sub4[11][4] = {{0, 1, -1, -1}, {0, 2, -1, -1}, {0, 3, -1, -1},
                                     {1, 2, -1, -1}, {1, 3, -1, -1}, {2, 3, -1, -1},
                                     {0, 1, 2, -1},  {0, 1, 3, -1},  {0, 2, 3, -1},
                                     {1, 2, 3, -1},  {0, 1, 2, 3}};

__device__ __forceinline__ int subset_size(int order, int b) {
  return order == 3 ? (b < 3 ? 2 : 3) : (b < 6 ? 2 : (b < 10 ? 3 : 4));
}

__device__ int64_t find_pair(const DevGraph& g, int32_t a, int32_t b) {
  const uint64_t key = pair_key(a, b);
  int64_t lo = 0, hi = g.m2;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (g.e2[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool tuple_less(const int4& x, const int4& y) {
  if (x.x != y.x) return x.x < y.x;
  if (x.y != y.y) return x.y < y.y;
  if (x.z != y.z) return x.z < y.z;
  return x.w < y.w;
}

__device__ int64_t find_tuple(const int4* e, int64_t m, int4 key) {
  int64_t lo = 0, hi = m;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (tuple_less(e[mid], key))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

template <class F>
__global__ void __launch_bounds__(256)
    k_contrib(const DevGraph g, const F fam, const uint64_t* __restrict__ ws, int64_t A,
              uint64_t total, int order, const uint8_t* __restrict__ lut, int ncls,
              unsigned int* __restrict__ contrib) {
  const int nsub = order == 3 ? 4 : 11;
  const int64_t base3 = g.m2, base4 = g.m2 + g.m3;
  const uint64_t nchunks = (total + CHUNK - 1) / CHUNK;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g0 = c * CHUNK, g1 = min(g0 + CHUNK, total);
    typename F::State st;
    int64_t a = 0;
    uint64_t r = 0, wa = 0;
    if (!F::kDirect) {
      a = anchor_of(ws, A, g0);
      r = g0 - ws[a];
      wa = ws[a + 1] - ws[a];
      fam.begin(g, a, r, st);
    }
    for (uint64_t gi = g0; gi < g1; ++gi) {
      uint32_t mask = 0;
      int32_t nd[4] = {0, 0, 0, 0};
      bool ok;
      if (F::kDirect) {
        ok = fam.item(g, (int64_t)gi, st, mask, nd);
      } else {
        if (r == wa) {
          do {
            ++a;
          } while (ws[a + 1] == ws[a]);
          r = 0;
          wa = ws[a + 1] - ws[a];
          fam.begin(g, a, 0, st);
        }
        ok = fam.item(g, a, st, mask, nd);
        ++r;
        fam.next(st);
      }
      if (!ok) continue;
      const uint8_t cls = lut[mask];
      if (cls == 0xFF) continue;
      int mc = 0;  // maxcard of the set
      for (int b = 0; b < nsub; ++b)
        if ((mask >> b) & 1u) mc = max(mc, subset_size(order, b));
      for (int b = 0; b < nsub; ++b) {
        if (!((mask >> b) & 1u)) continue;
        const int sz = subset_size(order, b);
        if (sz != mc) continue;
        const int8_t* sub = order == 3 ? c_sub3[b] : c_sub4[b];
        // the mask bit says the hyperedge exists, so the search finds it;
        // a miss (never expected) is skipped rather than written out of range
        int64_t row;
        if (sz == 2) {
          const int64_t i = find_pair(g, nd[sub[0]], nd[sub[1]]);
          if (i >= g.m2 || g.e2[i] != pair_key(nd[sub[0]], nd[sub[1]])) continue;
          row = i;
        } else {
          int32_t p = nd[sub[0]], q = nd[sub[1]], s = nd[sub[2]], t = sz == 4 ? nd[sub[3]] : -1;
          if (sz == 3) {
            sort3(p, q, s);
            const int4 key = make_int4(p, q, s, -1);
            const int64_t i = find_tuple(g.e3, g.m3, key);
            if (i >= g.m3 || tuple_less(g.e3[i], key) || tuple_less(key, g.e3[i])) continue;
            row = base3 + i;
          } else {
            sort4(p, q, s, t);
            const int4 key = make_int4(p, q, s, t);
            const int64_t i = find_tuple(g.e4, g.m4, key);
            if (i >= g.m4 || tuple_less(g.e4[i], key) || tuple_less(key, g.e4[i])) continue;
            row = base4 + i;
          }
        }
        atomicAdd(contrib + (size_t)row * ncls + cls, 1u);
      }
    }
  }
}

__device__ __forceinline__ float lg(float x) { return log1pf(x); }

// Number of 3-hyperedges containing both x and y: the shorter incidence list
// of the two, each triple checked for the other node.
__device__ int64_t common_triples(const DevGraph& g, int32_t x, int32_t y) {
  int64_t a0 = g.off3[x], a1 = g.off3[x + 1], b0 = g.off3[y], b1 = g.off3[y + 1];
  int32_t other = y;
  if (b1 - b0 < a1 - a0) {
    a0 = b0;
    a1 = b1;
    other = x;
  }
  int64_t c = 0;
  for (int64_t i = a0; i < a1; ++i) {
    const int4 t = g.e3[g.inc3[i]];
    c += (t.x == other || t.y == other || t.z == other) ? 1 : 0;
  }
  return c;
}

__global__ void k_features(const DevGraph g, int order, int64_t rows, float* __restrict__ out) {
  const int64_t m2 = g.m2, m3 = g.m3;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t x[4];
    int s;
    if (r < m2) {
      x[0] = (int32_t)(g.e2[r] >> 32);
      x[1] = (int32_t)(g.e2[r] & 0xFFFFFFFFull);
      s = 2;
    } else if (r < m2 + m3) {
      const int4 e = g.e3[r - m2];
      x[0] = e.x;
      x[1] = e.y;
      x[2] = e.z;
      s = 3;
    } else {
      const int4 e = g.e4[r - m2 - m3];
      x[0] = e.x;
      x[1] = e.y;
      x[2] = e.z;
      x[3] = e.w;
      s = 4;
    }
    float dmin = 3.4e38f, dmax = 0.f, dsum = 0.f, tmin = 3.4e38f, tmax = 0.f, tsum = 0.f;
    for (int i = 0; i < s; ++i) {
      const float d = (float)(g.off2[x[i] + 1] - g.off2[x[i]]);
      const float t = (float)(g.off3[x[i] + 1] - g.off3[x[i]]);
      dmin = fminf(dmin, d);
      dmax = fmaxf(dmax, d);
      dsum += d;
      tmin = fminf(tmin, t);
      tmax = fmaxf(tmax, t);
      tsum += t;
    }
    int npairs = 0;
    int64_t shared = 0;  // sum over member pairs of the 3-hyperedges through both
    for (int i = 0; i < s; ++i)
      for (int j = i + 1; j < s; ++j) {
        npairs += has_pair(g, x[i], x[j]) ? 1 : 0;
        if (m3) shared += common_triples(g, x[i], x[j]);
      }
    // 3-hyperedges inside a 4-hyperedge; then the 3-hyperedges other than e
    // sharing at least two nodes with e (a sub-triple of a quad is met at
    // three of its pairs, e itself at its three pairs)
    int nsub = 0;
    if (s == 4 && m3) {
      nsub = (has_triple(g, x[0], x[1], x[2]) ? 1 : 0) + (has_triple(g, x[0], x[1], x[3]) ? 1 : 0) +
             (has_triple(g, x[0], x[2], x[3]) ? 1 : 0) + (has_triple(g, x[1], x[2], x[3]) ? 1 : 0);
    }
    const int64_t overlap = s == 2 ? shared : s == 3 ? shared - 3 : shared - 2 * nsub;
    double work = 1.0;
    if (s == 2 && order > 2) {
      const double l = (double)(dsum - 2.f);
      work = order == 3 ? l : l * (l - 1.0) * 0.5;
    } else if (s == 3 && order == 4) {
      work = (double)(dsum + tsum);
    }
    float* f = out + r * 16;
    f[0] = 1.f;
    f[1] = (float)s * 0.25f;
    f[2] = lg(dmin);
    f[3] = lg(dsum / (float)s);
    f[4] = lg(dmax);
    f[5] = lg(tmin);
    f[6] = lg(tsum / (float)s);
    f[7] = lg(tmax);
    f[8] = lg((float)npairs);
    f[9] = lg((float)work);
    f[10] = lg(dsum);
    f[11] = lg(tsum);
    f[12] = lg((float)overlap);
    f[13] = lg((float)nsub);
    f[14] = f[15] = 0.f;
  }
}

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

template <class F>
void launch_contrib(const hm_graph* g, const F& f, const hm_graph::Space* sp, uint64_t total,
                    int order, const uint8_t* lut, unsigned int* contrib, cudaStream_t s) {
  if (total == 0) return;
  const uint64_t chunks = (total + CHUNK - 1) / CHUNK;
  int64_t blocks = (int64_t)((chunks + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_contrib<F><<<(unsigned)blocks, 256, 0, s>>>(g->view(), f, sp ? sp->ws : nullptr,
                                               sp ? sp->anchors : 0, total, order, lut,
                                               class_tables(order).ncls, contrib);
  HM_KCHECK();
}

}  // namespace

void contributions(hm_graph* g, int order, uint32_t* d_contrib, cudaStream_t s) {
  prepare_census(g, order, s);
  int64_t rows = 0;
  for (int k = 2; k <= order; ++k) rows += g->counts[k];
  const int ncls = class_tables(order).ncls;
  HM_CUDA(cudaMemsetAsync(d_contrib, 0, (size_t)rows * ncls * sizeof(uint32_t), s));
  const uint8_t* lut = device_lut(order);
  if (order == 3) {
    launch_contrib(g, FamT3{}, nullptr, (uint64_t)g->counts[3], 3, lut, d_contrib, s);
    launch_contrib(g, FamW{}, &g->W, g->W.total, 3, lut, d_contrib, s);
  } else {
    launch_contrib(g, FamQ{}, nullptr, (uint64_t)g->counts[4], 4, lut, d_contrib, s);
    launch_contrib(g, FamTX{}, &g->TX, g->TX.total, 4, lut, d_contrib, s);
    launch_contrib(g, FamS{}, &g->S, g->S.total, 4, lut, d_contrib, s);
    launch_contrib(g, FamP{}, &g->P, g->P.total, 4, lut, d_contrib, s);
  }
}

void features(const hm_graph* g, int order, float* d_feat, cudaStream_t s) {
  int64_t rows = 0;
  for (int k = 2; k <= order; ++k) rows += g->counts[k];
  if (rows == 0) return;
  k_features<<<grid_n(rows), 256, 0, s>>>(g->view(), order, rows, d_feat);
  HM_KCHECK();
}

}  // namespace hm

extern "C" hm_status hm_contributions(hm_graph* g, int order, uint32_t* d_contrib, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g != nullptr, HM_EINVAL, "NULL graph");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= g->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    HM_CHECK(g->block == 0, HM_EUNSUPPORTED, "not available for a union of graphs");
    hm::contributions(g, order, d_contrib, (cudaStream_t)stream);
  });
}

extern "C" hm_status hm_features(hm_graph* g, int order, float* d_feat, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g != nullptr, HM_EINVAL, "NULL graph");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= g->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    hm::features(g, order, d_feat, (cudaStream_t)stream);
  });
}
