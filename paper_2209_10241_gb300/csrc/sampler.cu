// Stratified hyperedge-sampling estimator (Alg. 4, Sec. 5).
//
// For every stratum s (hyperedge size 2..k) S_s hyperedges are drawn with
// replacement: draw t uses Philox4x32-10 (Salmon et al., SC'11) with key =
// seed and counter = (t lo, t hi, s, "SAMP"), and the 64-bit value
// (r0 << 32) | r1 picks mulhi64(value, |E_s|) -- or, with proposal weights q,
// the inverse CDF of q at mulhi64(value, Q_s). For each draw every k-node set
// V' containing the drawn hyperedge e with H[V'] connected and no hyperedge
// larger than e is enumerated and counted by class (the max-cardinality rule
// of Sec. 5). Counts accumulate as integers (weighted draws add
// floor(2^63 / q_e) into 128-bit sums), so the result is independent of the
// order of the atomic updates; the correction factor of Alg. 4 is applied in
// IEEE double in a fixed order.
//
// Per-sample enumeration (each set once per draw):
//   s = k        the drawn hyperedge itself (families T3 / Q with a map)
//   k=4, s=3     nodes d joined to e by a hyperedge h of size 2 or 3 through
//                x in e: kept when x = min(h ∩ e), h is the smallest hyperedge
//                containing d and there is no 4-hyperedge (TX without the
//                anchor-minimality test)
//   s=2, e={a,b} L1 = N2(a)\{b} followed by N2(b)\{a}, entries of the second
//                part also adjacent to a dropped. k=3: {a,b,c}, c in L1.
//                k=4: {c,d} from two L1 entries, or c in L1 and d a
//                pair-neighbour of c outside L1 ∪ e. Sets holding a 3- or
//                4-hyperedge are dropped (max-cardinality rule).
#include <cmath>
#include <cstdlib>
#include <functional>
#include <mutex>

#include "families.cuh"

namespace hm {
namespace {

using namespace fam;

constexpr uint32_t TAG_SAMPLE = 0x53414D50u;  // "SAMP"
constexpr int64_t SAMPLE_BATCH = 1 << 20;
constexpr int SAMPLE_THREADS = 256;

__device__ __forceinline__ int32_t deg2(const DevGraph& g, int32_t v) {
  return (int32_t)(g.off2[v + 1] - g.off2[v]);
}

// entry i of L1 = N2(a)\{b} ++ N2(b)\{a}
struct PairList {
  int32_t a, b;
  int64_t ao, bo;
  uint32_t la, pa, pb;
};

__device__ __forceinline__ PairList pair_list(const DevGraph& g, int64_t p) {
  PairList L;
  const uint64_t ab = g.e2[p];
  L.a = (int32_t)(ab >> 32);
  L.b = (int32_t)(ab & 0xFFFFFFFFull);
  L.ao = g.off2[L.a];
  L.bo = g.off2[L.b];
  L.la = (uint32_t)(g.off2[L.a + 1] - L.ao - 1);
  const int2 pp = g.pairpos[p];
  L.pa = (uint32_t)pp.x;
  L.pb = (uint32_t)pp.y;
  return L;
}

__device__ __forceinline__ int32_t list_elem(const DevGraph& g, const PairList& L, uint32_t i) {
  if (i < L.la) return g.adj2[L.ao + i + (i >= L.pa ? 1 : 0)];
  const uint32_t j = i - L.la;
  return g.adj2[L.bo + j + (j >= L.pb ? 1 : 0)];
}

struct DrawArgs {
  uint64_t seed;
  int s, order;
  uint64_t t0;
  int64_t count;
  int64_t len;
  const uint64_t* P;  // exclusive prefix of q over E_s (len + 1), NULL = uniform
  const uint32_t* q;  // weights of E_s
};

// Draws of one batch, the drawn hyperedge, its weight and its enumeration size.
__global__ void k_draw(const DevGraph g, const DrawArgs d, int64_t* __restrict__ sidx,
                       uint64_t* __restrict__ wt, uint64_t* __restrict__ work,
                       uint64_t* __restrict__ lsize) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t t = d.t0 + (uint64_t)i;
    uint32_t c[4] = {(uint32_t)t, (uint32_t)(t >> 32), (uint32_t)d.s, TAG_SAMPLE};
    philox4x32_10(c, (uint32_t)d.seed, (uint32_t)(d.seed >> 32));
    const uint64_t v = ((uint64_t)c[0] << 32) | c[1];
    int64_t idx;
    if (!d.P) {
      idx = (int64_t)__umul64hi(v, (uint64_t)d.len);
    } else {
      const uint64_t r = __umul64hi(v, d.P[d.len]);
      int64_t lo = 0, hi = d.len;  // last idx with P[idx] <= r
      while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (d.P[mid] <= r)
          lo = mid;
        else
          hi = mid;
      }
      idx = lo;
    }
    sidx[i] = idx;
    wt[i] = d.P ? (1ull << 63) / (uint64_t)d.q[idx] : 1ull;
    uint64_t w = 1, l = 0;
    if (d.s == 2 && d.s < d.order) {
      const uint64_t ab = g.e2[idx];
      const int32_t a = (int32_t)(ab >> 32), b = (int32_t)(ab & 0xFFFFFFFFull);
      l = (uint64_t)(deg2(g, a) - 1) + (uint64_t)(deg2(g, b) - 1);
      w = d.order == 3 ? l : choose2(l);
    } else if (d.s == 3 && d.order == 4) {
      const int4 e = g.e3[idx];
      const int32_t xs[3] = {e.x, e.y, e.z};
      w = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j)
        w += (uint64_t)deg2(g, xs[j]) + (uint64_t)(g.off3[xs[j] + 1] - g.off3[xs[j]]);
    }
    work[i] = w;
    if (lsize) lsize[i] = l;
  }
}

// L1 entries of every drawn pair (order 4), with the pair-degree of each
// valid entry as its enumeration size.
__global__ void k_elements(const DevGraph g, const int64_t* __restrict__ sidx, int64_t count,
                           const uint64_t* __restrict__ eoff, int2* __restrict__ elems,
                           uint64_t* __restrict__ ework) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const PairList L = pair_list(g, sidx[i]);
    const uint64_t base = eoff[i], n = eoff[i + 1] - base;
    for (uint64_t j = 0; j < n; ++j) {
      const int32_t c = list_elem(g, L, (uint32_t)j);
      const bool valid = j < L.la || !has_pair(g, L.a, c);
      elems[base + j] = make_int2((int32_t)i, valid ? c : -1);
      ework[base + j] = valid ? (uint64_t)deg2(g, c) : 0ull;
    }
  }
}

// k=3, s=2: {a, b, c}, c in L1
struct SamP3 {
  static constexpr const char* kName = "sample_P3";
  static constexpr bool kDirect = false;
  const int64_t* map;
  struct State {
    PairList L;
    uint32_t i;
  };
  __device__ void begin(const DevGraph& g, int64_t a, uint64_t r, State& s) const {
    s.L = pair_list(g, map[a]);
    s.i = (uint32_t)r;
  }
  __device__ void next(State& s) const { ++s.i; }
  __device__ bool item(const DevGraph& g, int64_t, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const PairList& L = s.L;
    const int32_t c = list_elem(g, L, s.i);
    nd[0] = L.a;
    nd[1] = L.b;
    nd[2] = c;
    const bool first = s.i < L.la;
    if (!first && has_pair(g, L.a, c)) return false;  // already listed from a
    if (has_triple(g, L.a, L.b, c)) return false;     // larger hyperedge than e
    const bool ac = first, bc = first ? has_pair(g, L.b, c) : true;
    mask = 1u | (ac ? 2u : 0u) | (bc ? 4u : 0u);  // a=0, b=1, c=2
    return true;
  }
};

// k=4, s=2: {a, b, c, d} with c, d two entries of L1
struct SamPA {
  static constexpr const char* kName = "sample_PA";
  static constexpr bool kDirect = false;
  const int64_t* map;
  struct State {
    PairList L;
    uint32_t i, j;
  };
  __device__ void begin(const DevGraph& g, int64_t a, uint64_t r, State& s) const {
    s.L = pair_list(g, map[a]);
    unrank2(r, s.i, s.j);
  }
  __device__ void next(State& s) const {
    if (++s.i == s.j) {
      s.i = 0;
      ++s.j;
    }
  }
  __device__ bool item(const DevGraph& g, int64_t, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const PairList& L = s.L;
    const int32_t a = L.a, b = L.b;
    const int32_t c = list_elem(g, L, s.i), d = list_elem(g, L, s.j);
    nd[0] = a;
    nd[1] = b;
    nd[2] = c;
    nd[3] = d;
    const bool cfirst = s.i < L.la, dfirst = s.j < L.la;
    const bool ac = cfirst ? true : has_pair(g, a, c);
    const bool ad = dfirst ? true : has_pair(g, a, d);
    if ((!cfirst && ac) || (!dfirst && ad)) return false;  // already listed from a
    const bool bc = cfirst ? has_pair(g, b, c) : true;
    const bool bd = dfirst ? has_pair(g, b, d) : true;
    const bool cd = has_pair(g, c, d);
    if (has_triple(g, a, b, c) || has_triple(g, a, b, d) || has_triple(g, a, c, d) ||
        has_triple(g, b, c, d) || has_quad(g, a, b, c, d))
      return false;
    mask = 1u | (ac ? 2u : 0u) | (ad ? 4u : 0u) | (bc ? 8u : 0u) | (bd ? 16u : 0u) |
           (cd ? 32u : 0u);  // a=0, b=1, c=2, d=3
    return true;
  }
};

// k=4, s=2: {a, b, c, d} with c in L1 and d a pair-neighbour of c outside L1 ∪ e
struct SamPB {
  static constexpr const char* kName = "sample_PB";
  static constexpr bool kDirect = false;
  const int64_t* map;
  const int2* elems;
  struct State {
    int32_t a, b, c;
    int64_t co;
    uint64_t r;
  };
  __device__ void begin(const DevGraph& g, int64_t j, uint64_t r, State& s) const {
    const int2 el = elems[j];
    const uint64_t ab = g.e2[map[el.x]];
    s.a = (int32_t)(ab >> 32);
    s.b = (int32_t)(ab & 0xFFFFFFFFull);
    s.c = el.y;
    s.co = g.off2[el.y];
    s.r = r;
  }
  __device__ void next(State& s) const { ++s.r; }
  __device__ bool item(const DevGraph& g, int64_t, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int32_t a = s.a, b = s.b, c = s.c;
    const int32_t d = g.adj2[s.co + s.r];
    nd[0] = a;
    nd[1] = b;
    nd[2] = c;
    nd[3] = d;
    if (d == a || d == b || has_pair(g, a, d) || has_pair(g, b, d)) return false;
    if (has_triple(g, a, b, c) || has_triple(g, a, b, d) || has_triple(g, a, c, d) ||
        has_triple(g, b, c, d) || has_quad(g, a, b, c, d))
      return false;
    const bool ac = has_pair(g, a, c), bc = has_pair(g, b, c);
    mask = 1u | (ac ? 2u : 0u) | (bc ? 8u : 0u) | 32u;  // pairs ab, (ac), (bc), cd
    return true;
  }
};

template <class F>
__device__ __forceinline__ int64_t sample_of(const F&, int64_t a) {
  return a;
}
__device__ __forceinline__ int64_t sample_of(const SamPB& f, int64_t a) { return f.elems[a].x; }

// Same index-space walk as the census driver; each counted set adds the
// weight of its draw (1 for uniform draws) into (lo, hi) 128-bit class sums.
template <class F, bool kWeighted>
__global__ void __launch_bounds__(SAMPLE_THREADS)
    k_sample(const DevGraph g, const F fam, const uint64_t* __restrict__ ws, int64_t A,
             uint64_t total, const uint64_t* __restrict__ wt, const uint8_t* __restrict__ lut_g,
             int nmask, int ncls, unsigned long long* __restrict__ raw) {
  __shared__ unsigned long long blo[176], bhi[176];
  __shared__ __align__(16) uint8_t lut[2048];
  load_lut(lut, lut_g, nmask);
  for (int i = threadIdx.x; i < ncls; i += blockDim.x) blo[i] = bhi[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t nchunks = (total + CHUNK - 1) / CHUNK;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t cb = warp * 32; cb < nchunks; cb += nwarps * 32) {
    const uint64_t g0 = (cb + lane) * CHUNK;
    const uint64_t g1 = min(g0 + CHUNK, total);
    typename F::State st;
    int64_t a = 0;
    uint64_t r = 0, wa = 0;
    if (!F::kDirect && g0 < total) {
      a = anchor_of(ws, A, g0);
      r = g0 - ws[a];
      wa = ws[a + 1] - ws[a];
      fam.begin(g, a, r, st);
    }
    for (int it = 0; it < CHUNK; ++it) {
      const uint64_t gi = g0 + it;
      int cls = -1;
      int64_t anchor = 0;
      if (gi < g1) {
        uint32_t mask = 0;
        int32_t nd[4];
        bool ok;
        if (F::kDirect) {
          anchor = (int64_t)gi;
          ok = fam.item(g, anchor, st, mask, nd);
        } else {
          if (r == wa) {
            do {
              ++a;
            } while (ws[a + 1] == ws[a]);
            r = 0;
            wa = ws[a + 1] - ws[a];
            fam.begin(g, a, 0, st);
          }
          anchor = a;
          ok = fam.item(g, a, st, mask, nd);
          ++r;
          fam.next(st);
        }
        if (ok) {
          const uint8_t c = lut[mask];
          cls = c == 0xFF ? -1 : (int)c;
        }
      }
      if (!kWeighted) {
        const unsigned peers = __match_any_sync(0xffffffffu, cls);
        if (cls >= 0 && lane == __ffs(peers) - 1)
          atomicAdd(&blo[cls], (unsigned long long)__popc(peers));
      } else {
        // lanes that counted the same class for the same sample add one
        // product weight x count (128-bit, exact in any order)
        const uint64_t sid = cls >= 0 ? (uint64_t)sample_of(fam, anchor) : ~0ull;
        const unsigned long long key = (sid << 8) | (uint64_t)(uint8_t)cls;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (cls >= 0 && lane == __ffs(peers) - 1) {
          const unsigned long long w = wt[sid], c = (unsigned long long)__popc(peers);
          const unsigned long long lo = w * c, hi = __umul64hi(w, c);
          const unsigned long long old = atomicAdd(&blo[cls], lo);
          const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
          if (hi + carry) atomicAdd(&bhi[cls], hi + carry);
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ncls; i += blockDim.x) {
    const unsigned long long lo = blo[i], hi = bhi[i];
    if (lo | hi) {
      const unsigned long long old = atomicAdd(&raw[2 * i], lo);
      const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
      if (hi + carry) atomicAdd(&raw[2 * i + 1], hi + carry);
    }
  }
}

struct EstArgs {
  double S[5];
  uint64_t E[5];  // |E_s|
  int weighted;
  int ncls;
  int8_t maxcard[176];
  int8_t countmax[176];
};

// Correction of Alg. 4: (n_c |E_m|) / (S_m countmax_c), or with weights
// (A_c 2^-63 Q_m) / (S_m countmax_c); round-to-nearest at every step, no
// contraction, in this order.
__global__ void k_estimate(const EstArgs e, const uint64_t* __restrict__ Q,
                           const unsigned long long* __restrict__ raw, double* __restrict__ est) {
  for (int c = threadIdx.x; c < e.ncls; c += blockDim.x) {
    const int m = e.maxcard[c];
    if (e.S[m] == 0.0 || e.E[m] == 0) {
      est[c] = 0.0;
      continue;
    }
    double a;
    if (e.weighted) {
      a = __dadd_rn(__dmul_rn(__ull2double_rn(raw[2 * c + 1]), 18446744073709551616.0),
                    __ull2double_rn(raw[2 * c]));
      a = __dmul_rn(a, 0x1p-63);
    } else {
      a = __ull2double_rn(raw[2 * c]);
    }
    const double num = __dmul_rn(a, __ull2double_rn(Q[m]));
    const double den = __dmul_rn(e.S[m], (double)e.countmax[c]);
    est[c] = __ddiv_rn(num, den);
  }
}

__global__ void k_widen(const uint32_t* __restrict__ q, int64_t n, uint64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = q[i];
}

__global__ void k_bad_weight(const uint32_t* __restrict__ q, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (q[i] == 0) atomicOr(flag, 1);
}

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

int sample_blocks(const void* kernel, uint64_t total) {
  int dev = 0, sms = 0, per_sm = 0;
  HM_CUDA(cudaGetDevice(&dev));
  HM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, SAMPLE_THREADS, 0));
  if (per_sm < 1) per_sm = 1;
  const uint64_t need = ((total + CHUNK - 1) / CHUNK + SAMPLE_THREADS - 1) / SAMPLE_THREADS;
  uint64_t b = (uint64_t)sms * per_sm;
  if (need < b) b = need;
  return (int)(b < 1 ? 1 : b);
}

template <class F>
void launch_sample(const hm_graph* g, const F& f, const uint64_t* ws, int64_t A, uint64_t total,
                   const uint64_t* wt, bool weighted, int order, unsigned long long* raw,
                   cudaStream_t s) {
  if (total == 0) return;
  const ClassTables& T = class_tables(order);
  const uint8_t* lut = device_lut(order);
  cudaEvent_t ev = nullptr;
  const bool tr = trace_on(F::kName);
  if (tr) trace_begin(s, &ev);
  if (weighted) {
    k_sample<F, true><<<sample_blocks((const void*)k_sample<F, true>, total), SAMPLE_THREADS, 0,
                        s>>>(g->view(), f, ws, A, total, wt, lut, (int)T.lut.size(), T.ncls, raw);
  } else {
    k_sample<F, false><<<sample_blocks((const void*)k_sample<F, false>, total), SAMPLE_THREADS, 0,
                         s>>>(g->view(), f, ws, A, total, wt, lut, (int)T.lut.size(), T.ncls, raw);
  }
  HM_KCHECK();
  if (tr) trace_end(F::kName, s, ev);
}

uint64_t scan_total(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s) {
  scan_exclusive_u64(in, out, n, s);
  uint64_t tot = 0;
  HM_CUDA(cudaMemcpyAsync(&tot, out + n, sizeof tot, cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  return tot;
}

// ---------------------------------------------------------------- order 4, pair stratum by types
// For a drawn pair e = {a, b} at order 4, the sets Alg. 4 counts are the
// 4-node sets V' containing e whose induced sub-hypergraph is connected and
// holds no 3- or 4-hyperedge, i.e. the connected induced 4-node subgraphs of
// the pair graph that contain the edge ab, less those holding a larger
// hyperedge. With N_a = N2(a)\{b}, N_b = N2(b)\{a}, T = N_a ∩ N_b, A = N_a \ T
// and B = N_b \ T (sizes sa, sb, t), every such set {a, b, c, d} is either
//  (1) c, d both in A ∪ B ∪ T: its pattern depends only on the types of c
//      and d and on whether cd is a pair -- C(sa+sb+t, 2) sets, counted from
//      sa, sb, t plus one correction per pair inside A ∪ B ∪ T;
//  (2) c in A ∪ B ∪ T and d a pair neighbour of c outside A ∪ B ∪ T ∪ {a, b}:
//      a path (c in A or B) or a paw (c in T).
// So instead of testing all C(sa+sb+t, 2) + Σ deg(c) candidates, each draw
// costs one scan of the pair neighbours of every c (two membership probes per
// neighbour); the sets that hold a 3- or 4-hyperedge all contain a 3- or
// 4-hyperedge through a or b, so they are found from those lists and
// subtracted (each once, by a fixed precedence among the hyperedges it
// holds). Sums are 128-bit two's complement (a subtraction adds the negated
// product), exact in any order, and equal the per-candidate enumeration's.

enum { PP_STAR = 0, PP_PATH = 1, PP_PAW = 2, PP_C4 = 3, PP_DIAMOND = 4, PP_K4 = 5 };
enum { TY_A = 0, TY_B = 1, TY_T = 2 };
// one labelled pair mask of each pairs-only pattern (a = 0, b = 1, c = 2, d = 3;
// bits ab, ac, ad, bc, bd, cd): star at a, path c-a-b-d, paw, 4-cycle, diamond, 4-clique
constexpr int kPatternMask[6] = {7, 19, 39, 51, 31, 63};

struct PairClasses {
  int cls[6];
};

// Adds (or subtracts) w * c to the 128-bit class sum (blo, bhi)[cls].
__device__ __forceinline__ void bins_add(unsigned long long* blo, unsigned long long* bhi, int cls,
                                         uint64_t w, uint64_t c, bool neg) {
  if (c == 0) return;
  unsigned long long lo = w * c, hi = __umul64hi(w, c);
  if (neg) {
    hi = ~hi + (lo == 0 ? 1ull : 0ull);
    lo = 0ull - lo;
  }
  const unsigned long long old = atomicAdd(&blo[cls], lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(&bhi[cls], hi + carry);
}

__device__ __forceinline__ void bins_flush(const unsigned long long* blo,
                                           const unsigned long long* bhi, int ncls,
                                           unsigned long long* raw) {
  for (int i = threadIdx.x; i < ncls; i += blockDim.x) {
    const unsigned long long lo = blo[i], hi = bhi[i];
    if (lo | hi) {
      const unsigned long long old = atomicAdd(&raw[2 * i], lo);
      const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
      if (hi + carry) atomicAdd(&raw[2 * i + 1], hi + carry);
    }
  }
}

// Lanes whose update has the same key add one w x count (uniform draws: the
// key is the class and sign; weighted: also the draw).
template <bool kWeighted>
__device__ __forceinline__ void bins_vote(unsigned long long* blo, unsigned long long* bhi, int cls,
                                          bool neg, uint32_t draw, const uint64_t* wt) {
  const int lane = threadIdx.x & 31;
  const unsigned long long key =
      cls < 0 ? ~0ull
              : ((kWeighted ? (unsigned long long)draw << 9 : 0ull) |
                 ((unsigned long long)neg << 8) | (unsigned long long)cls);
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (cls >= 0 && lane == __ffs(peers) - 1)
    bins_add(blo, bhi, cls, kWeighted ? wt[draw] : 1ull, (uint64_t)__popc(peers), neg);
}

// Membership tests that read the node signatures first (graphs without
// bitmaps): a clear signature bit proves the pair / 3-hyperedge absent
// without a probe.
__device__ __forceinline__ bool pair_s(const DevGraph& g, int32_t a, int32_t x) {
  return (!g.sig || (g.sig[a] & sig_bit(x))) && has_pair(g, a, x);
}
__device__ __forceinline__ bool triple_s(const DevGraph& g, int32_t a, int32_t b, int32_t x) {
  if (g.sig) {
    const uint64_t s = g.sig[(int64_t)g.n + a];
    if (!(s & sig_bit(b)) || !(s & sig_bit(x))) return false;
  }
  return has_triple(g, a, b, x);
}

// Pair mask of {a, b, x, y} (ab present) and whether its pairs connect it.
__device__ __forceinline__ bool pair_pattern(const DevGraph& g, int32_t a, int32_t b, int32_t x,
                                             int32_t y, uint32_t& mask) {
  const bool ax = pair_s(g, a, x), ay = pair_s(g, a, y), bx = pair_s(g, b, x),
             by = pair_s(g, b, y), xy = pair_s(g, x, y);
  mask = 1u | (ax ? 2u : 0u) | (ay ? 4u : 0u) | (bx ? 8u : 0u) | (by ? 16u : 0u) | (xy ? 32u : 0u);
  const bool xa = ax || bx, ya = ay || by;  // x / y adjacent to {a, b}
  return (xa || (xy && ya)) && (ya || (xy && xa));
}

// Elements of the drawn pairs' lists L1 = N2(a)\{b} ++ N2(b)\{a} (the second
// part without N2(a)): per element (draw | type << 30, node or -1), its pair
// degree (the neighbours stage (2) scans), and per draw the size t of T.
__global__ void k_pair_elems(const DevGraph g, const int64_t* __restrict__ sidx,
                             const uint64_t* __restrict__ eoff, int64_t cnt, uint64_t ne,
                             int2* __restrict__ elems, uint64_t* __restrict__ ework,
                             unsigned* __restrict__ tcnt) {
  const uint64_t nchunks = (ne + CHUNK - 1) / CHUNK;
  for (uint64_t ch = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; ch < nchunks;
       ch += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j0 = ch * CHUNK, j1 = min(j0 + (uint64_t)CHUNK, ne);
    int64_t i = anchor_of(eoff, cnt, j0);
    PairList L = pair_list(g, sidx[i]);
    unsigned tr = 0;
    for (uint64_t j = j0; j < j1; ++j) {
      if (j >= eoff[i + 1]) {
        if (tr) atomicAdd(&tcnt[i], tr);
        tr = 0;
        do {
          ++i;
        } while (eoff[i + 1] == eoff[i]);
        L = pair_list(g, sidx[i]);
      }
      const uint32_t r = (uint32_t)(j - eoff[i]);
      const int32_t c = list_elem(g, L, r);
      uint32_t ty;
      bool valid = true;
      if (r < L.la) {
        ty = pair_s(g, L.b, c) ? TY_T : TY_A;
        tr += ty == TY_T ? 1u : 0u;
      } else {
        ty = TY_B;
        valid = !pair_s(g, L.a, c);  // listed from a already (in T)
      }
      elems[j] = make_int2((int32_t)((uint32_t)i | (ty << 30)), valid ? c : -1);
      ework[j] = valid ? (uint64_t)deg2(g, c) : 0ull;
    }
    if (tr) atomicAdd(&tcnt[i], tr);
  }
}

// Per draw: the stage (1) sets without a pair cd (from sa, sb, t), and the
// sizes of the stage (3) spaces: 3-hyperedges through a and b and
// 4-hyperedges through a (xw), at most min(t3(a), t3(b)) 3-hyperedges
// through both (gw).
template <bool kWeighted>
__global__ void __launch_bounds__(SAMPLE_THREADS)
    k_pair_terms(const DevGraph g, const int64_t* __restrict__ sidx,
                 const unsigned* __restrict__ tcnt, int64_t cnt, const uint64_t* __restrict__ wt,
                 const int64_t* __restrict__ off4, const PairClasses pc, int ncls,
                 unsigned long long* __restrict__ raw, uint64_t* __restrict__ xw,
                 uint64_t* __restrict__ gw) {
  __shared__ unsigned long long blo[176], bhi[176];
  for (int i = threadIdx.x; i < ncls; i += blockDim.x) blo[i] = bhi[i] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t ab = g.e2[sidx[i]];
    const int32_t a = (int32_t)(ab >> 32), b = (int32_t)(ab & 0xFFFFFFFFull);
    const uint64_t t = tcnt[i];
    const uint64_t sa = (uint64_t)deg2(g, a) - 1 - t, sb = (uint64_t)deg2(g, b) - 1 - t;
    const uint64_t w = kWeighted ? wt[i] : 1ull;
    bins_add(blo, bhi, pc.cls[PP_STAR], w, sa * (sa - 1) / 2 + sb * (sb - 1) / 2, false);
    bins_add(blo, bhi, pc.cls[PP_PATH], w, sa * sb, false);
    bins_add(blo, bhi, pc.cls[PP_PAW], w, (sa + sb) * t, false);
    bins_add(blo, bhi, pc.cls[PP_DIAMOND], w, t * (t - 1) / 2, false);
    const uint64_t t3a = g.off3 ? (uint64_t)(g.off3[a + 1] - g.off3[a]) : 0,
                   t3b = g.off3 ? (uint64_t)(g.off3[b + 1] - g.off3[b]) : 0,
                   q4a = off4 ? (uint64_t)(off4[a + 1] - off4[a]) : 0;
    xw[i] = t3a + t3b + q4a;
    gw[i] = min(t3a, t3b);
  }
  __syncthreads();
  bins_flush(blo, bhi, ncls, raw);
}

// Stage (1) corrections and stage (2): items (element c of a draw, pair
// neighbour x of c). x outside A ∪ B ∪ T ∪ {a, b}: the set {a, b, c, x} (a
// path, or a paw when c is in T). x in A ∪ B ∪ T: the pair cx moves the set
// {a, b, c, x} from its pattern without cx to the one with it, counted once
// (from the endpoint of the lower type, or the lower id within a type).
template <bool kWeighted>
__global__ void __launch_bounds__(SAMPLE_THREADS)
    k_pair_bulk(const DevGraph g, const int64_t* __restrict__ sidx, const int2* __restrict__ elems,
                const uint64_t* __restrict__ ews, int64_t ne, uint64_t total,
                const uint64_t* __restrict__ wt, const PairClasses pc, int ncls,
                unsigned long long* __restrict__ raw) {
  __shared__ unsigned long long blo[176], bhi[176];
  __shared__ int pcs[6];
  for (int i = threadIdx.x; i < ncls; i += blockDim.x) blo[i] = bhi[i] = 0;
  if (threadIdx.x < 6) pcs[threadIdx.x] = pc.cls[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t nchunks = (total + CHUNK - 1) / CHUNK;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t cb = warp * 32; cb < nchunks; cb += nwarps * 32) {
    const uint64_t g0 = (cb + lane) * CHUNK;
    const uint64_t g1 = min(g0 + CHUNK, total);
    int64_t j = 0;
    uint64_t r = 0, wa = 0;
    int32_t a = 0, b = 0, c = 0;
    int64_t co = 0;
    uint32_t ty = 0, di = 0;
    auto load = [&](int64_t jj) {
      const int2 el = elems[jj];
      di = (uint32_t)el.x & 0x3FFFFFFFu;
      ty = (uint32_t)el.x >> 30;
      c = el.y;
      const uint64_t ab = g.e2[sidx[di]];
      a = (int32_t)(ab >> 32);
      b = (int32_t)(ab & 0xFFFFFFFFull);
      co = g.off2[c];
      wa = ews[jj + 1] - ews[jj];
    };
    if (g0 < total) {
      j = anchor_of(ews, ne, g0);
      r = g0 - ews[j];
      load(j);
    }
    for (int it = 0; it < CHUNK; ++it) {
      const uint64_t gi = g0 + it;
      int pp = -1, pn = -1;
      if (gi < g1) {
        if (r == wa) {
          do {
            ++j;
          } while (ews[j + 1] == ews[j]);
          r = 0;
          load(j);
        }
        const int32_t x = g.adj2[co + r];
        ++r;
        if (x != a && x != b) {
          const bool inA = pair_s(g, a, x), inB = pair_s(g, b, x);
          if (!inA && !inB) {
            pp = ty == TY_T ? PP_PAW : PP_PATH;
          } else {
            const uint32_t tx = inA ? (inB ? TY_T : TY_A) : TY_B;
            if (ty < tx || (ty == tx && c < x)) {
              const uint32_t hi = max(ty, tx), lo = min(ty, tx);
              if (hi == TY_T) {
                pp = lo == TY_T ? PP_K4 : PP_DIAMOND;
                pn = lo == TY_T ? PP_DIAMOND : PP_PAW;
              } else if (lo == hi) {  // both in A or both in B
                pp = PP_PAW;
                pn = PP_STAR;
              } else {  // one in A, one in B
                pp = PP_C4;
                pn = PP_PATH;
              }
            }
          }
        }
      }
      bins_vote<kWeighted>(blo, bhi, pp >= 0 ? pcs[pp] : -1, false, di, wt);
      bins_vote<kWeighted>(blo, bhi, pn >= 0 ? pcs[pn] : -1, true, di, wt);
    }
  }
  __syncthreads();
  bins_flush(blo, bhi, ncls, raw);
}

// Stage (3), sets holding a larger hyperedge, each subtracted once: items
// per draw run over the 3-hyperedges through a, then through b, then the
// 4-hyperedges through a. A 3-hyperedge {a, b, c} goes to a list (its sets
// are every d with {a, b, c, d} connected, handled by k_pair_g1). Otherwise
// the hyperedge names one set {a, b, x, y}, subtracted when its pairs connect
// it and it holds none of the hyperedges that come first: 3-hyperedges with
// a and b, then with a, then with b, then the 4-hyperedge.
template <bool kWeighted>
__global__ void __launch_bounds__(SAMPLE_THREADS)
    k_pair_excl(const DevGraph g, const int64_t* __restrict__ sidx,
                const uint64_t* __restrict__ xs, int64_t cnt, uint64_t total,
                const uint64_t* __restrict__ wt, const int64_t* __restrict__ off4,
                const int32_t* __restrict__ inc4, const uint8_t* __restrict__ lut_g, int ncls,
                unsigned long long* __restrict__ raw, int2* __restrict__ g1, uint64_t cap1,
                unsigned long long* __restrict__ g1n) {
  __shared__ unsigned long long blo[176], bhi[176];
  __shared__ uint8_t lut[64];
  for (int i = threadIdx.x; i < ncls; i += blockDim.x) blo[i] = bhi[i] = 0;
  if (threadIdx.x < 64) lut[threadIdx.x] = lut_g[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t nchunks = (total + CHUNK - 1) / CHUNK;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t cb = warp * 32; cb < nchunks; cb += nwarps * 32) {
    const uint64_t g0 = (cb + lane) * CHUNK;
    const uint64_t g1e = min(g0 + CHUNK, total);
    int64_t i = 0;
    uint64_t r = 0, wa = 0, t3a = 0, t3b = 0;
    int32_t a = 0, b = 0;
    auto load = [&](int64_t ii) {
      const uint64_t ab = g.e2[sidx[ii]];
      a = (int32_t)(ab >> 32);
      b = (int32_t)(ab & 0xFFFFFFFFull);
      t3a = g.off3 ? (uint64_t)(g.off3[a + 1] - g.off3[a]) : 0;
      t3b = g.off3 ? (uint64_t)(g.off3[b + 1] - g.off3[b]) : 0;
      wa = xs[ii + 1] - xs[ii];
    };
    if (g0 < total) {
      i = anchor_of(xs, cnt, g0);
      r = g0 - xs[i];
      load(i);
    }
    for (int it = 0; it < CHUNK; ++it) {
      const uint64_t gi = g0 + it;
      int cls = -1;
      if (gi < g1e) {
        if (r == wa) {
          do {
            ++i;
          } while (xs[i + 1] == xs[i]);
          r = 0;
          load(i);
        }
        int32_t x = -1, y = -1;
        bool emit = false;
        if (r < t3a) {
          const int4 e = g.e3[g.inc3[g.off3[a] + (int64_t)r]];
          x = e.x == a ? e.y : e.x;
          y = e.z == a ? e.y : e.z;
          if (x == b || y == b) {
            const unsigned long long slot = atomicAdd(g1n, 1ull);
            if (slot < cap1) g1[slot] = make_int2((int32_t)i, x == b ? y : x);
          } else {
            emit = !triple_s(g, a, b, x) && !triple_s(g, a, b, y);
          }
        } else if (r < t3a + t3b) {
          const int4 e = g.e3[g.inc3[g.off3[b] + (int64_t)(r - t3a)]];
          x = e.x == b ? e.y : e.x;
          y = e.z == b ? e.y : e.z;
          emit = x != a && y != a && !triple_s(g, a, b, x) && !triple_s(g, a, b, y) &&
                 !triple_s(g, a, x, y);
        } else {
          const int4 q = g.e4[inc4[off4[a] + (int64_t)(r - t3a - t3b)]];
          const int32_t m[4] = {q.x, q.y, q.z, q.w};
          int k = 0;
          bool hb = false;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (m[u] == b) hb = true;
            if (m[u] != a && m[u] != b) {
              if (k == 0) x = m[u];
              else y = m[u];
              ++k;
            }
          }
          emit = hb && !triple_s(g, a, b, x) && !triple_s(g, a, b, y) &&
                 !triple_s(g, a, x, y) && !triple_s(g, b, x, y);
        }
        ++r;
        uint32_t mask = 0;
        if (emit && pair_pattern(g, a, b, x, y, mask)) cls = lut[mask];
      }
      bins_vote<kWeighted>(blo, bhi, cls, true, (uint32_t)i, wt);
    }
  }
  __syncthreads();
  bins_flush(blo, bhi, ncls, raw);
}

// Per listed 3-hyperedge {a, b, c}: its units, the draw's list L1 then c's
// pair neighbours.
__global__ void k_pair_g1_units(const DevGraph g, const int2* __restrict__ g1, int64_t n1,
                                const uint64_t* __restrict__ eoff, uint64_t* __restrict__ uw) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n1;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 e = g1[k];
    uw[k] = (eoff[e.x + 1] - eoff[e.x]) + (uint64_t)deg2(g, e.y);
  }
}

// The sets {a, b, c, d} holding the 3-hyperedge {a, b, c}: d in L1 (an
// element of the draw's list) or a pair neighbour of c outside L1 ∪ {a, b};
// subtracted when connected by their pairs, unless {a, b, d} is a
// 3-hyperedge too and d < c (the set then goes with d).
template <bool kWeighted>
__global__ void __launch_bounds__(SAMPLE_THREADS)
    k_pair_g1(const DevGraph g, const int64_t* __restrict__ sidx, const int2* __restrict__ g1,
              const uint64_t* __restrict__ us, int64_t n1, uint64_t total,
              const uint64_t* __restrict__ eoff, const int2* __restrict__ elems,
              const uint64_t* __restrict__ wt, const uint8_t* __restrict__ lut_g, int ncls,
              unsigned long long* __restrict__ raw) {
  __shared__ unsigned long long blo[176], bhi[176];
  __shared__ uint8_t lut[64];
  for (int i = threadIdx.x; i < ncls; i += blockDim.x) blo[i] = bhi[i] = 0;
  if (threadIdx.x < 64) lut[threadIdx.x] = lut_g[threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t nchunks = (total + CHUNK - 1) / CHUNK;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t cb = warp * 32; cb < nchunks; cb += nwarps * 32) {
    const uint64_t g0 = (cb + lane) * CHUNK;
    const uint64_t g1e = min(g0 + CHUNK, total);
    int64_t k = 0;
    uint64_t r = 0, wa = 0, l = 0, e0 = 0;
    int32_t a = 0, b = 0, c = 0;
    int64_t co = 0;
    uint32_t di = 0;
    auto load = [&](int64_t kk) {
      const int2 e = g1[kk];
      di = (uint32_t)e.x;
      c = e.y;
      const uint64_t ab = g.e2[sidx[di]];
      a = (int32_t)(ab >> 32);
      b = (int32_t)(ab & 0xFFFFFFFFull);
      e0 = eoff[di];
      l = eoff[di + 1] - e0;
      co = g.off2[c];
      wa = us[kk + 1] - us[kk];
    };
    if (g0 < total) {
      k = anchor_of(us, n1, g0);
      r = g0 - us[k];
      load(k);
    }
    for (int it = 0; it < CHUNK; ++it) {
      const uint64_t gi = g0 + it;
      int cls = -1;
      if (gi < g1e) {
        if (r == wa) {
          do {
            ++k;
          } while (us[k + 1] == us[k]);
          r = 0;
          load(k);
        }
        int32_t d;
        bool ok;
        if (r < l) {
          d = elems[e0 + r].y;
          ok = d >= 0 && d != c;
        } else {
          d = g.adj2[co + (int64_t)(r - l)];
          ok = d != a && d != b && !pair_s(g, a, d) && !pair_s(g, b, d);
        }
        ++r;
        if (ok && !(d < c && triple_s(g, a, b, d))) {
          uint32_t mask = 0;
          if (pair_pattern(g, a, b, c, d, mask)) cls = lut[mask];
        }
      }
      bins_vote<kWeighted>(blo, bhi, cls, true, di, wt);
    }
  }
  __syncthreads();
  bins_flush(blo, bhi, ncls, raw);
}

__global__ void k_deg4(const int4* __restrict__ e4, int64_t m, uint64_t* __restrict__ deg) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 e = e4[t];
    atomicAdd((unsigned long long*)&deg[e.x], 1ull);
    atomicAdd((unsigned long long*)&deg[e.y], 1ull);
    atomicAdd((unsigned long long*)&deg[e.z], 1ull);
    atomicAdd((unsigned long long*)&deg[e.w], 1ull);
  }
}

__global__ void k_place4(const int4* __restrict__ e4, int64_t m, const int64_t* __restrict__ off,
                         uint32_t* __restrict__ cursor, int32_t* __restrict__ inc) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 e = e4[t];
    inc[off[e.x] + atomicAdd(&cursor[e.x], 1u)] = (int32_t)t;
    inc[off[e.y] + atomicAdd(&cursor[e.y], 1u)] = (int32_t)t;
    inc[off[e.z] + atomicAdd(&cursor[e.z], 1u)] = (int32_t)t;
    inc[off[e.w] + atomicAdd(&cursor[e.w], 1u)] = (int32_t)t;
  }
}

// node -> 4-hyperedges, kept in the graph (freed with it)
void ensure_inc4(hm_graph* g, cudaStream_t st) {
  if (g->off4 || g->kmax < 4 || g->counts[4] == 0) return;
  const int64_t n = g->n, m4 = g->counts[4];
  int64_t* off4 = dalloc<int64_t>((size_t)n + 1, st);
  g->owned.push_back(off4);
  int32_t* inc4 = dalloc<int32_t>((size_t)4 * m4, st);
  g->owned.push_back(inc4);
  DBuf<uint32_t> cursor((size_t)n, st);
  HM_CUDA(cudaMemsetAsync(off4, 0, ((size_t)n + 1) * 8, st));
  HM_CUDA(cudaMemsetAsync(cursor.p, 0, (size_t)n * 4, st));
  k_deg4<<<grid_n(m4), 256, 0, st>>>(g->e4, m4, reinterpret_cast<uint64_t*>(off4));
  HM_KCHECK();
  ScanJob oj{reinterpret_cast<uint64_t*>(off4), n, nullptr};
  scan_batch_inplace(&oj, 1, st);
  k_place4<<<grid_n(m4), 256, 0, st>>>(g->e4, m4, off4, cursor.p, inc4);
  HM_KCHECK();
  g->off4 = off4;
  g->inc4 = inc4;
}

// The class of each pairs-only pattern (host tables).
PairClasses pair_classes() {
  const ClassTables& T = class_tables(4);
  PairClasses pc;
  for (int p = 0; p < 6; ++p) pc.cls[p] = (int)T.lut[kPatternMask[p]];
  return pc;
}

// Whether the per-candidate enumeration (SamPA / SamPB) serves the order-4
// pair stratum instead (HM_SAMPLE_PAIR_ENUM=1, for tests).
bool pair_enum() {
  const char* env = std::getenv("HM_SAMPLE_PAIR_ENUM");
  return env && env[0] == '1';
}

template <class K>
void launch_walk(K kernel, uint64_t total, const char* name, cudaStream_t s,
                 const std::function<void(unsigned)>& go) {
  if (total == 0) return;
  cudaEvent_t ev = nullptr;
  const bool tr = trace_on(name);
  if (tr) trace_begin(s, &ev);
  go((unsigned)sample_blocks((const void*)kernel, total));
  HM_KCHECK();
  if (tr) trace_end(name, s, ev);
}

// The pair stratum of one batch at order 4 by types (see above).
void pair_batch_bulk(const hm_graph* g, const DrawArgs& da, const int64_t* sidx,
                     const uint64_t* wt, const uint64_t* lsize, bool weighted,
                     unsigned long long* raw, cudaStream_t st) {
  const int64_t cnt = da.count;
  const ClassTables& T = class_tables(4);
  const uint8_t* lut = device_lut(4);
  const PairClasses pc = pair_classes();
  const hm::DevGraph gv = g->view();
  DBuf<uint64_t> eoff(cnt + 1, st), xw(cnt, st), gw(cnt, st), xs(cnt + 1, st), gs(cnt + 1, st);
  DBuf<unsigned> tcnt(cnt, st);
  DBuf<unsigned long long> g1n(1, st);
  HM_CUDA(cudaMemsetAsync(tcnt.p, 0, (size_t)cnt * 4, st));
  HM_CUDA(cudaMemsetAsync(g1n.p, 0, 8, st));
  const uint64_t ne = scan_total(lsize, eoff.p, cnt, st);
  DBuf<int2> elems(std::max<uint64_t>(ne, 1), st);
  DBuf<uint64_t> ework(std::max<uint64_t>(ne, 1), st), ews(ne + 1, st);
  if (ne) {
    const uint64_t chunks = (ne + CHUNK - 1) / CHUNK;
    k_pair_elems<<<grid_n((int64_t)chunks), 256, 0, st>>>(gv, sidx, eoff.p, cnt, ne, elems.p,
                                                         ework.p, tcnt.p);
    HM_KCHECK();
  }
  if (weighted)
    k_pair_terms<true><<<grid_n(cnt), SAMPLE_THREADS, 0, st>>>(gv, sidx, tcnt.p, cnt, wt, g->off4,
                                                               pc, T.ncls, raw, xw.p, gw.p);
  else
    k_pair_terms<false><<<grid_n(cnt), SAMPLE_THREADS, 0, st>>>(gv, sidx, tcnt.p, cnt, wt, g->off4,
                                                                pc, T.ncls, raw, xw.p, gw.p);
  HM_KCHECK();
  if (ne) {
    const uint64_t tb = scan_total(ework.p, ews.p, (int64_t)ne, st);
    if (weighted)
      launch_walk(k_pair_bulk<true>, tb, "sample_pair_bulk", st, [&](unsigned blocks) {
        k_pair_bulk<true><<<blocks, SAMPLE_THREADS, 0, st>>>(gv, sidx, elems.p, ews.p,
                                                            (int64_t)ne, tb, wt, pc, T.ncls, raw);
      });
    else
      launch_walk(k_pair_bulk<false>, tb, "sample_pair_bulk", st, [&](unsigned blocks) {
        k_pair_bulk<false><<<blocks, SAMPLE_THREADS, 0, st>>>(gv, sidx, elems.p, ews.p,
                                                             (int64_t)ne, tb, wt, pc, T.ncls, raw);
      });
  }
  const uint64_t tx = scan_total(xw.p, xs.p, cnt, st);
  const uint64_t cap1 = scan_total(gw.p, gs.p, cnt, st);
  if (tx == 0) return;
  DBuf<int2> g1(std::max<uint64_t>(cap1, 1), st);
  if (weighted)
    launch_walk(k_pair_excl<true>, tx, "sample_pair_excl", st, [&](unsigned blocks) {
      k_pair_excl<true><<<blocks, SAMPLE_THREADS, 0, st>>>(gv, sidx, xs.p, cnt, tx, wt, g->off4,
                                                          g->inc4, lut, T.ncls, raw, g1.p, cap1, g1n.p);
    });
  else
    launch_walk(k_pair_excl<false>, tx, "sample_pair_excl", st, [&](unsigned blocks) {
      k_pair_excl<false><<<blocks, SAMPLE_THREADS, 0, st>>>(gv, sidx, xs.p, cnt, tx, wt, g->off4,
                                                           g->inc4, lut, T.ncls, raw, g1.p, cap1, g1n.p);
    });
  unsigned long long n1 = 0;
  HM_CUDA(cudaMemcpyAsync(&n1, g1n.p, 8, cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  HM_CHECK(n1 <= cap1, HM_EINVAL,
           "pair stratum: more 3-hyperedges through a drawn pair than min(t3(a), t3(b))");
  if (n1 == 0) return;
  DBuf<uint64_t> uw(n1, st), us(n1 + 1, st);
  k_pair_g1_units<<<grid_n((int64_t)n1), 256, 0, st>>>(gv, g1.p, (int64_t)n1, eoff.p, uw.p);
  HM_KCHECK();
  const uint64_t tu = scan_total(uw.p, us.p, (int64_t)n1, st);
  if (weighted)
    launch_walk(k_pair_g1<true>, tu, "sample_pair_g1", st, [&](unsigned blocks) {
      k_pair_g1<true><<<blocks, SAMPLE_THREADS, 0, st>>>(gv, sidx, g1.p, us.p, (int64_t)n1, tu,
                                                        eoff.p, elems.p, wt, lut, T.ncls, raw);
    });
  else
    launch_walk(k_pair_g1<false>, tu, "sample_pair_g1", st, [&](unsigned blocks) {
      k_pair_g1<false><<<blocks, SAMPLE_THREADS, 0, st>>>(gv, sidx, g1.p, us.p, (int64_t)n1, tu,
                                                         eoff.p, elems.p, wt, lut, T.ncls, raw);
    });
}

// One batch of draws of stratum s.
void sample_batch(const hm_graph* g, int order, int s, const DrawArgs& da, bool weighted,
                  unsigned long long* raw, cudaStream_t st) {
  const int64_t cnt = da.count;
  DBuf<int64_t> sidx(cnt, st);
  DBuf<uint64_t> wt(cnt, st), work(cnt, st), lsize(cnt, st), ws(cnt + 1, st);
  k_draw<<<grid_n(cnt), 256, 0, st>>>(g->view(), da, sidx.p, wt.p, work.p, lsize.p);
  HM_KCHECK();
  if (s == order) {
    if (order == 3) {
      FamT3 f;
      f.map = sidx.p;
      launch_sample(g, f, nullptr, 0, (uint64_t)cnt, wt.p, weighted, order, raw, st);
    } else {
      FamQ f;
      f.map = sidx.p;
      launch_sample(g, f, nullptr, 0, (uint64_t)cnt, wt.p, weighted, order, raw, st);
    }
    return;
  }
  if (order == 4 && s == 2 && !pair_enum()) {
    pair_batch_bulk(g, da, sidx.p, wt.p, lsize.p, weighted, raw, st);
    return;
  }
  const uint64_t total = scan_total(work.p, ws.p, cnt, st);
  if (order == 4 && s == 3) {
    FamTXT<false> f;
    f.map = sidx.p;
    launch_sample(g, f, ws.p, cnt, total, wt.p, weighted, order, raw, st);
  } else if (order == 3) {
    SamP3 f{sidx.p};
    launch_sample(g, f, ws.p, cnt, total, wt.p, weighted, order, raw, st);
  } else {
    SamPA fa{sidx.p};
    launch_sample(g, fa, ws.p, cnt, total, wt.p, weighted, order, raw, st);
    DBuf<uint64_t> eoff(cnt + 1, st);
    const uint64_t ne = scan_total(lsize.p, eoff.p, cnt, st);
    if (ne == 0) return;
    DBuf<int2> elems(ne, st);
    DBuf<uint64_t> ework(ne, st), ews(ne + 1, st);
    k_elements<<<grid_n(cnt), 256, 0, st>>>(g->view(), sidx.p, cnt, eoff.p, elems.p, ework.p);
    HM_KCHECK();
    const uint64_t tb = scan_total(ework.p, ews.p, (int64_t)ne, st);
    SamPB fb{sidx.p, elems.p};
    launch_sample(g, fb, ews.p, (int64_t)ne, tb, wt.p, weighted, order, raw, st);
  }
}

}  // namespace

void count_sampled(hm_graph* g, int order, const uint64_t* S, uint64_t seed, const uint32_t* d_q,
                   double* d_est, uint64_t* d_raw, cudaStream_t st) {
  const ClassTables& T = class_tables(order);
  if (order == 4 && S[2] > 0 && !pair_enum()) ensure_inc4(g, st);
  DBuf<unsigned long long> raw_tmp(d_raw ? 0 : 2 * T.ncls, st);
  unsigned long long* raw = d_raw ? (unsigned long long*)d_raw : raw_tmp.p;
  HM_CUDA(cudaMemsetAsync(raw, 0, 2 * T.ncls * sizeof(unsigned long long), st));
  DBuf<uint64_t> Q(5, st);
  uint64_t hostQ[5] = {0, 0, 0, 0, 0};
  for (int s = 2; s <= order; ++s) hostQ[s] = (uint64_t)g->counts[s];
  HM_CUDA(cudaMemcpyAsync(Q.p, hostQ, sizeof hostQ, cudaMemcpyHostToDevice, st));
  const bool weighted = d_q != nullptr;
  int64_t qoff = 0;
  for (int s = 2; s <= order; ++s) {
    const int64_t len = g->counts[s];
    DBuf<uint64_t> P;
    if (weighted && len > 0) {
      DBuf<int> bad(1, st);
      HM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
      k_bad_weight<<<grid_n(len), 256, 0, st>>>(d_q + qoff, len, bad.p);
      HM_KCHECK();
      int hb = 0;
      HM_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof hb, cudaMemcpyDeviceToHost, st));
      DBuf<uint64_t> wide(len, st);
      P.alloc(len + 1, st);
      k_widen<<<grid_n(len), 256, 0, st>>>(d_q + qoff, len, wide.p);
      HM_KCHECK();
      scan_exclusive_u64(wide.p, P.p, len, st);
      HM_CUDA(cudaMemcpyAsync(Q.p + s, P.p + len, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
      HM_CUDA(cudaStreamSynchronize(st));
      HM_CHECK(hb == 0, HM_EINVAL, "proposal weights must be >= 1");
    }
    if (len > 0) {
      for (uint64_t t0 = 0; t0 < S[s]; t0 += SAMPLE_BATCH) {
        DrawArgs da;
        da.seed = seed;
        da.s = s;
        da.order = order;
        da.t0 = t0;
        da.count = (int64_t)std::min<uint64_t>(SAMPLE_BATCH, S[s] - t0);
        da.len = len;
        da.P = weighted ? P.p : nullptr;
        da.q = weighted ? d_q + qoff : nullptr;
        sample_batch(g, order, s, da, weighted, raw, st);
      }
    }
    qoff += len;
  }
  EstArgs e{};
  for (int s = 2; s <= order; ++s) {
    e.S[s] = (double)S[s];
    e.E[s] = (uint64_t)g->counts[s];
  }
  e.weighted = weighted ? 1 : 0;
  e.ncls = T.ncls;
  for (int c = 0; c < T.ncls; ++c) {
    e.maxcard[c] = (int8_t)T.maxcard[c];
    e.countmax[c] = (int8_t)T.countmax[c];
  }
  k_estimate<<<1, 256, 0, st>>>(e, Q.p, raw, d_est);
  HM_KCHECK();
}

// ================================================================ allocation-free variant
// Some callers cannot allocate device memory while they count: applications
// that reserve the GPU's memory up front (a serving process with a fixed
// memory budget, or one whose other framework's caching allocator holds the
// rest), and latency-critical loops where cudaMalloc/cudaFree may block or
// synchronise the device. hm_count_sampled_noalloc serves them: every
// temporary lives in one file-scope device array of NOALLOC_BYTES, held by
// each GPU that loads the library until the process exits. The call itself
// synchronises its stream and reads values back to the host between batches,
// so it is made from ordinary host code, not from a stream callback.
namespace {

constexpr size_t NOALLOC_BYTES = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];
__device__ __align__(16) uint8_t g_noalloc_lut3[16];
__device__ __align__(16) uint8_t g_noalloc_lut4[2048];

struct NoallocDevice {
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  const uint8_t* lut3 = nullptr;
  const uint8_t* lut4 = nullptr;
};
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];
bool g_noalloc_ready[64] = {false};

// Once per device, with that device current: the symbols' device addresses
// (host code cannot use the arrays' names as device pointers) and the class
// tables copied into their symbols.
NoallocDevice noalloc_setup() {
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev));
  HM_CHECK(dev >= 0 && dev < 64, HM_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ready[dev]) {
    NoallocDevice d;
    void* p = nullptr;
    HM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    d.scratch = (unsigned char*)p;
    HM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_lut3));
    d.lut3 = (const uint8_t*)p;
    HM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_lut4));
    d.lut4 = (const uint8_t*)p;
    HM_CUDA(cudaMemcpyToSymbol(g_noalloc_lut3, class_tables(3).lut.data(), 16));
    HM_CUDA(cudaMemcpyToSymbol(g_noalloc_lut4, class_tables(4).lut.data(), 2048));
    g_noalloc_dev[dev] = d;
    g_noalloc_ready[dev] = true;
  }
  return g_noalloc_dev[dev];
}

// Bump allocation inside the static array (256-byte aligned pieces).
struct Arena {
  unsigned char* base;
  size_t cap, used;
  template <class T>
  T* take(size_t count) {
    const size_t off = (used + 255) & ~(size_t)255;
    HM_CHECK(off + count * sizeof(T) <= cap, HM_EINVAL,
             "request exceeds the 32 MiB static scratch of hm_count_sampled_noalloc");
    used = off + count * sizeof(T);
    return (T*)(base + off);
  }
};

uint64_t scan_total_in(const uint64_t* in, uint64_t* out, int64_t n, Arena& ar, cudaStream_t s) {
  const size_t need = scan_scratch_elems(n);
  uint64_t* tmp = need ? ar.take<uint64_t>(need) : nullptr;
  scan_exclusive_u64_in(in, out, n, s, tmp, need);
  uint64_t tot = 0;
  HM_CUDA(cudaMemcpyAsync(&tot, out + n, sizeof tot, cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  return tot;
}

template <class F>
void launch_sample_lut(const hm_graph* g, const F& f, const uint64_t* ws, int64_t A,
                       uint64_t total, const uint64_t* wt, bool weighted, int order,
                       const uint8_t* lut, unsigned long long* raw, cudaStream_t s) {
  if (total == 0) return;
  const ClassTables& T = class_tables(order);
  if (weighted) {
    k_sample<F, true><<<sample_blocks((const void*)k_sample<F, true>, total), SAMPLE_THREADS, 0,
                        s>>>(g->view(), f, ws, A, total, wt, lut, (int)T.lut.size(), T.ncls, raw);
  } else {
    k_sample<F, false><<<sample_blocks((const void*)k_sample<F, false>, total), SAMPLE_THREADS, 0,
                         s>>>(g->view(), f, ws, A, total, wt, lut, (int)T.lut.size(), T.ncls, raw);
  }
  HM_KCHECK();
}

void sample_batch_in(const hm_graph* g, int order, int s, const DrawArgs& da, bool weighted,
                     const uint8_t* lut, unsigned long long* raw, Arena& ar, cudaStream_t st) {
  const size_t mark = ar.used;
  const int64_t cnt = da.count;
  int64_t* sidx = ar.take<int64_t>(cnt);
  uint64_t* wt = ar.take<uint64_t>(cnt);
  uint64_t* work = ar.take<uint64_t>(cnt);
  uint64_t* lsize = ar.take<uint64_t>(cnt);
  uint64_t* ws = ar.take<uint64_t>(cnt + 1);
  k_draw<<<grid_n(cnt), 256, 0, st>>>(g->view(), da, sidx, wt, work, lsize);
  HM_KCHECK();
  if (s == order) {
    if (order == 3) {
      FamT3 f;
      f.map = sidx;
      launch_sample_lut(g, f, nullptr, 0, (uint64_t)cnt, wt, weighted, order, lut, raw, st);
    } else {
      FamQ f;
      f.map = sidx;
      launch_sample_lut(g, f, nullptr, 0, (uint64_t)cnt, wt, weighted, order, lut, raw, st);
    }
  } else {
    const uint64_t total = scan_total_in(work, ws, cnt, ar, st);
    if (order == 4 && s == 3) {
      FamTXT<false> f;
      f.map = sidx;
      launch_sample_lut(g, f, ws, cnt, total, wt, weighted, order, lut, raw, st);
    } else if (order == 3) {
      SamP3 f{sidx};
      launch_sample_lut(g, f, ws, cnt, total, wt, weighted, order, lut, raw, st);
    } else {
      SamPA fa{sidx};
      launch_sample_lut(g, fa, ws, cnt, total, wt, weighted, order, lut, raw, st);
      uint64_t* eoff = ar.take<uint64_t>(cnt + 1);
      const uint64_t ne = scan_total_in(lsize, eoff, cnt, ar, st);
      if (ne > 0) {
        int2* elems = ar.take<int2>(ne);
        uint64_t* ework = ar.take<uint64_t>(ne);
        uint64_t* ews = ar.take<uint64_t>(ne + 1);
        k_elements<<<grid_n(cnt), 256, 0, st>>>(g->view(), sidx, cnt, eoff, elems, ework);
        HM_KCHECK();
        const uint64_t tb = scan_total_in(ework, ews, (int64_t)ne, ar, st);
        SamPB fb{sidx, elems};
        launch_sample_lut(g, fb, ews, (int64_t)ne, tb, wt, weighted, order, lut, raw, st);
      }
    }
  }
  // the next batch may reuse this batch's pieces only after its kernels ran
  HM_CUDA(cudaStreamSynchronize(st));
  ar.used = mark;
}

}  // namespace

void count_sampled_noalloc(hm_graph* g, int order, const uint64_t* S, uint64_t seed,
                           const uint32_t* d_q, double* d_est, uint64_t* d_raw, cudaStream_t st) {
  const NoallocDevice nd = noalloc_setup();
  const ClassTables& T = class_tables(order);
  const uint8_t* lut = order == 3 ? nd.lut3 : nd.lut4;
  Arena ar{nd.scratch, NOALLOC_BYTES, 0};
  unsigned long long* raw = d_raw ? (unsigned long long*)d_raw
                                  : ar.take<unsigned long long>(2 * (size_t)T.ncls);
  HM_CUDA(cudaMemsetAsync(raw, 0, 2 * T.ncls * sizeof(unsigned long long), st));
  uint64_t* Q = ar.take<uint64_t>(5);
  uint64_t hostQ[5] = {0, 0, 0, 0, 0};
  for (int s = 2; s <= order; ++s) hostQ[s] = (uint64_t)g->counts[s];
  HM_CUDA(cudaMemcpyAsync(Q, hostQ, sizeof hostQ, cudaMemcpyHostToDevice, st));
  int* bad = ar.take<int>(1);
  const bool weighted = d_q != nullptr;
  int64_t qoff = 0;
  for (int s = 2; s <= order; ++s) {
    const int64_t len = g->counts[s];
    // worst-case bytes of one draw: per-draw arrays and scan temporaries, plus,
    // for the pair stratum at order 4 (the only one that builds second-level
    // entries), up to 2 * max pair degree entries of 24 bytes
    const size_t per_draw =
        6 * 8 + 8 + (order == 4 && s == 2 ? (size_t)2 * (size_t)g->max_d2 * 32 : 0);
    const size_t mark = ar.used;
    uint64_t* P = nullptr;
    if (weighted && len > 0) {
      HM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
      k_bad_weight<<<grid_n(len), 256, 0, st>>>(d_q + qoff, len, bad);
      HM_KCHECK();
      uint64_t* wide = ar.take<uint64_t>(len);
      P = ar.take<uint64_t>(len + 1);
      k_widen<<<grid_n(len), 256, 0, st>>>(d_q + qoff, len, wide);
      HM_KCHECK();
      scan_total_in(wide, P, len, ar, st);
      int hb = 0;
      HM_CUDA(cudaMemcpyAsync(&hb, bad, sizeof hb, cudaMemcpyDeviceToHost, st));
      HM_CUDA(cudaMemcpyAsync(Q + s, P + len, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
      HM_CUDA(cudaStreamSynchronize(st));
      HM_CHECK(hb == 0, HM_EINVAL, "proposal weights must be >= 1");
    }
    if (len > 0 && S[s] > 0) {
      const size_t avail = ar.cap - ((ar.used + 255) & ~(size_t)255);
      const size_t slack = (size_t)64 << 10;
      HM_CHECK(avail > slack + 2 * per_draw, HM_EINVAL,
               "graph too large for the 32 MiB static scratch of hm_count_sampled_noalloc");
      int64_t batch = (int64_t)((avail - slack) / (per_draw + per_draw / 1024 + 16));
      if (batch > SAMPLE_BATCH) batch = SAMPLE_BATCH;
      for (uint64_t t0 = 0; t0 < S[s]; t0 += (uint64_t)batch) {
        DrawArgs da;
        da.seed = seed;
        da.s = s;
        da.order = order;
        da.t0 = t0;
        da.count = (int64_t)std::min<uint64_t>((uint64_t)batch, S[s] - t0);
        da.len = len;
        da.P = P;
        da.q = weighted ? d_q + qoff : nullptr;
        sample_batch_in(g, order, s, da, weighted, lut, raw, ar, st);
      }
    }
    ar.used = mark;
    qoff += len;
  }
  EstArgs e{};
  for (int s = 2; s <= order; ++s) {
    e.S[s] = (double)S[s];
    e.E[s] = (uint64_t)g->counts[s];
  }
  e.weighted = weighted ? 1 : 0;
  e.ncls = T.ncls;
  for (int c = 0; c < T.ncls; ++c) {
    e.maxcard[c] = (int8_t)T.maxcard[c];
    e.countmax[c] = (int8_t)T.countmax[c];
  }
  k_estimate<<<1, 256, 0, st>>>(e, Q, raw, d_est);
  HM_KCHECK();
}

}  // namespace hm

extern "C" hm_status hm_count_sampled_noalloc(hm_graph* g, int order,
                                              const uint64_t* samples_per_size,
                                              uint64_t total_samples, uint64_t seed,
                                              const uint32_t* d_q, double* d_est,
                                              uint64_t* d_raw, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g != nullptr, HM_EINVAL, "NULL graph");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= g->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    HM_CHECK(d_est != nullptr, HM_EINVAL, "NULL estimate buffer");
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CHECK(dev == g->device, HM_EINVAL, "graph was built on another device");
    uint64_t S[5] = {0, 0, 0, 0, 0};
    if (samples_per_size) {
      for (int s = 2; s <= order; ++s) S[s] = samples_per_size[s];
    } else if (order == 4) {
      S[2] = total_samples / 6;
      S[4] = total_samples / 3;
      S[3] = total_samples - S[2] - S[4];
    } else {
      S[2] = total_samples / 4;
      S[3] = total_samples - S[2];
    }
    for (int s = 2; s <= order; ++s)
      HM_CHECK(g->counts[s] == 0 || S[s] > 0, HM_EINVAL,
               "a non-empty stratum has no samples (S_s == 0 with |E_s| > 0)");
    hm::count_sampled_noalloc(g, order, S, seed, d_q, d_est, d_raw, (cudaStream_t)stream);
  });
}

extern "C" hm_status hm_count_sampled(hm_graph* g, int order, const uint64_t* samples_per_size,
                                      uint64_t total_samples, uint64_t seed, const uint32_t* d_q,
                                      double* d_est, uint64_t* d_raw, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g != nullptr, HM_EINVAL, "NULL graph");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= g->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    HM_CHECK(d_est != nullptr, HM_EINVAL, "NULL estimate buffer");
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CHECK(dev == g->device, HM_EINVAL, "graph was built on another device");
    uint64_t S[5] = {0, 0, 0, 0, 0};
    if (samples_per_size) {
      for (int s = 2; s <= order; ++s) S[s] = samples_per_size[s];
    } else if (order == 4) {
      S[2] = total_samples / 6;
      S[4] = total_samples / 3;
      S[3] = total_samples - S[2] - S[4];
    } else {
      S[2] = total_samples / 4;
      S[3] = total_samples - S[2];
    }
    for (int s = 2; s <= order; ++s)
      HM_CHECK(g->counts[s] == 0 || S[s] > 0, HM_EINVAL,
               "a non-empty stratum has no samples (S_s == 0 with |E_s| > 0)");
    hm::count_sampled(g, order, S, seed, d_q, d_est, d_raw, (cudaStream_t)stream);
  });
}
