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
#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "baseline.cuh"
#include "families.cuh"

namespace hm {
namespace {

using namespace fam;

// Union of graphs (null-model batch): at most this many graphs per launch,
// each with its own histogram row; block bins are then uint32, read as signed
// when flushed (the launch keeps every block below 2^31 candidates, and a
// block's net count of a class may be negative when its sets are subtracted
// for the graphlet census).
constexpr int MAX_GRAPHS = 64;
constexpr int BIN_STRIDE = 176;

template <class F, bool kBatched>
__global__ void __launch_bounds__(CENSUS_THREADS)
    k_census(const DevGraph g, const F fam, const uint64_t* __restrict__ ws, int64_t A,
             uint64_t begin, uint64_t total, int chunk, const uint8_t* __restrict__ lut_g,
             int nmask, int ncls, int ngraphs, int sub, unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long bins[kBatched ? 1 : BIN_STRIDE];
  __shared__ unsigned int gbins[kBatched ? MAX_GRAPHS * BIN_STRIDE : 1];
  __shared__ __align__(16) uint8_t lut[2048];
  load_lut(lut, lut_g, nmask);
  if (kBatched) {
    for (int i = threadIdx.x; i < ngraphs * BIN_STRIDE; i += blockDim.x) gbins[i] = 0;
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x) bins[i] = 0;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  // candidates [begin, total) in chunks of `chunk` consecutive ones per lane
  const uint64_t nchunks = (total - begin + chunk - 1) / chunk;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t cb = warp * 32; cb < nchunks; cb += nwarps * 32) {
    const uint64_t g0 = begin + (cb + lane) * chunk;
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
      int key = -1, key2 = -1;
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
          // the graphlet census counts this set under its pair pattern too
          const uint8_t c2 = sub ? lut[mask & 63u] : (uint8_t)0xFF;
          if (c2 != 0xFF) key2 = (kBatched ? gid * BIN_STRIDE : 0) + (int)c2;
        }
      }
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      if (key >= 0 && lane == __ffs(peers) - 1) {
        if (kBatched)
          atomicAdd(&gbins[key], (unsigned int)__popc(peers));
        else
          atomicAdd(&bins[key], (unsigned long long)__popc(peers));
      }
      if (sub) {
        const unsigned peers2 = __match_any_sync(0xffffffffu, key2);
        if (key2 >= 0 && lane == __ffs(peers2) - 1) {
          if (kBatched)
            atomicAdd(&gbins[key2], 0u - (unsigned int)__popc(peers2));
          else
            atomicAdd(&bins[key2], 0ull - (unsigned long long)__popc(peers2));
        }
      }
    }
  }
  __syncthreads();
  if (kBatched) {
    for (int i = threadIdx.x; i < ngraphs * BIN_STRIDE; i += blockDim.x)
      if (gbins[i])
        atomicAdd(&hist[(i / BIN_STRIDE) * ncls + i % BIN_STRIDE],
                  (unsigned long long)(long long)(int)gbins[i]);
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x)
      if (bins[i]) atomicAdd(&hist[i], bins[i]);
  }
}

// Bit-sliced families: each item evaluates up to bwords*32 candidates and
// adds its class counts to the block's bins.
#ifndef HM_BITS_CHUNK
#define HM_BITS_CHUNK 1  // consecutive items per thread (1: best balance, measured)
#endif
constexpr int BITS_CHUNK = HM_BITS_CHUNK;
#ifndef HM_BITS_MINBLOCKS
#define HM_BITS_MINBLOCKS 4  // resident blocks per SM the register budget targets
#endif

template <class F, bool kBatched>
__global__ void __launch_bounds__(CENSUS_THREADS, HM_BITS_MINBLOCKS)
    k_census_bits(const DevGraph g, const F fam, const uint64_t* __restrict__ ws, int64_t A,
                  uint64_t begin, uint64_t total, const uint8_t* __restrict__ lut_g, int nmask,
                  int ncls, int ngraphs, unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long bins[kBatched ? 1 : BIN_STRIDE];
  __shared__ unsigned int gbins[kBatched ? MAX_GRAPHS * BIN_STRIDE : 1];
  __shared__ __align__(16) uint8_t lut[2048];
  load_lut(lut, lut_g, nmask);
  if (kBatched) {
    for (int i = threadIdx.x; i < ngraphs * BIN_STRIDE; i += blockDim.x) gbins[i] = 0;
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x) bins[i] = 0;
  }
  __syncthreads();
  // items [begin, total), BITS_CHUNK consecutive ones per thread
  const uint64_t nchunks = (total - begin + BITS_CHUNK - 1) / BITS_CHUNK;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t g0 = begin + c * BITS_CHUNK, g1 = min(g0 + BITS_CHUNK, total);
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
      if (gbins[i])
        atomicAdd(&hist[(i / BIN_STRIDE) * ncls + i % BIN_STRIDE],
                  (unsigned long long)(long long)(int)gbins[i]);
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x)
      if (bins[i]) atomicAdd(&hist[i], bins[i]);
  }
}

// Bit-sliced TX, sets whose largest hyperedges have 3 members: one warp per
// 3-hyperedge e = {a < b < c}, lane l taking the row words l, l + 32, ...; the
// fourth node d runs over the ids joined to e by a pair or a 3-hyperedge. A
// set is kept at its smallest 3-hyperedge -- {a,b,d} < e iff d < c,
// {a,c,d} < e iff d < b, {b,c,d} < e iff d < a -- and when it holds no
// 4-hyperedge. Candidates with no 3-hyperedge besides e and no possible
// 4-hyperedge are counted by popcount per pattern of their pairs to e (summed
// over the warp); the others one by one. kExact: exact triple rows decide the
// 3-hyperedges; otherwise the co-occurrence rows mark the candidates that get
// hash probes. sub: subtract every set from the class of its pair pattern too
// (graphlet census).
template <bool kExact, bool kBatched>
__global__ void __launch_bounds__(CENSUS_THREADS)
    k_census_txw(const DevGraph g, int64_t t0, int64_t t1, const uint8_t* __restrict__ lut_g,
                 int nmask, int ncls, int ngraphs, int sub, unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long bins[kBatched ? 1 : BIN_STRIDE];
  __shared__ unsigned int gbins[kBatched ? MAX_GRAPHS * BIN_STRIDE : 1];
  __shared__ __align__(16) uint8_t lut[2048];
  load_lut(lut, lut_g, nmask);
  if (kBatched) {
    for (int i = threadIdx.x; i < ngraphs * BIN_STRIDE; i += blockDim.x) gbins[i] = 0;
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x) bins[i] = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int32_t bw = g.bwords;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = t0 + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < t1;
       t += warps) {
    const int4 e = g.e3[t];
    const int32_t a = e.x, b = e.y, c = e.z, base = graph_base(g, a);
    const int32_t al = a - base, bl = b - base, cl = c - base;
    const bool ab = btest(g, g.bits2, a, b), ac = btest(g, g.bits2, a, c),
               bc = btest(g, g.bits2, b, c);
    const bool qd = btest(g, g.bits4, a, b) && btest(g, g.bits4, a, c) &&
                    btest(g, g.bits4, b, c);
    const uint32_t *Ba = brow(g.bits2, bw, a), *Bb = brow(g.bits2, bw, b),
                   *Bc = brow(g.bits2, bw, c);
    const uint32_t* R1 = kExact ? g.tri3 + ((size_t)a * g.n + b) * bw : brow(g.bits3, bw, a);
    const uint32_t* R2 = kExact ? g.tri3 + ((size_t)a * g.n + c) * bw : brow(g.bits3, bw, b);
    const uint32_t* R3 = kExact ? g.tri3 + ((size_t)b * g.n + c) * bw : brow(g.bits3, bw, c);
    unsigned int* gb = kBatched ? gbins + graph_of(g, a) * BIN_STRIDE : nullptr;
    uint32_t n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int32_t w = lane; w < bw; w += 32) {
      const uint32_t pa = __ldg(Ba + w), pb = __ldg(Bb + w), pc = __ldg(Bc + w);
      uint32_t r1, r2, r3;
      if (kExact) {
        r1 = __ldg(R1 + w);  // abd
        r2 = __ldg(R2 + w);  // acd
        r3 = __ldg(R3 + w);  // bcd
      } else {
        const uint32_t ta = __ldg(R1 + w), tb = __ldg(R2 + w), tc = __ldg(R3 + w);
        r1 = ta & tb;
        r2 = ta & tc;
        r3 = tb & tc;
      }
      const uint32_t self = selfbit(w, al) | selfbit(w, bl) | selfbit(w, cl);
      const uint32_t tr = r1 | r2 | r3;
      uint32_t z = (pa | pb | pc | tr) & ~self;
      if (kExact) z &= ~((r1 & below(w, cl)) | (r2 & below(w, bl)) | (r3 & below(w, al)));
      if (!z) continue;
      const uint32_t risky = qd ? (__ldg(brow(g.bits4, bw, a) + w) & __ldg(brow(g.bits4, bw, b) + w) &
                                   __ldg(brow(g.bits4, bw, c) + w))
                                : 0u;
      const uint32_t fast = z & ~tr & ~risky;
#pragma unroll
      for (int m = 1; m < 8; ++m)
        n[m] += __popc(fast & ((m & 1) ? pa : ~pa) & ((m & 2) ? pb : ~pb) & ((m & 4) ? pc : ~pc));
      uint32_t slow = z & (tr | risky);
      while (slow) {
        const int j = __ffs(slow) - 1;
        slow &= slow - 1;
        const int32_t d = base + w * 32 + j;
        const bool ad = (pa >> j) & 1u, bd = (pb >> j) & 1u, cd = (pc >> j) & 1u;
        bool abd, acd, bcd;
        if (kExact) {
          abd = (r1 >> j) & 1u;
          acd = (r2 >> j) & 1u;
          bcd = (r3 >> j) & 1u;
        } else {
          abd = ((r1 >> j) & 1u) && has_triple(g, a, b, d);
          acd = ((r2 >> j) & 1u) && has_triple(g, a, c, d);
          bcd = ((r3 >> j) & 1u) && has_triple(g, b, c, d);
          if ((abd && d < c) || (acd && d < b) || (bcd && d < a)) continue;
        }
        if (!(ad || bd || cd || abd || acd || bcd)) continue;
        if (((risky >> j) & 1u) && has_quad(g, a, b, c, d)) continue;
        const uint32_t mask = (ab ? 1u : 0u) | (ac ? 2u : 0u) | (ad ? 4u : 0u) | (bc ? 8u : 0u) |
                              (bd ? 16u : 0u) | (cd ? 32u : 0u) | 64u | (abd ? 128u : 0u) |
                              (acd ? 256u : 0u) | (bcd ? 512u : 0u);  // a=0, b=1, c=2, d=3
        const uint8_t c1 = lut[mask], c2 = sub ? lut[mask & 63u] : (uint8_t)0xFF;
        if (kBatched) {
          atomicAdd(&gb[c1], 1u);
          if (c2 != 0xFF) atomicAdd(&gb[c2], 0u - 1u);
        } else {
          atomicAdd(&bins[c1], 1ull);
          if (c2 != 0xFF) atomicAdd(&bins[c2], 0ull - 1ull);
        }
      }
    }
#pragma unroll
    for (int m = 1; m < 8; ++m)
#pragma unroll
      for (int o = 16; o; o >>= 1) n[m] += __shfl_xor_sync(0xffffffffu, n[m], o);
    if (lane == 0) {
      const uint32_t fixed = (ab ? 1u : 0u) | (ac ? 2u : 0u) | (bc ? 8u : 0u) | 64u;
#pragma unroll
      for (int m = 1; m < 8; ++m) {
        if (!n[m]) continue;
        const uint32_t mask =
            fixed | ((m & 1) ? 4u : 0u) | ((m & 2) ? 16u : 0u) | ((m & 4) ? 32u : 0u);
        const uint8_t c1 = lut[mask], c2 = sub ? lut[mask & 63u] : (uint8_t)0xFF;
        if (kBatched) {
          atomicAdd(&gb[c1], n[m]);
          if (c2 != 0xFF) atomicAdd(&gb[c2], 0u - n[m]);
        } else {
          atomicAdd(&bins[c1], (unsigned long long)n[m]);
          if (c2 != 0xFF) atomicAdd(&bins[c2], 0ull - (unsigned long long)n[m]);
        }
      }
    }
  }
  __syncthreads();
  if (kBatched) {
    for (int i = threadIdx.x; i < ngraphs * BIN_STRIDE; i += blockDim.x)
      if (gbins[i])
        atomicAdd(&hist[(i / BIN_STRIDE) * ncls + i % BIN_STRIDE],
                  (unsigned long long)(long long)(int)gbins[i]);
  } else {
    for (int i = threadIdx.x; i < ncls; i += blockDim.x)
      if (bins[i]) atomicAdd(&hist[i], bins[i]);
  }
}

// ---------------------------------------------------------------- work spaces
// Candidates per anchor of up to 8 families in one pass over the anchors.
struct WsArgs {
  int nj;
  char fam[8];
  int64_t A[8];
  uint64_t* out[8];
  uint64_t groups;  // 4-word groups per row (bit-sliced TX items per 3-hyperedge)
};

__global__ void k_ws_all(const int64_t* __restrict__ off2, const int64_t* __restrict__ off3,
                         const uint64_t* __restrict__ e2, const int4* __restrict__ e3,
                         const WsArgs W, int64_t maxA) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < maxA;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < W.nj; ++k) {
      if (i >= W.A[k] || W.fam[k] == 'c' || W.fam[k] == 'o') continue;  // c4_bounds, out_lists
      const char f = W.fam[k];
      uint64_t v = 0;
      if (f == 'W' || f == 'S' || f == 'w' || f == 's') {
        const uint64_t d = (uint64_t)(off2[i + 1] - off2[i]);
        v = f == 'W' ? choose2(d) : f == 'S' ? choose3(d) : f == 'w' ? (d >= 2 ? d : 0) : choose2(d);
      } else if (f == 'P' || f == 'p') {
        const int32_t u = (int32_t)(e2[i] >> 32), x = (int32_t)(e2[i] & 0xFFFFFFFFull);
        const uint64_t du = (uint64_t)(off2[u + 1] - off2[u]), dx = (uint64_t)(off2[x + 1] - off2[x]);
        v = f == 'P' ? (du - 1) * (dx - 1) : (dx > 1 ? du - 1 : 0);
      } else if (f == 'x') {
        v = W.groups;
      } else {
        const int4 e = e3[i];
        const int32_t xs[3] = {e.x, e.y, e.z};
#pragma unroll
        for (int j = 0; j < 3; ++j)
          v += (uint64_t)(off2[xs[j] + 1] - off2[xs[j]]) + (uint64_t)(off3[xs[j] + 1] - off3[xs[j]]);
      }
      W.out[k][i] = v;
    }
  }
}

// TX on graphs without bitmaps, one warp per 3-hyperedge e = {a, b, c}
// (a < b < c). A fourth node d outside e makes the 4-set V' = e + {d}; write
// P(d) for its pairs to a, b, c, T(d) for the 3-hyperedges it forms with two
// members, Q(d) for the 4-hyperedge e + {d}. A pair neighbour d of member x
// is "plain" when P(d) = {x}, T(d) is empty and Q(d) is false: then V' is a
// TX set whose pattern depends only on x, and e is its only 3-hyperedge. So
// plain candidates are counted, not enumerated:
//   plain(x) = d2(x) - (members adjacent to x) - (special pair neighbours of x),
// where the special nodes of e are the d with two or more pairs to e, with a
// 3-hyperedge through two members, or with the 4-hyperedge. They are found
// by six scans, each node kept at its first source only:
//   0-2. N(a) & N(b), N(a) & N(c), N(b) & N(c). With nodes ranked by
//        (degree, id), a common neighbour d of p and q is either above the
//        lower-ranked of the two, r, and so in r's out-list (its neighbours
//        of higher rank), or below both, and then the lowest node of the
//        wedge p - d - q: those come as wedge records, made once per graph
//        from every pair of every out-list that is the member pair of exactly
//        one 3-hyperedge. So r's out-list is scanned, membership in the other
//        row by a signature test and a probe, and the records are read; a
//        member pair inside two or more 3-hyperedges has no records, and its
//        shorter row is scanned whole instead;
//   3-5. the third nodes of the 3-hyperedges through (a, b), (a, c), (b, c):
//        the shorter of the two members' incidence lists scanned, for the
//        member pairs that lie in another 3-hyperedge too (the others have
//        none);
//   6.   where the three members' 4-hyperedge signatures share a bit and a
//        Bloom filter of the 4-hyperedges' 3-subsets does not rule e out, the
//        pair neighbours d of each member with Q(d) (others are found above).
// Each special d gets its full P, T and Q by probes (a signature test first),
// adds to the special count of every member it is a pair neighbour of, and is
// counted when V' is a TX set of this anchor: no 4-hyperedge, and e the
// smallest 3-hyperedge of V' ({a,b,d} < e iff d < c, {a,c,d} < e iff d < b,
// {b,c,d} < e iff d < a). The three pair sources and the records form one
// index space over the group's lanes, so that short lists take one round;
// member indices are three-way selects, so the per-member state stays in
// registers, and all sources share one call site of the candidate code.
struct TxsAnchor {
  int32_t m0, m1, m2;
  int32_t od0, od1, od2;  // out-list lengths
  int64_t o20, o21, o22;
  int32_t d20, d21, d22;
  uint64_t s20, s21, s22, s30, s31, s32, s4;
  bool pab, pac, pbc;
};

template <class T>
__device__ __forceinline__ T sel3(int i, T x0, T x1, T x2) {
  return i == 0 ? x0 : (i == 1 ? x1 : x2);
}

struct TxsBins {
  unsigned long long* bins;
  const uint8_t* lut;
  int sub;
  __device__ void count(uint32_t mask, unsigned long long n) const {
    const uint8_t c1 = lut[mask];
    if (c1 != 0xFF) atomicAdd(&bins[c1], n);
    if (sub) {
      const uint8_t c2 = lut[mask & 63u];
      if (c2 != 0xFF) atomicAdd(&bins[c2], 0ull - n);
    }
  }
};

// One candidate d of source src (0-2 pair intersections of members (0,1),
// (0,2), (1,2); 3-5 third nodes of 3-hyperedges through the same pairs;
// 6-8 quad scan of member src - 6); kp: pair bits known to be set. Adds to
// the special counts sp0..sp2 and counts the set when it is a TX set of this
// anchor.
__device__ __forceinline__ void txs_candidate(const DevGraph& g, const TxsAnchor& A, int src,
                                              int32_t d, uint32_t kp, const TxsBins& B,
                                              uint32_t& sp0, uint32_t& sp1, uint32_t& sp2) {
  const int32_t a = A.m0, b = A.m1, c = A.m2;
  if (d == a || d == b || d == c) return;
  const uint64_t db = sig_bit(d);
  bool Q = false;
  if (src >= 6) {  // quad scan: only the nodes that close the 4-hyperedge
    Q = (A.s4 & db) && has_quad(g, a, b, c, d);
    if (!Q) return;
  }
  const bool p0 = (kp & 1u) || ((A.s20 & db) && has_pair(g, a, d));
  const bool p1 = (kp & 2u) || ((A.s21 & db) && has_pair(g, b, d));
  const bool p2 = (kp & 4u) || ((A.s22 & db) && has_pair(g, c, d));
  if (src == 0 && !(p0 && p1)) return;
  if (src == 1 && (!(p0 && p2) || p1)) return;
  if (src == 2 && (!(p1 && p2) || p0)) return;
  const int np = (p0 ? 1 : 0) + (p1 ? 1 : 0) + (p2 ? 1 : 0);
  if (src >= 3 && np >= 2) return;  // found by a pair intersection
  const bool t01 = src == 3 || ((A.s30 & A.s31 & db) && has_triple(g, a, b, d));
  if (src == 4 && t01) return;
  const bool t02 = src == 4 || ((A.s30 & A.s32 & db) && has_triple(g, a, c, d));
  if (src == 5 && (t01 || t02)) return;
  const bool t12 = src == 5 || ((A.s31 & A.s32 & db) && has_triple(g, b, c, d));
  if (src >= 6 && (t01 || t02 || t12)) return;  // found by a triple scan
  if (src < 6) Q = (A.s4 & db) && has_quad(g, a, b, c, d);
  sp0 += p0 ? 1u : 0u;
  sp1 += p1 ? 1u : 0u;
  sp2 += p2 ? 1u : 0u;
  if (Q) return;  // family Q
  if ((t01 && d < c) || (t02 && d < b) || (t12 && d < a)) return;  // a smaller 3-hyperedge
  const uint32_t mask = (A.pab ? 1u : 0u) | (A.pac ? 2u : 0u) | (p0 ? 4u : 0u) |
                        (A.pbc ? 8u : 0u) | (p1 ? 16u : 0u) | (p2 ? 32u : 0u) | 64u |
                        (t01 ? 128u : 0u) | (t02 ? 256u : 0u) | (t12 ? 512u : 0u);
  B.count(mask, 1ull);
}

// The list of pair source j (member pair (p, q): 0 (a, b), 1 (a, c), 2 (b, c)):
// for a pair inside another 3-hyperedge too, the shorter of the two rows;
// else the out-list of the lower-ranked member (the wedges below both come as
// records). kp: the member known to be adjacent.
__device__ __forceinline__ void txs_pair_list(const TxsAnchor& A, uint32_t shared, int j,
                                              int64_t& o, int32_t& len, uint32_t& kp,
                                              bool& out) {
  const int p = j == 2 ? 1 : 0, q = j == 0 ? 1 : 2;
  const int32_t lp = sel3(p, A.d20, A.d21, A.d22), lq = sel3(q, A.d20, A.d21, A.d22);
  int r;
  out = !((shared >> j) & 1u);
  if (out)
    r = (lp < lq || (lp == lq && sel3(p, A.m0, A.m1, A.m2) < sel3(q, A.m0, A.m1, A.m2))) ? p : q;
  else
    r = lp <= lq ? p : q;
  o = sel3(r, A.o20, A.o21, A.o22);
  len = out ? sel3(r, A.od0, A.od1, A.od2) : sel3(r, A.d20, A.d21, A.d22);
  kp = 1u << r;
}

#ifndef HM_TXS_MINBLOCKS
#define HM_TXS_MINBLOCKS 4
#endif
// One persistent kernel over two lists of 3-hyperedges: the warp list (a warp
// per 3-hyperedge) and the short list (8 lanes per 3-hyperedge, four per
// warp, for those whose lists are all short). Warps take work from two
// counters: one 3-hyperedge of the warp list at a time, then chunks of
// TXS_CHUNK of the short list, so that warps done with the long 3-hyperedges
// (few, taken first) go on to short ones and no long one is left for the
// end. G, the lanes per 3-hyperedge, is a run-time value (32 or 8), so one
// copy of the code serves both. The only cross-lane operations (the pairs
// inside e, the special-count sums) stay within a group.
constexpr uint32_t TXS_CHUNK = 32;
__global__ void __launch_bounds__(CENSUS_THREADS, HM_TXS_MINBLOCKS)
    k_census_txs(const DevGraph g, const int32_t* __restrict__ large,
                 const int32_t* __restrict__ small, unsigned int* __restrict__ counts,
                 const uint8_t* __restrict__ share, const int32_t* __restrict__ out_deg,
                 const int32_t* __restrict__ out_adj, const uint64_t* __restrict__ rec,
                 const int64_t* __restrict__ rs, const int64_t* __restrict__ re,
                 const uint8_t* __restrict__ lut_g, int nmask, int ncls, int sub,
                 unsigned long long* __restrict__ hist) {
  __shared__ unsigned long long bins[BIN_STRIDE];
  __shared__ __align__(16) uint8_t lut[2048];
  load_lut(lut, lut_g, nmask);
  for (int i = threadIdx.x; i < ncls; i += blockDim.x) bins[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const TxsBins B{bins, lut, sub};
  // counts: [0] short list size, [1] warp list size, [2] / [3] their work counters
  const uint32_t nsmall = counts[0], nlarge = counts[1];
  uint32_t base = 0, rounds = 0;
  int G = 32;
  bool large_done = false;
  for (;;) {
    if (rounds == 0) {  // the warp's next piece of work (warp-uniform)
      uint32_t got = 0;
      if (!large_done) {
        if (lane == 0) got = atomicAdd(&counts[3], 1u);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got < nlarge) {
          base = got;
          rounds = 1;
          G = 32;
        } else {
          large_done = true;
        }
      }
      if (large_done) {
        if (lane == 0) got = atomicAdd(&counts[2], TXS_CHUNK);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got >= nsmall) break;
        base = got;
        rounds = TXS_CHUNK / 4;
        G = 8;
      }
    }
    const int glane = lane & (G - 1), gbase = lane - glane;
    const unsigned gmask = G == 32 ? 0xffffffffu : (0xFFu << gbase);
    int64_t t = -1;
    if (G == 32) {
      t = large[base];
    } else {
      const uint32_t idx = base + (TXS_CHUNK / 4 - rounds) * 4 + (uint32_t)(lane >> 3);
      if (idx < nsmall) t = small[idx];
    }
    --rounds;
    if (t < 0) continue;  // a group with no 3-hyperedge this round
    TxsAnchor A;
    const int4 e = g.e3[t];
    A.m0 = e.x;
    A.m1 = e.y;
    A.m2 = e.z;
    A.od0 = out_deg[e.x];
    A.od1 = out_deg[e.y];
    A.od2 = out_deg[e.z];
    A.o20 = g.off2[e.x];
    A.o21 = g.off2[e.y];
    A.o22 = g.off2[e.z];
    A.d20 = (int32_t)(g.off2[e.x + 1] - A.o20);
    A.d21 = (int32_t)(g.off2[e.y + 1] - A.o21);
    A.d22 = (int32_t)(g.off2[e.z + 1] - A.o22);
    A.s20 = g.sig[e.x];
    A.s21 = g.sig[e.y];
    A.s22 = g.sig[e.z];
    A.s30 = g.sig[(int64_t)g.n + e.x];
    A.s31 = g.sig[(int64_t)g.n + e.y];
    A.s32 = g.sig[(int64_t)g.n + e.z];
    A.s4 = g.sig[2 * (int64_t)g.n + e.x] & g.sig[2 * (int64_t)g.n + e.y] &
           g.sig[2 * (int64_t)g.n + e.z];
    // the pairs inside e: group lanes 0-2 probe, the group shares
    bool mine = false;
    if (glane < 3) {  // lane 0: {a, b}, 1: {a, c}, 2: {b, c}
      const int32_t u = glane == 2 ? e.y : e.x, v = glane == 0 ? e.y : e.z;
      mine = ((glane == 2 ? A.s21 : A.s20) & sig_bit(v)) && has_pair(g, u, v);
    }
    const unsigned pb = (__ballot_sync(gmask, mine) >> gbase) & 7u;
    A.pab = pb & 1u;
    A.pac = pb & 2u;
    A.pbc = pb & 4u;
    uint32_t sp0 = 0, sp1 = 0, sp2 = 0;
    const uint32_t shared = share[t];
    const int64_t r0 = rs[t];
    const int32_t lr = (int32_t)(re[t] - r0 < 0x7FFFFFFF ? re[t] - r0 : 0x7FFFFFFF);
    int32_t l0, l1, l2;
    {
      int64_t o;
      uint32_t kp;
      bool out;
      txs_pair_list(A, shared, 0, o, l0, kp, out);
      txs_pair_list(A, shared, 1, o, l1, kp, out);
      txs_pair_list(A, shared, 2, o, l2, kp, out);
    }
    // Segment 0: the three pair sources and the wedge records, one index
    // space over the group's lanes (most lists are short); 1-3: the third
    // nodes of a member pair inside another 3-hyperedge (sources 3-5); 4-6:
    // the quad scans (sources 6-8) where the filters allow.
#pragma unroll 1
    for (int seg = 0; seg < 7; ++seg) {
      if (seg >= 1 && seg <= 3 && !((shared >> (seg - 1)) & 1u)) continue;
      if (seg >= 4 && !(shared & 8u)) continue;
      const int src = seg + 2;  // sources 3-8
      const int p = src < 6 ? (src % 3 == 2 ? 1 : 0) : src - 6;
      const int q = src % 3 == 0 ? 1 : 2;
      int64_t o = 0;
      int32_t len;
      int32_t mp = 0, mq = 0;
      if (seg == 0) {
        len = l0 + l1 + l2 + lr;
      } else if (seg <= 3) {  // the shorter of the two incidence lists
        mp = sel3(p, A.m0, A.m1, A.m2);
        mq = sel3(q, A.m0, A.m1, A.m2);
        const int64_t op = g.off3[mp], oq = g.off3[mq];
        const int32_t lp = (int32_t)(g.off3[mp + 1] - op), lq = (int32_t)(g.off3[mq + 1] - oq);
        o = lp <= lq ? op : oq;
        len = lp <= lq ? lp : lq;
      } else {  // member p's pair row
        o = sel3(p, A.o20, A.o21, A.o22);
        len = sel3(p, A.d20, A.d21, A.d22);
      }
      for (int32_t i0 = 0; i0 < len; i0 += G) {
        int32_t idx = i0 + glane;
        if (idx >= len) continue;
        int32_t d;
        int csrc = src;
        uint32_t kpx = 1u << p;
        if (seg == 0) {
          if (idx < l0 + l1 + l2) {
            csrc = idx < l0 ? 0 : (idx < l0 + l1 ? 1 : 2);
            idx -= csrc == 0 ? 0 : (csrc == 1 ? l0 : l0 + l1);
            int64_t ol;
            int32_t ll;
            bool out;
            txs_pair_list(A, shared, csrc, ol, ll, kpx, out);
            d = __ldg((out ? out_adj : g.adj2) + ol + idx);
          } else {  // a wedge record: d adjacent to both members of pair csrc
            const uint64_t r = __ldg(rec + r0 + (idx - l0 - l1 - l2));
            d = (int32_t)(r >> 33);
            csrc = (int)((r >> 31) & 3u);
            kpx = csrc == 0 ? 3u : (csrc == 1 ? 5u : 6u);
          }
        } else if (seg <= 3) {
          const int64_t th = __ldg(g.inc3 + o + idx);
          if (th == t) continue;
          const int4 h = g.e3[th];
          const bool hp = h.x == mp || h.y == mp || h.z == mp;
          const bool hq = h.x == mq || h.y == mq || h.z == mq;
          if (!hp || !hq) continue;
          d = (h.x != mp && h.x != mq) ? h.x : (h.y != mp && h.y != mq) ? h.y : h.z;
          kpx = 0;
        } else {
          d = __ldg(g.adj2 + o + idx);
        }
        txs_candidate(g, A, csrc, d, kpx, B, sp0, sp1, sp2);
      }
    }
    for (int o = G / 2; o; o >>= 1) {
      sp0 += __shfl_xor_sync(gmask, sp0, o);
      sp1 += __shfl_xor_sync(gmask, sp1, o);
      sp2 += __shfl_xor_sync(gmask, sp2, o);
    }
    if (glane == 0) {
      const uint32_t fixed = (A.pab ? 1u : 0u) | (A.pac ? 2u : 0u) | (A.pbc ? 8u : 0u) | 64u;
      const unsigned long long pa =
          (unsigned long long)A.d20 - (A.pab ? 1 : 0) - (A.pac ? 1 : 0) - sp0;
      const unsigned long long pbn =
          (unsigned long long)A.d21 - (A.pab ? 1 : 0) - (A.pbc ? 1 : 0) - sp1;
      const unsigned long long pc =
          (unsigned long long)A.d22 - (A.pac ? 1 : 0) - (A.pbc ? 1 : 0) - sp2;
      if (pa) B.count(fixed | 4u, pa);
      if (pbn) B.count(fixed | 16u, pbn);
      if (pc) B.count(fixed | 32u, pc);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ncls; i += blockDim.x)
    if (bins[i]) atomicAdd(&hist[i], bins[i]);
}

// The member pairs of the 3-hyperedges: an open-addressing set of pair keys
// whose top bit (free: node ids are below 2^31) marks a pair inside two or
// more 3-hyperedges. A pair inside e only has third nodes other than e's to
// scan for (sources 3-5 of k_census_txs) when it is so marked, and few are.
constexpr uint64_t TP_SHARED = 1ull << 63;

__device__ __forceinline__ void tp_insert(unsigned long long* tab, int32_t* val, uint64_t mask,
                                          uint64_t key, int32_t v) {
  uint64_t slot = hash_pair(key) & mask;
  for (uint64_t it = 0; it <= mask; ++it) {
    const unsigned long long prev = atomicCAS(tab + slot, EMPTY64, key);
    if (prev == EMPTY64) {
      val[slot] = v;
      return;
    }
    if ((prev & ~TP_SHARED) == key) {
      if (!(prev & TP_SHARED)) atomicOr(tab + slot, TP_SHARED);
      return;
    }
    slot = (slot + 1) & mask;
  }
}

// The slot of a pair of the set, or -1.
__device__ __forceinline__ int64_t tp_find(const unsigned long long* tab, uint64_t mask,
                                           uint64_t key) {
  uint64_t slot = hash_pair(key) & mask;
  for (uint64_t it = 0; it <= mask; ++it) {
    const unsigned long long v = tab[slot];
    if ((v & ~TP_SHARED) == key) return (int64_t)slot;
    if (v == EMPTY64) return -1;
    slot = (slot + 1) & mask;
  }
  return -1;
}

// Whether the pair lies in two or more 3-hyperedges (true when it is not
// found, which cannot happen for a member pair: scanning is always safe).
__device__ __forceinline__ bool tp_shared(const unsigned long long* tab, uint64_t mask,
                                          uint64_t key) {
  uint64_t slot = hash_pair(key) & mask;
  for (uint64_t it = 0; it <= mask; ++it) {
    const unsigned long long v = tab[slot];
    if ((v & ~TP_SHARED) == key) return (v & TP_SHARED) != 0;
    if (v == EMPTY64) return true;
    slot = (slot + 1) & mask;
  }
  return true;
}

// A Bloom filter of the 3-subsets of the 4-hyperedges (two bits of a
// nbits-bit array per subset, nbits a power of two): a clear bit proves that
// no 4-hyperedge contains the 3-hyperedge, so that it has no quad scan.
__device__ __forceinline__ uint64_t tq_hash(int32_t a, int32_t b, int32_t c) {
  return hash_tuple(a, b, c, -1);
}

__global__ void k_tq_bloom(const DevGraph g, uint32_t* __restrict__ bloom, uint32_t nbits) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.m4;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 e = g.e4[t];  // a < b < c < d
    const int32_t m[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
    for (int skip = 0; skip < 4; ++skip) {
      int32_t k3[3];
      int j = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i != skip) k3[j++] = m[i];
      const uint64_t h = tq_hash(k3[0], k3[1], k3[2]);
      const uint32_t b0 = (uint32_t)h & (nbits - 1u), b1 = (uint32_t)(h >> 32) & (nbits - 1u);
      atomicOr(&bloom[b0 >> 5], 1u << (b0 & 31));
      atomicOr(&bloom[b1 >> 5], 1u << (b1 & 31));
    }
  }
}

// The value of a pair is 4 t + j for the first 3-hyperedge t inserting it, j
// its member pair (0: (a, b), 1: (a, c), 2: (b, c)); it is read only for
// unflagged pairs, which have one 3-hyperedge.
__global__ void k_tp_insert(const DevGraph g, unsigned long long* __restrict__ tab,
                            int32_t* __restrict__ val, uint64_t mask) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < g.m3;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 e = g.e3[t];
    tp_insert(tab, val, mask, pair_key(e.x, e.y), (int32_t)(4 * t + 0));
    tp_insert(tab, val, mask, pair_key(e.x, e.z), (int32_t)(4 * t + 1));
    tp_insert(tab, val, mask, pair_key(e.y, e.z), (int32_t)(4 * t + 2));
  }
}

// Wedge records: a common pair neighbour d of a member pair (p, q) that is
// ranked below both is the lowest node of the wedge p - d - q, so p and q
// both lie in out(d). Item k of the TXO space (node d, pair (i, j) of its
// out-list) writes record k: (d << 33) | (j << 31) | t when the pair is the
// member pair j of exactly one 3-hyperedge t (an unflagged pair of the set),
// else REC_NONE. A warp takes 32 consecutive nodes and spreads their pairs
// over its lanes.
constexpr uint64_t REC_NONE = ~0ull;
constexpr uint64_t REC_T = (1ull << 31) - 1;
__global__ void __launch_bounds__(256)
    k_txs_wedges(const DevGraph g, const int32_t* __restrict__ out_deg,
                 const int32_t* __restrict__ out_adj, const uint64_t* __restrict__ ws,
                 const unsigned long long* __restrict__ tab, const int32_t* __restrict__ val,
                 uint64_t mask, uint64_t* __restrict__ rec) {
  __shared__ uint64_t pre_s[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t* pre = pre_s[wid];
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c0 = gw * 32; c0 < g.n; c0 += warps * 32) {
    const int64_t dl = c0 + lane;
    const uint64_t k = dl < g.n ? (uint64_t)out_deg[dl] : 0;
    const uint64_t np = k * (k - (k > 0 ? 1 : 0)) / 2;
    uint64_t incl = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    pre[lane] = incl - np;
    const uint64_t tot = __shfl_sync(0xffffffffu, incl, 31);
    const uint64_t base = ws[c0];
    __syncwarp();
    for (uint64_t p = lane; p < tot; p += 32) {
      int lo = 0, hi = 32;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= p) lo = mid;
        else hi = mid;
      }
      const int32_t d = (int32_t)(c0 + lo);
      uint32_t i, j;
      unrank2(p - pre[lo], i, j);
      const int64_t od = g.off2[d];
      const int32_t x = out_adj[od + i], y = out_adj[od + j];
      uint64_t r = REC_NONE;
      const int64_t sl = tp_find(tab, mask, pair_key(x, y));
      if (sl >= 0 && !(tab[sl] & TP_SHARED)) {
        const uint32_t v = (uint32_t)val[sl];
        r = ((uint64_t)(uint32_t)d << 33) | ((uint64_t)(v & 3u) << 31) | (uint64_t)(v >> 2);
      }
      rec[base + p] = r;
    }
    __syncwarp();
  }
}

// Records grouped by 3-hyperedge without a sort (their order within a
// 3-hyperedge does not matter): counts per t into the zeroed rs, an exclusive
// scan of rs (so t's records are [rs[t], rs[t + 1])), then each record placed
// at rs[t] plus a per-t cursor.
__global__ void k_txs_rec_count(const uint64_t* __restrict__ rec, uint64_t nrec,
                                unsigned long long* __restrict__ cnt) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nrec;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = rec[i];
    if (r != REC_NONE) atomicAdd(&cnt[r & REC_T], 1ull);
  }
}

__global__ void k_txs_rec_place(const uint64_t* __restrict__ rec, uint64_t nrec,
                                const int64_t* __restrict__ rs, unsigned int* __restrict__ cur,
                                uint64_t* __restrict__ out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nrec;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = rec[i];
    if (r == REC_NONE) continue;
    const uint64_t t = r & REC_T;
    out[rs[t] + atomicAdd(&cur[t], 1u)] = r;
  }
}


// Splits E_3 for k_census_txs: a 3-hyperedge whose every scanned list (per
// member pair, the out-list of its lower-ranked member or, for a pair inside
// another 3-hyperedge too, the shorter row and the shorter incidence list;
// its wedge records; each member's row where the 4-hyperedge signatures
// meet) has at most TXS_SMALL entries goes to the 8-lane list, the others to
// the warp list. share[t] gets the member pairs
// that lie in another 3-hyperedge (bit 0: (a, b), 1: (a, c), 2: (b, c)) and
// bit 3 when the quad scans run: the members' 4-hyperedge signatures meet and
// the Bloom filter does not rule out a 4-hyperedge containing e.
#ifndef HM_TXS_SMALL
#define HM_TXS_SMALL 32
#endif
constexpr int TXS_SMALL = HM_TXS_SMALL;
__global__ void k_txs_split(const DevGraph g, const unsigned long long* __restrict__ tab,
                            uint64_t mask, const uint32_t* __restrict__ bloom, uint32_t nbits,
                            const int32_t* __restrict__ out_deg, const int64_t* __restrict__ rs,
                            const int64_t* __restrict__ re, uint8_t* __restrict__ share,
                            int32_t* __restrict__ small, int32_t* __restrict__ large,
                            unsigned int* __restrict__ counts) {
  __shared__ unsigned int wcnt[2][32], bbase[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // whole blocks per round (the appends take one atomic per list per block)
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < g.m3;
       t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = t0 + threadIdx.x;
    bool valid = t < g.m3, is_small = false;
    if (valid) {
      const int4 e = g.e3[t];
      const int32_t m[3] = {e.x, e.y, e.z};
      int32_t d2[3], d3[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        d2[j] = (int32_t)(g.off2[m[j] + 1] - g.off2[m[j]]);
        d3[j] = (int32_t)(g.off3[m[j] + 1] - g.off3[m[j]]);
      }
      const bool s01 = tp_shared(tab, mask, pair_key(e.x, e.y));
      const bool s02 = tp_shared(tab, mask, pair_key(e.x, e.z));
      const bool s12 = tp_shared(tab, mask, pair_key(e.y, e.z));
      const uint64_t s4 = g.sig[2 * (int64_t)g.n + e.x] & g.sig[2 * (int64_t)g.n + e.y] &
                          g.sig[2 * (int64_t)g.n + e.z];
      bool quad = s4 != 0;
      if (quad) {
        const uint64_t h = tq_hash(e.x, e.y, e.z);
        const uint32_t b0 = (uint32_t)h & (nbits - 1u), b1 = (uint32_t)(h >> 32) & (nbits - 1u);
        quad = ((bloom[b0 >> 5] >> (b0 & 31)) & 1u) && ((bloom[b1 >> 5] >> (b1 & 31)) & 1u);
      }
      share[t] = (uint8_t)((s01 ? 1u : 0u) | (s02 ? 2u : 0u) | (s12 ? 4u : 0u) | (quad ? 8u : 0u));
      // per member pair: the out-list of its lower-ranked member, or for a
      // shared pair the shorter row and the shorter incidence list
      auto low = [&](int i, int j) { return d2[i] < d2[j] || (d2[i] == d2[j] && m[i] < m[j]) ? i : j; };
      const int64_t nr = re[t] - rs[t];
      int32_t mx = (int32_t)(nr < (1 << 30) ? nr : (1 << 30));
      mx = max(mx, s01 ? max(min(d2[0], d2[1]), min(d3[0], d3[1])) : out_deg[m[low(0, 1)]]);
      mx = max(mx, s02 ? max(min(d2[0], d2[2]), min(d3[0], d3[2])) : out_deg[m[low(0, 2)]]);
      mx = max(mx, s12 ? max(min(d2[1], d2[2]), min(d3[1], d3[2])) : out_deg[m[low(1, 2)]]);
      if (quad) mx = max(mx, max(d2[0], max(d2[1], d2[2])));
      is_small = mx <= TXS_SMALL;
    }
    // block-aggregated appends: warp counts, one atomic per list, warp offsets
    const unsigned bs = __ballot_sync(0xffffffffu, valid && is_small);
    const unsigned bl = __ballot_sync(0xffffffffu, valid && !is_small);
    if (lane == 0) {
      wcnt[0][wid] = (unsigned)__popc(bs);
      wcnt[1][wid] = (unsigned)__popc(bl);
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      const int k = threadIdx.x;
      unsigned run = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        const unsigned c = wcnt[k][w];
        wcnt[k][w] = run;
        run += c;
      }
      bbase[k] = run ? atomicAdd(&counts[k], run) : 0u;
    }
    __syncthreads();
    const unsigned base_s = bbase[0] + wcnt[0][wid], base_l = bbase[1] + wcnt[1][wid];
    __syncthreads();  // wcnt and bbase are rewritten next round
    const unsigned below = (1u << lane) - 1u;
    if (valid && is_small) small[base_s + __popc(bs & below)] = (int32_t)t;
    if (valid && !is_small) large[base_l + __popc(bl & below)] = (int32_t)t;
  }
}

unsigned grid1d(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

// Out-lists: each pair (u, v) goes to the out-list of its lower-ranked end
// (rank = (degree, id)), at that node's next free slot.
__global__ void k_out_fill(const DevGraph g, int32_t* __restrict__ out_deg,
                           int32_t* __restrict__ out_adj) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < g.m2;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t e = g.e2[p];
    const int32_t u = (int32_t)(e >> 32), v = (int32_t)(e & 0xFFFFFFFFull);
    const int32_t du = (int32_t)(g.off2[u + 1] - g.off2[u]);
    const int32_t dv = (int32_t)(g.off2[v + 1] - g.off2[v]);
    const bool u_low = du < dv || (du == dv && u < v);
    const int32_t lo = u_low ? u : v, hi = u_low ? v : u;
    const int32_t at = atomicAdd(&out_deg[lo], 1);
    out_adj[g.off2[lo] + at] = hi;
  }
}

__global__ void k_out_pairs(const int32_t* __restrict__ out_deg, int64_t n,
                            uint64_t* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = (uint64_t)out_deg[v];
    out[v] = k * (k - (k > 0 ? 1 : 0)) / 2;
  }
}

}  // namespace

void out_lists(hm_graph* g, uint64_t* out, cudaStream_t s) {
  if (!g->out_deg) {
    g->out_deg = dalloc<int32_t>((size_t)g->n, s);
    g->owned.push_back(g->out_deg);
    g->out_adj = dalloc<int32_t>(std::max<size_t>(1, (size_t)2 * g->counts[2]), s);
    g->owned.push_back(g->out_adj);
  }
  HM_CUDA(cudaMemsetAsync(g->out_deg, 0, (size_t)g->n * sizeof(int32_t), s));
  if (g->counts[2]) {
    k_out_fill<<<grid1d(g->counts[2]), 256, 0, s>>>(g->view(), g->out_deg, g->out_adj);
    HM_KCHECK();
  }
  k_out_pairs<<<grid1d(g->n), 256, 0, s>>>(g->out_deg, g->n, out);
  HM_KCHECK();
}

// Prefix sums of the candidates per anchor for every family in `todo` that is
// not ready: enqueued on s (one temporary for all families), with the totals
// copied to P.h; spaces_finish, after s has completed, marks them ready.
void spaces_enqueue(hm_graph* g, const std::vector<std::pair<hm_graph::Space*, char>>& todo,
                    cudaStream_t s, PendingSpaces& P) {
  P.g = g;
  P.need.clear();
  P.made.clear();
  for (auto& t : todo)
    if (!t.first->ready) P.need.push_back(t);
  if (P.need.empty()) return;
  const int nj = (int)P.need.size();
  HM_CHECK(nj <= 8, HM_EINVAL, "too many work spaces");
  // one allocation: the scan's scratch (zeroed), the totals, then the
  // prefix-sum arrays (anchors + 1 entries each)
  WsArgs W{};
  W.nj = nj;
  W.groups = (uint64_t)(g->bwords / 4);
  int64_t maxA = 0;
  size_t off[8];
  ScanJob jobs[8];
  for (int i = 0; i < nj; ++i) {
    const char fam = P.need[i].second;
    int64_t a = 0;
    if (fam == 'W' || fam == 'S' || fam == 'w' || fam == 's' || fam == 'c' || fam == 'o') a = g->n;
    if (fam == 'P' || fam == 'p') a = g->counts[2];
    if (fam == 'X' || fam == 'x') a = g->kmax >= 3 ? g->counts[3] : 0;
    W.fam[i] = fam;
    W.A[i] = a;
    maxA = std::max(maxA, a);
    jobs[i].n = a;
  }
  // scan_batch_scratch reads only the sizes
  const size_t scan_bytes = (scan_batch_scratch(jobs, nj) + 255) & ~(size_t)255;
  size_t bytes = scan_bytes + 256;  // totals
  for (int i = 0; i < nj; ++i) {
    off[i] = bytes;
    bytes += (((size_t)W.A[i] + 1) * sizeof(uint64_t) + 255) & ~(size_t)255;
  }
  unsigned char* base = dalloc<unsigned char>(bytes, s);
  P.made.push_back(reinterpret_cast<uint64_t*>(base));
  try {
    uint64_t* totals = reinterpret_cast<uint64_t*>(base + scan_bytes);
    for (int i = 0; i < nj; ++i) {
      W.out[i] = reinterpret_cast<uint64_t*>(base + off[i]);
      jobs[i].a = W.out[i];
      jobs[i].total = totals + i;
      P.ws[i] = W.out[i];
      P.need[i].first->anchors = W.A[i];
    }
    if (scan_bytes) HM_CUDA(cudaMemsetAsync(base, 0, scan_bytes, s));
    if (maxA > 0) {
      k_ws_all<<<grid1d(maxA), 256, 0, s>>>(g->off2, g->off3, g->e2, g->e3, W, maxA);
      HM_KCHECK();
    }
    for (int i = 0; i < nj; ++i)
      if (W.fam[i] == 'c' && W.A[i] > 0) c4_bounds(g, W.out[i], s);
    for (int i = 0; i < nj; ++i)
      if (W.fam[i] == 'o' && W.A[i] > 0) out_lists(g, W.out[i], s);
    scan_batch_inplace(jobs, nj, s, scan_bytes ? base : nullptr, true);
    P.h = pinned_words() + 64;
    HM_CUDA(cudaMemcpyAsync(P.h, totals, nj * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  } catch (...) {
    for (uint64_t* p : P.made) cudaFreeAsync(p, s);
    P.made.clear();
    P.need.clear();
    throw;
  }
}

void spaces_finish(PendingSpaces& P) {
  for (size_t i = 0; i < P.need.size(); ++i) {
    P.need[i].first->ws = P.ws[i];
    P.need[i].first->total = P.h[i];
    P.need[i].first->ready = true;
  }
  for (uint64_t* p : P.made) P.g->owned.push_back(p);
  P.need.clear();
  P.made.clear();
}

namespace {

void ensure_spaces(hm_graph* g, const std::vector<std::pair<hm_graph::Space*, char>>& todo,
                   cudaStream_t s) {
  PendingSpaces P;
  spaces_enqueue(g, todo, s, P);
  if (P.need.empty()) return;
  try {
    HM_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    for (uint64_t* p : P.made) cudaFreeAsync(p, s);
    throw;
  }
  spaces_finish(P);
}

// Persistent grid: SMs x resident blocks, capped by the work; with a union
// of graphs, enough blocks that no block counts 2^31 candidates.
// SM count and resident blocks per SM of a census kernel on the current
// device, queried once per (kernel, device).
void resident_blocks(const void* kernel, int& sms, int& per_sm) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, std::pair<int, int>> cache;
  int dev = 0;
  HM_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({kernel, dev});
    if (it != cache.end()) {
      sms = it->second.first;
      per_sm = it->second.second;
      return;
    }
  }
  HM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, CENSUS_THREADS, 0));
  std::lock_guard<std::mutex> lock(mu);
  cache[{kernel, dev}] = {sms, per_sm};
}

int grid_for(const void* kernel, uint64_t lanes_needed, uint64_t max_candidates, bool batched) {
  int sms = 0, per_sm = 0;
  resident_blocks(kernel, sms, per_sm);
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

// Launch one family over its index range [begin, end) (items for bit-sliced
// families, candidates otherwise). chunk = candidates per lane of a
// per-candidate family; 0 = as many as fill the GPU, at most CHUNK.
template <class F, bool kBatched>
void launch_bits_t(const hm_graph* g, const F& fam, const hm_graph::Space& sp, uint64_t begin,
                   uint64_t end, int order, unsigned long long* hist, cudaStream_t s,
                   bool traced) {
  const ClassTables& T = class_tables(order);
  const uint8_t* lut = device_lut(order);
  const uint64_t lanes = (end - begin + BITS_CHUNK - 1) / BITS_CHUNK;
  const uint64_t max_cand = (end - begin) * (uint64_t)g->bwords * 32;
  const int blocks = grid_for((const void*)k_census_bits<F, kBatched>, lanes, max_cand, kBatched);
  cudaEvent_t ev = nullptr;
  const bool tr = traced && trace_on(F::kName);
  if (tr) trace_begin(s, &ev);
  k_census_bits<F, kBatched><<<blocks, CENSUS_THREADS, 0, s>>>(
      g->view(), fam, sp.ws, sp.anchors, begin, end, lut, (int)T.lut.size(), T.ncls,
      num_graphs(g), hist);
  HM_KCHECK();
  if (tr) trace_end(F::kName, s, ev);
}

template <class F>
void launch_bits(const hm_graph* g, const F& fam, const hm_graph::Space& sp, int order,
                 unsigned long long* hist, cudaStream_t s, uint64_t begin = 0,
                 uint64_t end = ~0ull, bool traced = true) {
  if (end > sp.total) end = sp.total;
  if (begin >= end) return;
  if (g->block)
    launch_bits_t<F, true>(g, fam, sp, begin, end, order, hist, s, traced);
  else
    launch_bits_t<F, false>(g, fam, sp, begin, end, order, hist, s, traced);
}

int fill_chunk(uint64_t candidates) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const uint64_t lanes_wanted = (uint64_t)sms * 2048;
  const int chunk = (int)std::min<uint64_t>(CHUNK, (candidates + lanes_wanted - 1) / lanes_wanted);
  return chunk < 1 ? 1 : chunk;
}

template <class F, bool kBatched>
void launch_family_t(const hm_graph* g, const F& fam, const hm_graph::Space* sp, uint64_t begin,
                     uint64_t end, int chunk, int order, unsigned long long* hist,
                     cudaStream_t s, bool traced, int sub) {
  const ClassTables& T = class_tables(order);
  const uint8_t* lut = device_lut(order);
  // consecutive candidates per lane (every lane of a warp takes the same)
  if (chunk <= 0) chunk = fill_chunk(end - begin);
  if (chunk > CHUNK) chunk = CHUNK;
  const int blocks = grid_for((const void*)k_census<F, kBatched>, (end - begin + chunk - 1) / chunk,
                              end - begin, kBatched);
  cudaEvent_t ev = nullptr;
  const bool tr = traced && trace_on(F::kName);
  if (tr) trace_begin(s, &ev);
  k_census<F, kBatched><<<blocks, CENSUS_THREADS, 0, s>>>(
      g->view(), fam, sp ? sp->ws : nullptr, sp ? sp->anchors : 0, begin, end, chunk, lut,
      (int)T.lut.size(), T.ncls, num_graphs(g), sub, hist);
  HM_KCHECK();
  if (tr) trace_end(F::kName, s, ev);
}

template <class F>
void launch_family(const hm_graph* g, const F& fam, const hm_graph::Space* sp, uint64_t total,
                   int order, unsigned long long* hist, cudaStream_t s, int chunk = 0,
                   uint64_t begin = 0, uint64_t end = ~0ull, bool traced = true, int sub = 0) {
  if (end > total) end = total;
  if (begin >= end) return;
  if (g->block)
    launch_family_t<F, true>(g, fam, sp, begin, end, chunk, order, hist, s, traced, sub);
  else
    launch_family_t<F, false>(g, fam, sp, begin, end, chunk, order, hist, s, traced, sub);
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

std::vector<std::pair<hm_graph::Space*, char>> census_spaces(hm_graph* g, int order) {
  if (order == 3) {
    if (g->bits2) return {{&g->W, 'W'}, {&g->Wb, 'w'}};
    return {{&g->W, 'W'}};
  }
  if (g->bits2)
    return {{&g->S, 'S'}, {&g->P, 'P'}, {&g->TX, 'X'}, {&g->Sb, 's'}, {&g->Pb, 'p'}, {&g->TXb, 'x'}};
  if (g->sig && !g->block)
    return {{&g->S, 'S'}, {&g->P, 'P'}, {&g->TX, 'X'}, {&g->C4, 'c'}, {&g->TXO, 'o'}};
  return {{&g->S, 'S'}, {&g->P, 'P'}, {&g->TX, 'X'}, {&g->C4, 'c'}};
}

// The graphlet census replaces S and P: with pair bitmaps, when its word
// operations (a word operation taken as a tenth of one candidate's
// evaluation) cost less than the cheaper variant of each; without, when S and
// P hold more than 5e8 candidates (its pair and 4-cycle passes cost about the
// degrees squared, far less on such graphs). HM_GRAPHLETS=0 / 1 forces it off
// / on; HM_DENSE_FAMILIES, which forces the S and P variants, keeps it off
// unless HM_GRAPHLETS=1.
bool prefer_graphlets(const hm_graph* g) {
  const char* env = std::getenv("HM_GRAPHLETS");
  if (env && env[0] == '0') return false;
  if (env && env[0] == '1') return true;
  if (std::getenv("HM_DENSE_FAMILIES")) return false;
  // without pair bitmaps (hash probes): when the S and P enumeration is large
  if (!g->bits2) return (double)g->S.total + (double)g->P.total > 5e8;
  const double bw = g->bwords;
  const double s_cost = std::min((double)g->S.total, (double)g->Sb.total * (2 + bw * 0.5) * 0.35);
  const double p_cost = std::min((double)g->P.total, (double)g->Pb.total * (2 + bw) * 0.35);
  return graphlet_cost(g) * 0.1 < s_cost + p_cost;
}

void choose_variants(hm_graph* g, int order) {
  if (order == 4) g->useGL = prefer_graphlets(g);
  if (!g->bits2) return;
  if (order == 3) {
    g->useWb = prefer_bits(g, g->Wb, g->W.total, 0.5);
  } else {
    g->useSb = prefer_bits(g, g->Sb, g->S.total, 0.5);
    g->usePb = prefer_bits(g, g->Pb, g->P.total, 1.0);
    // a bit-sliced TX item scans one 4-word group
    g->useTXb = g->bwords >= 4 && prefer_bits(g, g->TXb, g->TX.total, 4.0 / g->bwords);
  }
}

void schedule_census(hm_graph* g, int order, cudaStream_t s);

void prepare_census(hm_graph* g, int order, cudaStream_t s) {
  if (order == 4)
    HM_CHECK(g->max_d2 < (1 << 21), HM_EUNSUPPORTED,
             "a node has 2^21 or more pair neighbours; order-4 star space overflows");
  ensure_spaces(g, census_spaces(g, order), s);
  if (!g->tuned[order]) choose_variants(g, order);
  schedule_census(g, order, s);
}

namespace {

// One family of the census over the range [b, e) of the chosen variant's index
// space (bits: the bit-sliced space, else the per-candidate one).
// Bit-sliced TX over the items [b, e) of its space (whole 3-hyperedges:
// item index = 3-hyperedge x groups + group), one warp per 3-hyperedge.
template <bool kExact, bool kBatched>
void launch_txw_t(const hm_graph* g, int64_t t0, int64_t t1, unsigned long long* hist,
                  cudaStream_t s, bool traced, bool sub) {
  const ClassTables& T = class_tables(4);
  const uint8_t* lut = device_lut(4);
  const int64_t warps_per_block = CENSUS_THREADS / 32;
  int64_t blocks = (t1 - t0 + warps_per_block - 1) / warps_per_block;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (kBatched) {  // every block below 2^31 candidates (its uint32 bins)
    const int64_t floor_blocks = (int64_t)(((uint64_t)(t1 - t0) * g->bwords * 32) >> 31) + 1;
    if (blocks < floor_blocks) blocks = floor_blocks;
  }
  if (blocks < 1) blocks = 1;
  cudaEvent_t ev = nullptr;
  const bool tr = traced && trace_on("census_TXb");
  if (tr) trace_begin(s, &ev);
  k_census_txw<kExact, kBatched><<<(unsigned)blocks, CENSUS_THREADS, 0, s>>>(
      g->view(), t0, t1, lut, (int)T.lut.size(), T.ncls, num_graphs(g), sub ? 1 : 0, hist);
  HM_KCHECK();
  if (tr) trace_end("census_TXb", s, ev);
}

void launch_txw(const hm_graph* g, uint64_t b, uint64_t e, unsigned long long* hist,
                cudaStream_t s, bool traced, bool sub) {
  const uint64_t groups = (uint64_t)(g->bwords / 4);
  if (groups == 0) return;
  if (e > g->TXb.total) e = g->TXb.total;
  const int64_t t0 = (int64_t)(b / groups), t1 = (int64_t)((e + groups - 1) / groups);
  if (t0 >= t1) return;
  if (g->tri3) {
    if (g->block) launch_txw_t<true, true>(g, t0, t1, hist, s, traced, sub);
    else launch_txw_t<true, false>(g, t0, t1, hist, s, traced, sub);
  } else {
    if (g->block) launch_txw_t<false, true>(g, t0, t1, hist, s, traced, sub);
    else launch_txw_t<false, false>(g, t0, t1, hist, s, traced, sub);
  }
}

// sub: the set's pair pattern is subtracted too (graphlet census, TX only).
// TX of a whole graph with node signatures: k_census_txs.
void launch_txs(const hm_graph* g, unsigned long long* hist, cudaStream_t s, bool traced,
                bool sub) {
  if (g->counts[3] == 0) return;
  const ClassTables& T = class_tables(4);
  const uint8_t* lut = device_lut(4);
  // 3-hyperedges with short lists go four to a warp, the rest a warp each,
  // in one persistent grid (every SM's resident blocks) that reads the list
  // lengths on the device
  const int64_t m3 = g->counts[3];
  HM_CHECK(m3 < (1ll << 29), HM_EUNSUPPORTED, "2^29 or more 3-hyperedges on the sparse TX path");
  HM_CHECK(g->TXO.ready && g->out_deg, HM_EINVAL, "out-lists not built");
  // the member-pair set: a power of two >= 2 x (3 m3) slots, so it never fills
  uint64_t tcap = 16;
  while (tcap < (uint64_t)(6 * m3)) tcap <<= 1;
  // the quad Bloom filter: a power of two >= 32 bits per 4-hyperedge (8 per 3-subset)
  uint32_t nbits = 1024;
  while ((uint64_t)nbits < 32ull * (uint64_t)g->counts[4] && nbits < (1u << 31)) nbits <<= 1;
  const uint64_t nrec = g->TXO.total;  // wedge records, one per pair of an out-list
  size_t at = 0;
  auto take = [&](size_t bytes) {
    const size_t o = at;
    at += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t o_lists = take((size_t)2 * m3 * 4), o_counts = take(16), o_share = take((size_t)m3),
               o_tab = take((size_t)tcap * 8), o_val = take((size_t)tcap * 4),
               o_bloom = take((size_t)nbits / 8), o_runs = take(((size_t)m3 + 1) * 8),
               o_cur = take((size_t)m3 * 4), o_rec = take((size_t)std::max<uint64_t>(1, nrec) * 8),
               o_grp = take((size_t)std::max<uint64_t>(1, nrec) * 8);
  DBuf<unsigned char> buf(at, s);
  int32_t* small = reinterpret_cast<int32_t*>(buf.p + o_lists);
  int32_t* large = small + m3;
  unsigned int* counts = reinterpret_cast<unsigned int*>(buf.p + o_counts);
  uint8_t* share = buf.p + o_share;
  unsigned long long* tab = reinterpret_cast<unsigned long long*>(buf.p + o_tab);
  int32_t* tval = reinterpret_cast<int32_t*>(buf.p + o_val);
  uint32_t* bloom = reinterpret_cast<uint32_t*>(buf.p + o_bloom);
  // t's records are [rs[t], re[t]) = [rs[t], rs[t + 1]) of grp
  int64_t* rs = reinterpret_cast<int64_t*>(buf.p + o_runs);
  int64_t* re = rs + 1;
  unsigned int* cur = reinterpret_cast<unsigned int*>(buf.p + o_cur);
  uint64_t* rec = reinterpret_cast<uint64_t*>(buf.p + o_rec);
  uint64_t* grp = reinterpret_cast<uint64_t*>(buf.p + o_grp);
  // two trace spans: the preparation (member-pair set, quad filter, wedge
  // records grouped by 3-hyperedge, the split) and the TX kernel itself
  cudaEvent_t ev = nullptr;
  const bool trp = traced && trace_on("census_TX_prep");
  if (trp) trace_begin(s, &ev);
  HM_CUDA(cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned int), s));
  HM_CUDA(cudaMemsetAsync(tab, 0xFF, (size_t)tcap * 8, s));
  HM_CUDA(cudaMemsetAsync(bloom, 0, (size_t)nbits / 8, s));
  HM_CUDA(cudaMemsetAsync(rs, 0, ((size_t)m3 + 1) * 8, s));
  HM_CUDA(cudaMemsetAsync(cur, 0, (size_t)m3 * 4, s));
  k_tp_insert<<<grid1d(m3), 256, 0, s>>>(g->view(), tab, tval, tcap - 1);
  HM_KCHECK();
  if (g->counts[4]) {
    k_tq_bloom<<<grid1d(g->counts[4]), 256, 0, s>>>(g->view(), bloom, nbits);
    HM_KCHECK();
  }
  if (nrec) {
    // records grouped by 3-hyperedge: counts, offsets, placement
    const uint64_t want = ((uint64_t)g->n + 255) / 256;
    k_txs_wedges<<<(unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, 152 * 8)), 256, 0, s>>>(
        g->view(), g->out_deg, g->out_adj, g->TXO.ws, tab, tval, tcap - 1, rec);
    HM_KCHECK();
    k_txs_rec_count<<<grid1d((int64_t)nrec), 256, 0, s>>>(
        rec, nrec, reinterpret_cast<unsigned long long*>(rs));
    HM_KCHECK();
    ScanJob sj{reinterpret_cast<uint64_t*>(rs), m3, nullptr};
    scan_batch_inplace(&sj, 1, s);
    k_txs_rec_place<<<grid1d((int64_t)nrec), 256, 0, s>>>(rec, nrec, rs, cur, grp);
    HM_KCHECK();
  }
  k_txs_split<<<grid1d(m3), 256, 0, s>>>(g->view(), tab, tcap - 1, bloom, nbits, g->out_deg, rs,
                                         re, share, small, large, counts);
  HM_KCHECK();
  if (trp) trace_end("census_TX_prep", s, ev);
  const bool tr = traced && trace_on("census_TX");
  if (tr) trace_begin(s, &ev);
  int sms = 0, per = 0;
  resident_blocks((const void*)k_census_txs, sms, per);
  const int64_t want = (m3 + CENSUS_THREADS / 8 - 1) / (CENSUS_THREADS / 8);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * per));
  k_census_txs<<<blocks, CENSUS_THREADS, 0, s>>>(g->view(), large, small, counts, share,
                                                 g->out_deg, g->out_adj, grp, rs, re, lut,
                                                 (int)T.lut.size(), T.ncls, sub ? 1 : 0, hist);
  HM_KCHECK();
  if (tr) trace_end("census_TX", s, ev);
}

void launch_one(const hm_graph* g, char fam, bool bits, int chunk, int order,
                unsigned long long* hist, cudaStream_t s, uint64_t b = 0, uint64_t e = ~0ull,
                bool traced = true, bool sub = false) {
  switch (fam) {
    case 'W':
      if (bits && g->tri3)
        launch_bits(g, BitsWT<true>{}, g->Wb, order, hist, s, b, e, traced);
      else if (bits)
        launch_bits(g, BitsWT<false>{}, g->Wb, order, hist, s, b, e, traced);
      else
        launch_family(g, FamW{}, &g->W, g->W.total, order, hist, s, chunk, b, e, traced);
      break;
    case 'S':
      if (bits && g->tri3)
        launch_bits(g, BitsST<true>{}, g->Sb, order, hist, s, b, e, traced);
      else if (bits)
        launch_bits(g, BitsST<false>{}, g->Sb, order, hist, s, b, e, traced);
      else
        launch_family(g, FamS{}, &g->S, g->S.total, order, hist, s, chunk, b, e, traced);
      break;
    case 'P':
      if (bits && g->tri3)
        launch_bits(g, BitsPT<true>{}, g->Pb, order, hist, s, b, e, traced);
      else if (bits)
        launch_bits(g, BitsPT<false>{}, g->Pb, order, hist, s, b, e, traced);
      else
        launch_family(g, FamP{}, &g->P, g->P.total, order, hist, s, chunk, b, e, traced);
      break;
    default:
      if (bits) {
        launch_txw(g, b, e, hist, s, traced, sub);
      } else if (g->sig && !g->block && b == 0 && e == ~0ull && !std::getenv("HM_TX_PER_CANDIDATE")) {
        launch_txs(g, hist, s, traced, sub);
      } else {
        launch_family(g, FamTX{}, &g->TX, g->TX.total, order, hist, s, chunk, b, e, traced,
                      sub ? 1 : 0);
      }
      break;
  }
}

}  // namespace

// HM_CENSUS_CHUNK=c forces c candidates per lane on every per-candidate family
void launch_census(const hm_graph* g, int order, unsigned long long* hist, cudaStream_t s) {
  const char* env = std::getenv("HM_CENSUS_CHUNK");
  const int forced = env ? std::atoi(env) : 0;
  auto pick = [&](int c) { return forced > 0 ? forced : c; };
  if (order == 3) {
    launch_family(g, FamT3{}, nullptr, (uint64_t)g->counts[3], 3, hist, s, pick(0));
    launch_one(g, 'W', g->useWb, pick(g->chunkW), 3, hist, s);
  } else {
    // with the graphlet census, Q and TX subtract their sets from the class of
    // their pair pattern, and the graphlet launches replace S and P
    const bool gl = g->useGL;
    if (gl) {
      // four independent launches, each too small to fill the GPU, run side
      // by side: Q, TX, the graphlet pair sums, the graphlet node-pair sums;
      // then the finisher
      GraphletScratch G;
      graphlet_prepare(g, G, s);
      Fork f(s);
      launch_family(g, FamQ{}, nullptr, (uint64_t)g->counts[4], 4, hist, s, pick(0), 0, ~0ull,
                    true, 1);
      launch_one(g, 'X', g->useTXb, pick(g->chunkTX), 4, hist, f[0], 0, ~0ull, true, true);
      graphlet_edges(g, G, f[1]);
      graphlet_pairs(g, G, f[2]);
      f.join();
      graphlet_finish(g, G, hist, s);
    } else {
      launch_family(g, FamQ{}, nullptr, (uint64_t)g->counts[4], 4, hist, s, pick(0));
      launch_one(g, 'X', g->useTXb, pick(g->chunkTX), 4, hist, s);
      launch_one(g, 'S', g->useSb, pick(g->chunkS), 4, hist, s);
      launch_one(g, 'P', g->usePb, pick(g->chunkP), 4, hist, s);
    }
  }
}

// ------------------------------------------------------------------ generation check
namespace {

// Every connected set a per-candidate family accepts, as its sorted nodes
// packed into one key (bits per node, most significant first); count holds
// the number of sets, keys the first cap of them.
template <class F>
__global__ void k_emit_keys(const DevGraph g, const F fam, const uint64_t* __restrict__ ws,
                            int64_t A, uint64_t total, const uint8_t* __restrict__ lut, int k,
                            int bits, unsigned long long* __restrict__ count,
                            uint64_t* __restrict__ keys, uint64_t cap) {
  for (uint64_t gi = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; gi < total;
       gi += (uint64_t)gridDim.x * blockDim.x) {
    typename F::State st;
    uint32_t mask = 0;
    int32_t nd[4];
    bool ok;
    if (F::kDirect) {
      ok = fam.item(g, (int64_t)gi, st, mask, nd);
    } else {
      const int64_t a = anchor_of(ws, A, gi);
      fam.begin(g, a, gi - ws[a], st);
      ok = fam.item(g, a, st, mask, nd);
    }
    if (!ok || lut[mask] == 0xFF) continue;
    for (int i = 1; i < k; ++i) {  // insertion sort of the k nodes
      const int32_t x = nd[i];
      int j = i - 1;
      while (j >= 0 && nd[j] > x) {
        nd[j + 1] = nd[j];
        --j;
      }
      nd[j + 1] = x;
    }
    uint64_t key = 0;
    for (int i = 0; i < k; ++i) key = (key << bits) | (uint64_t)(uint32_t)nd[i];
    const unsigned long long at = atomicAdd(count, 1ull);
    if (at < cap) keys[at] = key;
  }
}

__global__ void k_count_dups(const uint64_t* __restrict__ keys, uint64_t n,
                             unsigned long long* __restrict__ dups) {
  unsigned long long mine = 0;
  for (uint64_t i = 1 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    mine += keys[i] == keys[i - 1] ? 1ull : 0ull;
  if (mine) atomicAdd(dups, mine);
}

template <class F>
void emit_keys(const hm_graph* g, const F& fam, const hm_graph::Space* sp, uint64_t total,
               int order, unsigned long long* count, uint64_t* keys, uint64_t cap,
               cudaStream_t s) {
  if (total == 0) return;
  const uint64_t blocks = std::min<uint64_t>((total + 255) / 256, 152 * 16);
  k_emit_keys<F><<<(unsigned)blocks, 256, 0, s>>>(g->view(), fam, sp ? sp->ws : nullptr,
                                                  sp ? sp->anchors : 0, total, device_lut(order),
                                                  order, g->bits, count, keys, cap);
  HM_KCHECK();
}

void emit_all(hm_graph* g, int order, unsigned long long* count, uint64_t* keys, uint64_t cap,
              cudaStream_t s) {
  if (order == 3) {
    emit_keys(g, FamT3{}, nullptr, (uint64_t)g->counts[3], 3, count, keys, cap, s);
    emit_keys(g, FamW{}, &g->W, g->W.total, 3, count, keys, cap, s);
  } else {
    emit_keys(g, FamQ{}, nullptr, (uint64_t)g->counts[4], 4, count, keys, cap, s);
    emit_keys(g, FamTX{}, &g->TX, g->TX.total, 4, count, keys, cap, s);
    emit_keys(g, FamS{}, &g->S, g->S.total, 4, count, keys, cap, s);
    emit_keys(g, FamP{}, &g->P, g->P.total, 4, count, keys, cap, s);
  }
}

}  // namespace

// The per-candidate families' canonical generation checked directly: every
// accepted connected set emitted as a key, the keys radix-sorted, repeats
// counted. out = {sets, repeated keys}.
void debug_canonical(hm_graph* g, int order, uint64_t* out, cudaStream_t s) {
  HM_CHECK(order * g->bits <= 64, HM_EUNSUPPORTED, "node ids too wide for one 64-bit key");
  HM_CHECK(g->block == 0, HM_EUNSUPPORTED, "not available for a union of graphs");
  ensure_spaces(g, order == 3 ? std::vector<std::pair<hm_graph::Space*, char>>{{&g->W, 'W'}}
                              : std::vector<std::pair<hm_graph::Space*, char>>{
                                    {&g->S, 'S'}, {&g->P, 'P'}, {&g->TX, 'X'}},
                s);
  DBuf<unsigned long long> cnt(2, s);
  HM_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(unsigned long long), s));
  emit_all(g, order, cnt.p, nullptr, 0, s);  // count only
  unsigned long long n = 0;
  HM_CUDA(cudaMemcpyAsync(&n, cnt.p, sizeof n, cudaMemcpyDeviceToHost, s));
  HM_CUDA(cudaStreamSynchronize(s));
  DBuf<uint64_t> keys(n ? n : 1, s);
  HM_CUDA(cudaMemsetAsync(cnt.p, 0, 2 * sizeof(unsigned long long), s));
  emit_all(g, order, cnt.p, keys.p, n, s);
  if (n > 1) {
    radix_sort_u64(keys.p, nullptr, (int64_t)n, order * g->bits, s);
    k_count_dups<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(
        keys.p, n, cnt.p + 1);
    HM_KCHECK();
  }
  unsigned long long h[2] = {0, 0};
  HM_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof h, cudaMemcpyDeviceToHost, s));
  unsigned timeouts = 0;
  wait_timeouts_async(&timeouts, s);
  HM_CUDA(cudaStreamSynchronize(s));
  wait_timeouts_check(timeouts, s);
  out[0] = h[0];
  out[1] = h[1];
}

// Alg. 1 on the projection graph p, with fill-in against the hypergraph h:
// the connected k-sets of p (wedges and triangles for k = 3; stars, paths and
// 4-cycles for k = 4), each counted by the class of the sub-hypergraph of h it
// induces when that is connected. Returns the candidates generated.
uint64_t launch_baseline(hm_graph* p, const hm_graph* h, int order, unsigned long long* hist,
                         cudaStream_t s) {
  if (order == 3) {
    ensure_spaces(p, {{&p->W, 'W'}}, s);
    launch_family(p, base::BaseW{h->view()}, &p->W, p->W.total, 3, hist, s);
    return p->W.total;
  }
  ensure_spaces(p, {{&p->S, 'S'}, {&p->P, 'P'}}, s);
  launch_family(p, base::BaseS{h->view()}, &p->S, p->S.total, 4, hist, s);
  launch_family(p, base::BaseP{h->view()}, &p->P, p->P.total, 4, hist, s);
  return p->S.total + p->P.total;
}

// ------------------------------------------------------------------ autotuner
// Schedules of the census: for each family with alternatives, the variant
// (bit-sliced or per-candidate, where bitmaps exist) and the candidates per
// lane (8, 16 or 32) of the per-candidate kernel, picked by timing the
// alternatives on the same node sets: 8 evenly spaced slices of the family's
// anchors, together sized for ~1e7 per-candidate candidates (all anchors
// when the family is smaller than 2e7). The cost rule's choice is timed
// first and kept unless another is 5 % faster; when it is the bit-sliced
// variant, the per-candidate kernel is tried with 32 candidates per lane only. Choices are cached by graph shape
// (order, nodes, block, row words, exact rows, and the binary orders of
// magnitude of |E_2|, |E_3|, |E_4| and of each family's size), so graphs of
// one shape are tuned once. HM_AUTOTUNE=0 keeps the cost rule.
namespace {

struct FamChoice {
  bool bits = false;
  int chunk = 0;
};
struct TuneEntry {
  FamChoice f[4];  // W, S, P, TX
};
std::mutex g_tune_mu;
std::map<std::string, TuneEntry> g_tune_cache;

int ilog2(uint64_t x) { return x ? 63 - __builtin_clzll(x) : -1; }

std::string shape_key(const hm_graph* g, int order) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "o%d n%d b%d bw%d t%d m%d,%d,%d s%d,%d,%d,%d", order, g->n,
                g->block, g->bwords, g->tri3 ? 1 : 0, ilog2((uint64_t)g->counts[2]),
                g->kmax >= 3 ? ilog2((uint64_t)g->counts[3]) : -1,
                g->kmax >= 4 ? ilog2((uint64_t)g->counts[4]) : -1, ilog2(g->W.total),
                ilog2(g->S.total), ilog2(g->P.total), ilog2(g->TX.total));
  return buf;
}

// off with HM_AUTOTUNE=0, and while a variant or chunk is forced
bool autotune_on() {
  const char* env = std::getenv("HM_AUTOTUNE");
  if (env && env[0] == '0') return false;
  return !std::getenv("HM_DENSE_FAMILIES") && !std::getenv("HM_CENSUS_CHUNK");
}

__global__ void k_gather_u64(const uint64_t* const* __restrict__ src,
                             const int64_t* __restrict__ idx, int n, uint64_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = src[i][idx[i]];
}

// Anchor slices [lo, hi) of one family and their index ranges in the
// per-candidate space (pc) and the bit-sliced space (bt).
struct Slices {
  int k = 0;
  int64_t lo[8] = {}, hi[8] = {};
  uint64_t pc_b[8] = {}, pc_e[8] = {}, bt_b[8] = {}, bt_e[8] = {};
};

void plan_slices(const hm_graph::Space& pc, Slices& sl) {
  const int64_t A = pc.anchors;
  sl.k = 0;
  if (A <= 0 || pc.total == 0) return;
  double f = 1e7 / (double)pc.total;
  if (f < 1.0 / 1024) f = 1.0 / 1024;
  if (f >= 0.5) {
    sl.k = 1;
    sl.lo[0] = 0;
    sl.hi[0] = A;
    return;
  }
  sl.k = 8;
  int64_t w = (int64_t)((double)A * f / 8);
  if (w < 1) w = 1;
  if (w > A) w = A;
  for (int i = 0; i < 8; ++i) {
    int64_t lo = (int64_t)((2 * i + 1) * (double)A / 16) - w / 2;
    if (lo < 0) lo = 0;
    if (lo + w > A) lo = A - w;
    sl.lo[i] = lo;
    sl.hi[i] = lo + w;
  }
}

struct Tuned {
  char id;
  hm_graph::Space* pc;
  hm_graph::Space* bt;
  Slices sl;
};

void tune_census(hm_graph* g, int order, cudaStream_t s) {
  const ClassTables& T = class_tables(order);
  DBuf<unsigned long long> scratch((size_t)T.ncls * num_graphs(g), s);
  std::vector<Tuned> fams;
  if (order == 3) {
    fams.push_back({'W', &g->W, g->bits2 ? &g->Wb : nullptr, {}});
  } else {
    if (!g->useGL) {  // the graphlet census replaces S and P
      fams.push_back({'S', &g->S, g->bits2 ? &g->Sb : nullptr, {}});
      fams.push_back({'P', &g->P, g->bits2 ? &g->Pb : nullptr, {}});
    }
    // with node signatures TX runs k_census_txs, which has no schedule
    if (!(g->sig && !g->block && !std::getenv("HM_TX_PER_CANDIDATE")))
      fams.push_back({'X', &g->TX, g->bits2 ? &g->TXb : nullptr, {}});
  }
  // slice boundaries in both spaces (bt = pc where there is no bit-sliced
  // variant), read back in one copy
  std::vector<const uint64_t*> src;
  std::vector<int64_t> idx;
  for (auto& F : fams) {
    plan_slices(*F.pc, F.sl);
    const uint64_t* bws = (F.bt && F.bt->ready && F.bt->ws) ? F.bt->ws : F.pc->ws;
    for (int i = 0; i < F.sl.k; ++i) {
      src.push_back(F.pc->ws);
      idx.push_back(F.sl.lo[i]);
      src.push_back(F.pc->ws);
      idx.push_back(F.sl.hi[i]);
      src.push_back(bws);
      idx.push_back(F.sl.lo[i]);
      src.push_back(bws);
      idx.push_back(F.sl.hi[i]);
    }
  }
  if (!idx.empty()) {
    const int nq = (int)idx.size();
    DBuf<const uint64_t*> dsrc(nq, s);
    DBuf<int64_t> didx(nq, s);
    DBuf<uint64_t> dout(nq, s);
    HM_CUDA(cudaMemcpyAsync(dsrc.p, src.data(), nq * sizeof(void*), cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyAsync(didx.p, idx.data(), nq * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_gather_u64<<<(nq + 127) / 128, 128, 0, s>>>(dsrc.p, didx.p, nq, dout.p);
    HM_KCHECK();
    std::vector<uint64_t> h(nq);
    HM_CUDA(cudaMemcpyAsync(h.data(), dout.p, nq * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    HM_CUDA(cudaStreamSynchronize(s));
    size_t q = 0;
    for (auto& F : fams)
      for (int i = 0; i < F.sl.k; ++i) {
        F.sl.pc_b[i] = h[q++];
        F.sl.pc_e[i] = h[q++];
        F.sl.bt_b[i] = h[q++];
        F.sl.bt_e[i] = h[q++];
      }
  }
  TuneEntry out;
  out.f[0] = {g->useWb, g->chunkW};
  out.f[1] = {g->useSb, g->chunkS};
  out.f[2] = {g->usePb, g->chunkP};
  out.f[3] = {g->useTXb, g->chunkTX};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HM_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    HM_CHECK(false, HM_ECUDA, "cudaEventCreate failed");
  }
  try {
    for (auto& F : fams) {
      if (F.sl.k == 0) continue;
      // the cost rule's choice first: another one must be 5 % faster to win
      std::vector<FamChoice> cands;
      const int slot0 = F.id == 'W' ? 0 : F.id == 'S' ? 1 : F.id == 'P' ? 2 : 3;
      const bool rule_bits = out.f[slot0].bits && F.bt && F.bt->ready && F.bt->total;
      cands.push_back({rule_bits, rule_bits ? 0 : 32});
      if (rule_bits) {
        cands.push_back({false, 32});
      } else {
        cands.push_back({false, 8});
        cands.push_back({false, 16});
        if (F.bt && F.bt->ready && F.bt->total) cands.push_back({true, 0});
      }
      auto run = [&](const FamChoice& c, bool warm) {
        for (int i = 0; i < F.sl.k; ++i) {
          const uint64_t b = c.bits ? F.sl.bt_b[i] : F.sl.pc_b[i];
          uint64_t e = c.bits ? F.sl.bt_e[i] : F.sl.pc_e[i];
          if (warm && e > b + 4096) e = b + 4096;  // a kernel's first launch loads it
          launch_one(g, F.id, c.bits, c.chunk, order, scratch.p, s, b, e, false);
          if (warm) break;
        }
      };
      float best = 0.f;
      FamChoice pick = cands[0];
      for (size_t ci = 0; ci < cands.size(); ++ci) {
        run(cands[ci], true);
        HM_CUDA(cudaEventRecord(e0, s));
        run(cands[ci], false);
        HM_CUDA(cudaEventRecord(e1, s));
        HM_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        HM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ci == 0 || ms < 0.95f * best) {
          best = ms;
          pick = cands[ci];
        }
      }
      const int slot = F.id == 'W' ? 0 : F.id == 'S' ? 1 : F.id == 'P' ? 2 : 3;
      out.f[slot] = pick;
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[shape_key(g, order)] = out;
  }
  g->useWb = out.f[0].bits;
  g->chunkW = out.f[0].chunk;
  g->useSb = out.f[1].bits;
  g->chunkS = out.f[1].chunk;
  g->usePb = out.f[2].bits;
  g->chunkP = out.f[2].chunk;
  g->useTXb = out.f[3].bits;
  g->chunkTX = out.f[3].chunk;
}

}  // namespace

// Schedules of one order: from the cache, else by tuning (one synchronisation
// and a few slices of each family), unless HM_AUTOTUNE=0 (the cost rule).
void schedule_census(hm_graph* g, int order, cudaStream_t s) {
  if (g->tuned[order] || !autotune_on()) return;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(shape_key(g, order));
    if (it != g_tune_cache.end()) {
      const TuneEntry& t = it->second;
      g->useWb = t.f[0].bits && g->bits2;
      g->chunkW = t.f[0].chunk;
      g->useSb = t.f[1].bits && g->bits2;
      g->chunkS = t.f[1].chunk;
      g->usePb = t.f[2].bits && g->bits2;
      g->chunkP = t.f[2].chunk;
      g->useTXb = t.f[3].bits && g->bits2;
      g->chunkTX = t.f[3].chunk;
      g->tuned[order] = true;
      return;
    }
  }
  tune_census(g, order, s);
  g->tuned[order] = true;
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
    for (int i = 0; i < 10; ++i) totals[i] = 0;
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
      totals[8] = g->TXb.total;
      totals[9] = g->useTXb ? 1 : 0;
    }
  });
}

extern "C" hm_status hm_debug_canonical_check(hm_graph* g, int order, uint64_t* h_out,
                                              void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g && h_out, HM_EINVAL, "NULL argument");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= g->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    hm::debug_canonical(g, order, h_out, (cudaStream_t)stream);
  });
}
