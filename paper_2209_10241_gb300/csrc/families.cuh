// Candidate families of the exact census and the per-sample enumeration of
// the sampling estimator: index-space decoding and the canonical-generation
// rules, shared by census.cu and sampler.cu. See census.cu for the rules.
#pragma once

#include "hm_internal.cuh"

namespace hm {
namespace fam {

constexpr int CENSUS_THREADS = 256;
constexpr int CHUNK = 32;  // consecutive items per lane

__host__ __device__ __forceinline__ uint64_t choose2(uint64_t x) { return x * (x - 1) / 2; }
__host__ __device__ __forceinline__ uint64_t choose3(uint64_t x) {
  return x < 3 ? 0 : x * (x - 1) / 2 * (x - 2) / 3;
}

// r = C(j,2) + i with 0 <= i < j
__device__ __forceinline__ void unrank2(uint64_t r, uint32_t& i, uint32_t& j) {
  // the estimate is corrected exactly below; single precision is close
  // enough for r < 2^22 and much cheaper than double on this part
  uint64_t jj = r < (1ull << 22) ? (uint64_t)((1.0f + sqrtf(1.0f + 8.0f * (float)r)) * 0.5f)
                                 : (uint64_t)((1.0 + sqrt(1.0 + 8.0 * (double)r)) * 0.5);
  if (jj < 1) jj = 1;
  while (choose2(jj) > r) --jj;
  while (choose2(jj + 1) <= r) ++jj;
  j = (uint32_t)jj;
  i = (uint32_t)(r - choose2(jj));
}

// r = C(l,3) + C(j,2) + i with 0 <= i < j < l
__device__ __forceinline__ void unrank3(uint64_t r, uint32_t& i, uint32_t& j, uint32_t& l) {
  uint64_t ll = r < (1ull << 20) ? (uint64_t)cbrtf(6.0f * (float)r) + 1
                                 : (uint64_t)cbrt(6.0 * (double)r) + 1;
  if (ll < 2) ll = 2;
  while (choose3(ll) > r) --ll;
  while (choose3(ll + 1) <= r) ++ll;
  l = (uint32_t)ll;
  unrank2(r - choose3(ll), i, j);
}

// sorted member tuple of a 3-hyperedge, comparable
struct Tri {
  uint64_t hi;
  uint32_t lo;
};
__device__ __forceinline__ Tri make_tri(int32_t a, int32_t b, int32_t c) {
  sort3(a, b, c);
  return Tri{((uint64_t)(uint32_t)a << 32) | (uint32_t)b, (uint32_t)c};
}
__device__ __forceinline__ bool tri_less(const Tri& x, const Tri& y) {
  return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo);
}
__device__ __forceinline__ bool tri_eq(const Tri& x, const Tri& y) {
  return x.hi == y.hi && x.lo == y.lo;
}

// ---------------------------------------------------------------- families
// Direct families: one candidate per anchor. With `map` set (sampling), the
// anchor is a sample and map[anchor] the sampled hyperedge.
struct FamT3 {
  static constexpr const char* kName = "census_T3";
  static constexpr bool kDirect = true;
  const int64_t* map = nullptr;
  struct State {};
  __device__ int32_t graph_node(const DevGraph& g, int64_t t) const {
    return g.e3[map ? map[t] : t].x;
  }
  __device__ void begin(const DevGraph&, int64_t, uint64_t, State&) const {}
  __device__ void next(State&) const {}
  __device__ bool item(const DevGraph& g, int64_t t, State&, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int4 e = g.e3[map ? map[t] : t];
    mask = (has_pair(g, e.x, e.y) ? 1u : 0u) | (has_pair(g, e.x, e.z) ? 2u : 0u) |
           (has_pair(g, e.y, e.z) ? 4u : 0u) | 8u;
    nd[0] = e.x;
    nd[1] = e.y;
    nd[2] = e.z;
    return true;
  }
};

struct FamQ {
  static constexpr const char* kName = "census_Q";
  static constexpr bool kDirect = true;
  const int64_t* map = nullptr;
  struct State {};
  __device__ int32_t graph_node(const DevGraph& g, int64_t q) const {
    return g.e4[map ? map[q] : q].x;
  }
  __device__ void begin(const DevGraph&, int64_t, uint64_t, State&) const {}
  __device__ void next(State&) const {}
  __device__ bool item(const DevGraph& g, int64_t q, State&, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int4 e = g.e4[map ? map[q] : q];
    const int32_t a = e.x, b = e.y, c = e.z, d = e.w;
    nd[0] = a;
    nd[1] = b;
    nd[2] = c;
    nd[3] = d;
    mask = (has_pair(g, a, b) ? 1u : 0u) | (has_pair(g, a, c) ? 2u : 0u) |
           (has_pair(g, a, d) ? 4u : 0u) | (has_pair(g, b, c) ? 8u : 0u) |
           (has_pair(g, b, d) ? 16u : 0u) | (has_pair(g, c, d) ? 32u : 0u) |
           (has_triple(g, a, b, c) ? 64u : 0u) | (has_triple(g, a, b, d) ? 128u : 0u) |
           (has_triple(g, a, c, d) ? 256u : 0u) | (has_triple(g, b, c, d) ? 512u : 0u) | 1024u;
    return true;
  }
};

struct FamW {
  static constexpr const char* kName = "census_W";
  static constexpr bool kDirect = false;
  __device__ int32_t graph_node(const DevGraph&, int64_t v) const { return (int32_t)v; }
  struct State {
    uint32_t i, j;
    int64_t o;
  };
  __device__ void begin(const DevGraph& g, int64_t v, uint64_t r, State& s) const {
    s.o = g.off2[v];
    unrank2(r, s.i, s.j);
  }
  __device__ void next(State& s) const {
    if (++s.i == s.j) {
      s.i = 0;
      ++s.j;
    }
  }
  __device__ bool item(const DevGraph& g, int64_t a, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int32_t v = (int32_t)a;
    const int32_t x = g.adj2[s.o + s.i], y = g.adj2[s.o + s.j];
    nd[0] = v;
    nd[1] = x;
    nd[2] = y;
    const bool xy = has_pair(g, x, y);
    if (xy && (x < v || y < v)) return false;  // a triangle is kept at its smallest node
    if (has_triple(g, v, x, y)) return false;  // counted with its 3-hyperedge
    mask = 3u | (xy ? 4u : 0u);                // positions v=0, x=1, y=2
    return true;
  }
};

struct FamS {
  static constexpr const char* kName = "census_S";
  static constexpr bool kDirect = false;
  __device__ int32_t graph_node(const DevGraph&, int64_t v) const { return (int32_t)v; }
  struct State {
    uint32_t i, j, l;
    int64_t o;
  };
  __device__ void begin(const DevGraph& g, int64_t v, uint64_t r, State& s) const {
    s.o = g.off2[v];
    unrank3(r, s.i, s.j, s.l);
  }
  __device__ void next(State& s) const {
    if (++s.i == s.j) {
      s.i = 0;
      if (++s.j == s.l) {
        s.j = 1;
        ++s.l;
      }
    }
  }
  __device__ bool item(const DevGraph& g, int64_t a, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int32_t v = (int32_t)a;
    const int32_t x = g.adj2[s.o + s.i], y = g.adj2[s.o + s.j], z = g.adj2[s.o + s.l];
    nd[0] = v;
    nd[1] = x;
    nd[2] = y;
    nd[3] = z;
    const bool xy = has_pair(g, x, y), xz = has_pair(g, x, z), yz = has_pair(g, y, z);
    // v has induced degree 3; it must be the smallest node of degree 3
    if ((xy && xz && x < v) || (xy && yz && y < v) || (xz && yz && z < v)) return false;
    if (has_triple(g, v, x, y) || has_triple(g, v, x, z) || has_triple(g, v, y, z) ||
        has_triple(g, x, y, z) || has_quad(g, v, x, y, z))
      return false;  // not a pairs-only set: counted by Q or TX
    mask = 7u | (xy ? 8u : 0u) | (xz ? 16u : 0u) | (yz ? 32u : 0u);  // v=0,x=1,y=2,z=3
    return true;
  }
};

struct FamP {
  static constexpr const char* kName = "census_P";
  static constexpr bool kDirect = false;
  __device__ int32_t graph_node(const DevGraph& g, int64_t p) const {
    return (int32_t)(g.e2[p] >> 32);
  }
  struct State {
    int32_t u, v;
    int64_t ou, ov;
    uint32_t pu, pv, dv1, i2, j2;
  };
  __device__ void begin(const DevGraph& g, int64_t p, uint64_t r, State& s) const {
    const uint64_t uv = g.e2[p];
    s.u = (int32_t)(uv >> 32);
    s.v = (int32_t)(uv & 0xFFFFFFFFull);
    s.ou = g.off2[s.u];
    s.ov = g.off2[s.v];
    s.dv1 = (uint32_t)(g.off2[s.v + 1] - s.ov - 1);
    const int2 pp = g.pairpos[p];
    s.pu = (uint32_t)pp.x;
    s.pv = (uint32_t)pp.y;
    s.i2 = (uint32_t)(r / s.dv1);
    s.j2 = (uint32_t)(r % s.dv1);
  }
  __device__ void next(State& s) const {
    if (++s.j2 == s.dv1) {
      s.j2 = 0;
      ++s.i2;
    }
  }
  __device__ bool item(const DevGraph& g, int64_t, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int32_t u = s.u, v = s.v;
    const int32_t x = g.adj2[s.ou + s.i2 + (s.i2 >= s.pu ? 1 : 0)];  // N2(u) \ {v}
    const int32_t y = g.adj2[s.ov + s.j2 + (s.j2 >= s.pv ? 1 : 0)];  // N2(v) \ {u}
    nd[0] = u;
    nd[1] = v;
    nd[2] = x;
    nd[3] = y;
    if (x == y) return false;
    if (has_pair(g, u, y) || has_pair(g, v, x)) return false;  // a degree-3 node: family S
    const bool xy = has_pair(g, x, y);
    if (xy) {  // 4-cycle: kept at its smallest pair
      const uint64_t kuv = pair_key(u, v);
      if (pair_key(u, x) < kuv || pair_key(v, y) < kuv || pair_key(x, y) < kuv) return false;
    }
    if (has_triple(g, u, v, x) || has_triple(g, u, v, y) || has_triple(g, u, x, y) ||
        has_triple(g, v, x, y) || has_quad(g, u, v, x, y))
      return false;
    mask = 1u | 2u | 16u | (xy ? 32u : 0u);  // u=0, v=1, x=2, y=3: pairs 01, 02, 13 (+23)
    return true;
  }
};

// kCensus: the anchor is a 3-hyperedge and a set is kept only at its smallest
// 3-hyperedge. Otherwise (sampling, Alg. 4) the anchor is a sample whose
// 3-hyperedge is map[anchor] and every set through it whose largest hyperedges
// have 3 members is kept.
template <bool kCensus>
struct FamTXT {
  static constexpr const char* kName = kCensus ? "census_TX" : "sample_TX";
  static constexpr bool kDirect = false;
  const int64_t* map = nullptr;
  __device__ int32_t graph_node(const DevGraph& g, int64_t a) const {
    return g.e3[kCensus ? a : map[a]].x;
  }
  // Per anchor: its members, their pair and triple degrees, its own pairs and
  // (graphs with signatures) the members' signatures, so that a candidate d
  // probes only what its signature bit allows.
  struct State {
    int32_t x[3];
    int32_t d2[3];
    uint64_t w[3];
    uint64_t r;
    int64_t t;
    uint64_t s2[3], s3[3], s4;
    bool ab, ac, bc;
  };
  __device__ void begin(const DevGraph& g, int64_t anchor, uint64_t r, State& s) const {
    const int64_t t = kCensus ? anchor : map[anchor];
    s.t = t;
    const int4 e = g.e3[t];
    s.x[0] = e.x;
    s.x[1] = e.y;
    s.x[2] = e.z;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int32_t n = s.x[j];
      s.d2[j] = (int32_t)(g.off2[n + 1] - g.off2[n]);
      s.w[j] = (uint64_t)s.d2[j] + (uint64_t)(g.off3[n + 1] - g.off3[n]);
    }
    s.r = r;
    s.ab = has_pair(g, e.x, e.y);
    s.ac = has_pair(g, e.x, e.z);
    s.bc = has_pair(g, e.y, e.z);
    s.s4 = ~0ull;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      s.s2[j] = g.sig ? g.sig[s.x[j]] : ~0ull;
      s.s3[j] = g.sig ? g.sig[(int64_t)g.n + s.x[j]] : ~0ull;
      if (g.sig) s.s4 &= g.sig[2 * (int64_t)g.n + s.x[j]];
    }
  }
  __device__ void next(State& s) const { ++s.r; }
  __device__ bool item(const DevGraph& g, int64_t, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int64_t t = s.t;
    uint64_t r = s.r;
    int which = 0;
    if (r >= s.w[0]) {
      r -= s.w[0];
      which = 1;
      if (r >= s.w[1]) {
        r -= s.w[1];
        which = 2;
      }
    }
    const int32_t a = s.x[0], b = s.x[1], c = s.x[2];
    const int32_t x = s.x[which];
    int32_t d;
    bool hpair;
    Tri htri{0, 0};
    if (r < (uint64_t)s.d2[which]) {
      d = g.adj2[g.off2[x] + r];
      if (d == a || d == b || d == c) return false;
      hpair = true;
    } else {
      const int32_t th = g.inc3[g.off3[x] + (int64_t)(r - s.d2[which])];
      if (th == t) return false;
      const int4 h = g.e3[th];
      const int32_t hm[3] = {h.x, h.y, h.z};
      int outside = 0;
      int32_t o = -1, inmin = 0x7FFFFFFF;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (hm[j] == a || hm[j] == b || hm[j] == c) {
          inmin = min(inmin, hm[j]);
        } else {
          ++outside;
          o = hm[j];
        }
      }
      if (outside != 1 || x != inmin) return false;
      d = o;
      hpair = false;
      htri = make_tri(h.x, h.y, h.z);
    }
    return evaluate(g, s, which, d, hpair, htri, mask, nd);
  }
  // The candidate {a, b, c, d} generated from member `which` by the pair
  // {x, d} (hpair) or the 3-hyperedge htri: the canonical rules and its mask.
  __device__ bool evaluate(const DevGraph& g, const State& s, int which, int32_t d, bool hpair,
                           Tri htri, uint32_t& mask, int32_t (&nd)[4]) const {
    const int32_t a = s.x[0], b = s.x[1], c = s.x[2];
    const int32_t x = s.x[which];
    // h must be the smallest hyperedge of the set containing d. A pair
    // hyperedge h = {x, d} is known to exist; other probes run only where
    // the members' signatures hold d's bit.
    const uint64_t db = sig_bit(d);
    const bool ad = (hpair && which == 0) || ((s.s2[0] & db) && has_pair(g, a, d));
    const bool bd = (hpair && which == 1) || ((s.s2[1] & db) && has_pair(g, b, d));
    const bool cd = (hpair && which == 2) || ((s.s2[2] & db) && has_pair(g, c, d));
    if (ad || bd || cd) {
      if (!hpair) return false;
      uint64_t mn = ~0ull;
      if (ad) mn = min(mn, pair_key(a, d));
      if (bd) mn = min(mn, pair_key(b, d));
      if (cd) mn = min(mn, pair_key(c, d));
      if (pair_key(x, d) != mn) return false;
    }
    const bool abd = (s.s3[0] & s.s3[1] & db) && has_triple(g, a, b, d);
    const bool acd = (s.s3[0] & s.s3[2] & db) && has_triple(g, a, c, d);
    const bool bcd = (s.s3[1] & s.s3[2] & db) && has_triple(g, b, c, d);
    const Tri e = make_tri(a, b, c);
    const Tri tabd = make_tri(a, b, d), tacd = make_tri(a, c, d), tbcd = make_tri(b, c, d);
    // census: e must be the smallest 3-hyperedge of the set
    if (kCensus &&
        ((abd && tri_less(tabd, e)) || (acd && tri_less(tacd, e)) || (bcd && tri_less(tbcd, e))))
      return false;
    if (!hpair) {
      Tri mn{~0ull, 0xFFFFFFFFu};
      if (abd && tri_less(tabd, mn)) mn = tabd;
      if (acd && tri_less(tacd, mn)) mn = tacd;
      if (bcd && tri_less(tbcd, mn)) mn = tbcd;
      if (!tri_eq(htri, mn)) return false;
    }
    if ((s.s4 & db) && has_quad(g, a, b, c, d)) return false;  // a 4-hyperedge (family Q)
    nd[0] = a;
    nd[1] = b;
    nd[2] = c;
    nd[3] = d;
    const bool ab = s.ab, ac = s.ac, bc = s.bc;
    mask = (ab ? 1u : 0u) | (ac ? 2u : 0u) | (ad ? 4u : 0u) | (bc ? 8u : 0u) |
           (bd ? 16u : 0u) | (cd ? 32u : 0u) | 64u | (abd ? 128u : 0u) | (acd ? 256u : 0u) |
           (bcd ? 512u : 0u);  // a=0, b=1, c=2, d=3
    return true;
  }
};
using FamTX = FamTXT<true>;

__device__ __forceinline__ int64_t anchor_of(const uint64_t* __restrict__ ws, int64_t A,
                                             uint64_t g0) {
  // last a with ws[a] <= g0 (ws non-decreasing, ws[0] = 0)
  int64_t lo = 0, hi = A;  // answer in [0, A)
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (ws[mid] <= g0)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- bit-sliced families
// On graphs small enough for dense bitmaps, the last node of W, S and P runs
// over 32 node ids per bitmap word: the fill-in bits of 32 candidates come
// from word-wide ANDs, the canonical rules become masks, and each candidate
// group is counted with one popc. A 3-/4-hyperedge can only lie in a
// candidate whose node pairs all co-occur in some 3-/4-hyperedge, so those
// bitmaps mark the few "risky" candidates that get exact hash probes; every
// other candidate is proven free of larger hyperedges.
__device__ __forceinline__ const uint32_t* brow(const uint32_t* bm, int32_t bw, int32_t v) {
  return bm + (size_t)v * bw;
}
// bit of node b in the row of node a (rows span a's block of ids)
__device__ __forceinline__ bool btest(const DevGraph& g, const uint32_t* bm, int32_t a, int32_t b) {
  const int32_t c = b - graph_base(g, a);
  return (__ldg(bm + (size_t)a * g.bwords + (c >> 5)) >> (c & 31)) & 1u;
}
// four consecutive words of a bitmap row (rows are padded to a multiple of
// four words, so w % 4 == 0 is 16-byte aligned)
__device__ __forceinline__ void ld4(const uint32_t* p, uint32_t (&o)[4]) {
  const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}

// bits of word w whose (local) id exceeds t
__device__ __forceinline__ uint32_t above(int32_t w, int32_t t) {
  const int32_t tw = t >> 5;
  if (w < tw) return 0u;
  if (w > tw) return ~0u;
  const int32_t b = t & 31;
  return b == 31 ? 0u : (~0u << (b + 1));
}

// k = 3, pairs-only triples: anchor v, item x in N2(v), y over ids > x in N2(v).
// kExact: the graph has exact 3-hyperedge rows (otherwise the co-occurrence
// filter and exact probes of the risky candidates).
template <bool kExact>
struct BitsWT {
  static constexpr const char* kName = "census_Wb";
  struct State {
    int64_t o;
    uint32_t i;
  };
  __device__ int32_t graph_node(const DevGraph&, int64_t v) const { return (int32_t)v; }
  __device__ void begin(const DevGraph& g, int64_t v, uint64_t r, State& s) const {
    s.o = g.off2[v];
    s.i = (uint32_t)r;
  }
  __device__ void next(State& s) const { ++s.i; }
  template <class Bin>
  __device__ void item(const DevGraph& g, int64_t a, State& s, const uint8_t* lut, Bin* bins) const {
    const int32_t v = (int32_t)a, bw = g.bwords, base = graph_base(g, v);
    const int32_t x = g.adj2[s.o + s.i], xl = x - base;
    const uint32_t *Bv = brow(g.bits2, bw, v), *Bx = brow(g.bits2, bw, x);
    const uint32_t *Tv = brow(g.bits3, bw, v), *Tx = brow(g.bits3, bw, x);
    const bool tvx = !kExact && btest(g, g.bits3, v, x);
    const bool tri_ok = x > v;  // a triangle is kept at its smallest node
    // exact rows: the 3-hyperedges {v, x, y} are known per word
    const uint32_t* Rvx = kExact ? g.tri3 + ((size_t)v * g.n + x) * bw : nullptr;
    unsigned long long nw = 0, nt = 0;
    for (int32_t w4 = (xl >> 5) & ~3; w4 < bw; w4 += 4) {
      uint32_t Y4[4], bx4[4], r4[4] = {0, 0, 0, 0}, tv4[4] = {0, 0, 0, 0}, tx4[4] = {0, 0, 0, 0};
      ld4(Bv + w4, Y4);
      if (!((Y4[0] & above(w4, xl)) | (Y4[1] & above(w4 + 1, xl)) | (Y4[2] & above(w4 + 2, xl)) |
            (Y4[3] & above(w4 + 3, xl))))
        continue;
      ld4(Bx + w4, bx4);
      if (kExact) ld4(Rvx + w4, r4);
      if (!kExact && tvx) {
        ld4(Tv + w4, tv4);
        ld4(Tx + w4, tx4);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int32_t w = w4 + k;
        const uint32_t Y = Y4[k] & above(w, xl) & ~r4[k];
        if (!Y) continue;
        const uint32_t bx = bx4[k];
        const uint32_t tri = tri_ok ? (Y & bx) : 0u, wed = Y & ~bx;
        const uint32_t risky = tv4[k] & tx4[k];
        nt += __popc(tri & ~risky);
        nw += __popc(wed & ~risky);
        uint32_t rb = (tri | wed) & risky;
        while (rb) {
          const int b = __ffs(rb) - 1;
          rb &= rb - 1;
          if (!has_triple(g, v, x, base + w * 32 + b)) {
            if ((tri >> b) & 1u)
              ++nt;
            else
              ++nw;
          }
        }
      }
    }
    if (nw) atomicAdd(&bins[lut[3]], (Bin)nw);  // v=0, x=1, y=2: pairs 01, 02
    if (nt) atomicAdd(&bins[lut[7]], (Bin)nt);  // + pair 12
  }
};

// k = 4, stars: anchor v, item x < y in N2(v), z over ids > y in N2(v)
template <bool kExact>
struct BitsST {
  static constexpr const char* kName = "census_Sb";
  struct State {
    uint32_t i, j;
    int64_t o;
  };
  __device__ int32_t graph_node(const DevGraph&, int64_t v) const { return (int32_t)v; }
  __device__ void begin(const DevGraph& g, int64_t v, uint64_t r, State& s) const {
    s.o = g.off2[v];
    unrank2(r, s.i, s.j);
  }
  __device__ void next(State& s) const {
    if (++s.i == s.j) {
      s.i = 0;
      ++s.j;
    }
  }
  template <class Bin>
  __device__ void item(const DevGraph& g, int64_t a, State& s, const uint8_t* lut, Bin* bins) const {
    const int32_t v = (int32_t)a, bw = g.bwords, base = graph_base(g, v);
    const int32_t x = g.adj2[s.o + s.i], y = g.adj2[s.o + s.j];
    const int32_t vl = v - base, yl = y - base;
    // exact rows (when present) decide every 3-hyperedge of the candidates;
    // otherwise the co-occurrence bitmaps filter and the risky bits are probed
    const uint32_t* R = g.tri3;
    constexpr bool exact = kExact;
    const bool tvx = !exact && btest(g, g.bits3, v, x), tvy = !exact && btest(g, g.bits3, v, y),
               txy = !exact && btest(g, g.bits3, x, y);
    if (exact) {
      if (btest(g, R + (size_t)v * g.n * bw, x, y)) return;  // {v, x, y}
    } else if (tvx && tvy && txy && has_triple(g, v, x, y)) {
      return;
    }
    const uint32_t* Rvx = exact ? R + ((size_t)v * g.n + x) * bw : nullptr;
    const uint32_t* Rvy = exact ? R + ((size_t)v * g.n + y) * bw : nullptr;
    const uint32_t* Rxy = exact ? R + ((size_t)x * g.n + y) * bw : nullptr;
    const bool qd = btest(g, g.bits4, v, x) && btest(g, g.bits4, v, y) &&
                    btest(g, g.bits4, x, y);
    const bool xy = btest(g, g.bits2, x, y);
    // a node of degree 3 smaller than v rejects the set
    const bool rx = xy && x < v, ry = xy && y < v;
    const uint32_t *Bv = brow(g.bits2, bw, v), *Bx = brow(g.bits2, bw, x), *By = brow(g.bits2, bw, y);
    const uint32_t *Tv = brow(g.bits3, bw, v), *Tx = brow(g.bits3, bw, x), *Ty = brow(g.bits3, bw, y);
    const uint32_t *Qv = brow(g.bits4, bw, v), *Qx = brow(g.bits4, bw, x), *Qy = brow(g.bits4, bw, y);
    unsigned long long c[4] = {0, 0, 0, 0};  // (xz, yz) = 00, 10, 01, 11
    for (int32_t w4 = (yl >> 5) & ~3; w4 < bw; w4 += 4) {
      uint32_t Z4[4];
      ld4(Bv + w4, Z4);
#pragma unroll
      for (int k = 0; k < 4; ++k) Z4[k] &= above(w4 + k, yl);
      if (!(Z4[0] | Z4[1] | Z4[2] | Z4[3])) continue;
      if (exact) {
        uint32_t a4[4], b4[4], c4[4];
        ld4(Rvx + w4, a4);
        ld4(Rvy + w4, b4);
        ld4(Rxy + w4, c4);
#pragma unroll
        for (int k = 0; k < 4; ++k) Z4[k] &= ~(a4[k] | b4[k] | c4[k]);
      }
      uint32_t bx4[4], by4[4];
      ld4(Bx + w4, bx4);
      ld4(By + w4, by4);
      uint32_t rk4[4] = {0, 0, 0, 0};
      if (!exact && (tvx || tvy || txy)) {
        uint32_t tv4[4], tx4[4], ty4[4];
        ld4(Tv + w4, tv4);
        ld4(Tx + w4, tx4);
        ld4(Ty + w4, ty4);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          rk4[k] = (tvx ? tv4[k] & tx4[k] : 0u) | (tvy ? tv4[k] & ty4[k] : 0u) |
                   (txy ? tx4[k] & ty4[k] : 0u);
      }
      if (qd) {
        uint32_t qv4[4], qx4[4], qy4[4];
        ld4(Qv + w4, qv4);
        ld4(Qx + w4, qx4);
        ld4(Qy + w4, qy4);
#pragma unroll
        for (int k = 0; k < 4; ++k) rk4[k] |= qv4[k] & qx4[k] & qy4[k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int32_t w = w4 + k;
        const uint32_t Z = Z4[k];
        if (!Z) continue;
        const uint32_t bx = bx4[k], by = by4[k], risky = rk4[k];
        uint32_t grp[4];
        grp[0] = Z & ~bx & ~by;
        grp[1] = rx ? 0u : (Z & bx & ~by);
        grp[2] = ry ? 0u : (Z & ~bx & by);
        grp[3] = (rx || ry) ? 0u : (Z & bx & by & above(w, vl));
#pragma unroll
        for (int q = 0; q < 4; ++q) c[q] += __popc(grp[q] & ~risky);
        uint32_t rb = (grp[0] | grp[1] | grp[2] | grp[3]) & risky;
        while (rb) {
          const int b = __ffs(rb) - 1;
          rb &= rb - 1;
          const int32_t z = base + w * 32 + b;
          if ((!exact && (has_triple(g, v, x, z) || has_triple(g, v, y, z) ||
                          has_triple(g, x, y, z))) ||
              has_quad(g, v, x, y, z))
            continue;
          const uint32_t gi = ((bx >> b) & 1u) | (((by >> b) & 1u) << 1);
          c[0] += gi == 0u;
          c[1] += gi == 1u;
          c[2] += gi == 2u;
          c[3] += gi == 3u;
        }
      }
    }
    const uint32_t basem = 7u | (xy ? 8u : 0u);  // v=0, x=1, y=2, z=3
    if (c[0]) atomicAdd(&bins[lut[basem]], (Bin)c[0]);
    if (c[1]) atomicAdd(&bins[lut[basem | 16u]], (Bin)c[1]);
    if (c[2]) atomicAdd(&bins[lut[basem | 32u]], (Bin)c[2]);
    if (c[3]) atomicAdd(&bins[lut[basem | 48u]], (Bin)c[3]);
  }
};

// k = 4, paths and 4-cycles: anchor pair (u, v), u < v, item x in N2(u)\{v},
// y over N2(v) \ N2[u]
template <bool kExact>
struct BitsPT {
  static constexpr const char* kName = "census_Pb";
  struct State {
    int32_t u, v;
    int64_t ou;
    uint32_t pu, i;
  };
  __device__ int32_t graph_node(const DevGraph& g, int64_t p) const {
    return (int32_t)(g.e2[p] >> 32);
  }
  __device__ void begin(const DevGraph& g, int64_t p, uint64_t r, State& s) const {
    const uint64_t uv = g.e2[p];
    s.u = (int32_t)(uv >> 32);
    s.v = (int32_t)(uv & 0xFFFFFFFFull);
    s.ou = g.off2[s.u];
    s.pu = (uint32_t)g.pairpos[p].x;
    s.i = (uint32_t)r;
  }
  __device__ void next(State& s) const { ++s.i; }
  template <class Bin>
  __device__ void item(const DevGraph& g, int64_t, State& s, const uint8_t* lut, Bin* bins) const {
    const int32_t u = s.u, v = s.v, bw = g.bwords, base = graph_base(g, u);
    const int32_t x = g.adj2[s.ou + s.i + (s.i >= s.pu ? 1 : 0)];
    if (btest(g, g.bits2, v, x)) return;  // v would have degree 3: family S
    const uint32_t* R = g.tri3;
    constexpr bool exact = kExact;
    const bool tuv = !exact && btest(g, g.bits3, u, v), tux = !exact && btest(g, g.bits3, u, x),
               tvx = !exact && btest(g, g.bits3, v, x);
    if (exact) {
      if (btest(g, R + (size_t)u * g.n * bw, v, x)) return;  // {u, v, x}
    } else if (tuv && tux && tvx && has_triple(g, u, v, x)) {
      return;
    }
    const uint32_t* Ruv = exact ? R + ((size_t)u * g.n + v) * bw : nullptr;
    const uint32_t* Rux = exact ? R + ((size_t)u * g.n + x) * bw : nullptr;
    const uint32_t* Rvx = exact ? R + ((size_t)v * g.n + x) * bw : nullptr;
    const bool qd = btest(g, g.bits4, u, v) && btest(g, g.bits4, u, x) &&
                    btest(g, g.bits4, v, x);
    const bool c4ok = x > v;  // a 4-cycle is kept at its smallest pair: x > v, y > u
    const int32_t ul = u - base;
    const uint32_t *Bu = brow(g.bits2, bw, u), *Bv = brow(g.bits2, bw, v), *Bx = brow(g.bits2, bw, x);
    const uint32_t *Tu = brow(g.bits3, bw, u), *Tv = brow(g.bits3, bw, v), *Tx = brow(g.bits3, bw, x);
    const uint32_t *Qu = brow(g.bits4, bw, u), *Qv = brow(g.bits4, bw, v), *Qx = brow(g.bits4, bw, x);
    const int32_t uw = ul >> 5;
    const uint32_t ubit = 1u << (ul & 31);
    unsigned long long np = 0, nc = 0;
    for (int32_t w4 = 0; w4 < bw; w4 += 4) {
      uint32_t Y4[4], u4[4];
      ld4(Bv + w4, Y4);
      ld4(Bu + w4, u4);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Y4[k] &= ~u4[k];
        if (w4 + k == uw) Y4[k] &= ~ubit;
      }
      if (!(Y4[0] | Y4[1] | Y4[2] | Y4[3])) continue;
      if (exact) {
        uint32_t a4[4], b4[4], e4[4];
        ld4(Ruv + w4, a4);
        ld4(Rux + w4, b4);
        ld4(Rvx + w4, e4);
#pragma unroll
        for (int k = 0; k < 4; ++k) Y4[k] &= ~(a4[k] | b4[k] | e4[k]);
      }
      uint32_t bx4[4];
      ld4(Bx + w4, bx4);
      uint32_t rk4[4] = {0, 0, 0, 0};
      if (!exact && (tuv || tux || tvx)) {
        uint32_t tu4[4], tv4[4], tx4[4];
        ld4(Tu + w4, tu4);
        ld4(Tv + w4, tv4);
        ld4(Tx + w4, tx4);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          rk4[k] = (tuv ? tu4[k] & tv4[k] : 0u) | (tux ? tu4[k] & tx4[k] : 0u) |
                   (tvx ? tv4[k] & tx4[k] : 0u);
      }
      if (qd) {
        uint32_t qu4[4], qv4[4], qx4[4];
        ld4(Qu + w4, qu4);
        ld4(Qv + w4, qv4);
        ld4(Qx + w4, qx4);
#pragma unroll
        for (int k = 0; k < 4; ++k) rk4[k] |= qu4[k] & qv4[k] & qx4[k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int32_t w = w4 + k;
        const uint32_t Y = Y4[k];
        if (!Y) continue;
        const uint32_t bx = bx4[k], risky = rk4[k];
        const uint32_t c4 = c4ok ? (Y & bx & above(w, ul)) : 0u, p4 = Y & ~bx;
        np += __popc(p4 & ~risky);
        nc += __popc(c4 & ~risky);
        uint32_t rb = (c4 | p4) & risky;
        while (rb) {
          const int b = __ffs(rb) - 1;
          rb &= rb - 1;
          const int32_t y = base + w * 32 + b;
          if ((!exact && (has_triple(g, u, v, y) || has_triple(g, u, x, y) ||
                          has_triple(g, v, x, y))) ||
              has_quad(g, u, v, x, y))
            continue;
          if ((c4 >> b) & 1u)
            ++nc;
          else
            ++np;
        }
      }
    }
    if (np) atomicAdd(&bins[lut[19]], (Bin)np);  // u=0, v=1, x=2, y=3: pairs 01, 02, 13
    if (nc) atomicAdd(&bins[lut[51]], (Bin)nc);  // + pair 23
  }
};

// bits of word w whose (local) id is below t
__device__ __forceinline__ uint32_t below(int32_t w, int32_t t) {
  const int32_t tw = t >> 5;
  if (w < tw) return ~0u;
  if (w > tw) return 0u;
  const int32_t b = t & 31;
  return b == 0 ? 0u : (~0u >> (32 - b));
}
// the bit of (local) id t in word w, if it lies there
__device__ __forceinline__ uint32_t selfbit(int32_t w, int32_t t) {
  return (t >> 5) == w ? (1u << (t & 31)) : 0u;
}

}  // namespace fam
}  // namespace hm
