// The baseline of Sec. 4.1 (Alg. 1): enumerate the connected k-node subgraphs
// of the projection of the hypergraph (every pair of nodes that share any
// hyperedge, of any size), build the sub-hypergraph each induces (fill-in,
// Sec. 4.3) and count it by class when it is connected. A projection-
// connected set need not induce a connected sub-hypergraph (Fig. 2: the
// hyperedge that joins it may be larger than k); its mask then maps to no
// class and it is dropped. The result equals the exact census; the work is
// the number of projection-connected sets.
//
// The families walk the projection graph (the DevGraph the census kernel is
// given) with the canonical rules of simple graphs, each connected k-set
// once: a wedge or triangle at its smallest node of induced degree 2 (k = 3);
// a set with a node of induced degree 3 at its smallest such node, a path or
// 4-cycle at its smallest pair whose ends have induced degree 2 (k = 4).
// Fill-in probes the real hypergraph `h`.
#pragma once

#include "families.cuh"

namespace hm {
namespace base {

using fam::FamP;
using fam::FamS;
using fam::FamW;
using fam::unrank2;
using fam::unrank3;

// k = 3: centre v of the projection with neighbours x < y (positions i < j).
struct BaseW {
  static constexpr const char* kName = "baseline_W";
  static constexpr bool kDirect = false;
  DevGraph h;
  __device__ int32_t graph_node(const DevGraph&, int64_t v) const { return (int32_t)v; }
  using State = FamW::State;
  __device__ void begin(const DevGraph& g, int64_t v, uint64_t r, State& s) const {
    s.o = g.off2[v];
    unrank2(r, s.i, s.j);
  }
  __device__ void next(State& s) const { FamW{}.next(s); }
  __device__ bool item(const DevGraph& g, int64_t a, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int32_t v = (int32_t)a;
    const int32_t x = g.adj2[s.o + s.i], y = g.adj2[s.o + s.j];
    nd[0] = v;
    nd[1] = x;
    nd[2] = y;
    const bool pxy = has_pair(g, x, y);
    if (pxy && (x < v || y < v)) return false;  // a triangle at its smallest node
    // fill-in against the hypergraph (a pair absent from the projection is absent)
    // (a 3-hyperedge {v, x, y} needs the projection pair x - y)
    mask = (has_pair(h, v, x) ? 1u : 0u) | (has_pair(h, v, y) ? 2u : 0u) |
           ((pxy && has_pair(h, x, y)) ? 4u : 0u) | ((pxy && has_triple(h, v, x, y)) ? 8u : 0u);
    return true;
  }
};

// k = 4, a node of induced degree 3: centre v with neighbours x < y < z.
struct BaseS {
  static constexpr const char* kName = "baseline_S";
  static constexpr bool kDirect = false;
  DevGraph h;
  __device__ int32_t graph_node(const DevGraph&, int64_t v) const { return (int32_t)v; }
  using State = FamS::State;
  __device__ void begin(const DevGraph& g, int64_t v, uint64_t r, State& s) const {
    s.o = g.off2[v];
    unrank3(r, s.i, s.j, s.l);
  }
  __device__ void next(State& s) const { FamS{}.next(s); }
  __device__ bool item(const DevGraph& g, int64_t a, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int32_t v = (int32_t)a;
    const int32_t x = g.adj2[s.o + s.i], y = g.adj2[s.o + s.j], z = g.adj2[s.o + s.l];
    nd[0] = v;
    nd[1] = x;
    nd[2] = y;
    nd[3] = z;
    const bool pxy = has_pair(g, x, y), pxz = has_pair(g, x, z), pyz = has_pair(g, y, z);
    // v has induced degree 3 in the projection; keep the set at the smallest such node
    if ((pxy && pxz && x < v) || (pxy && pyz && y < v) || (pxz && pyz && z < v)) return false;
    // positions v = 0, x = 1, y = 2, z = 3; a 3- or 4-hyperedge needs the
    // projection pairs of all its members
    const bool all = pxy && pxz && pyz;
    mask = (has_pair(h, v, x) ? 1u : 0u) | (has_pair(h, v, y) ? 2u : 0u) |
           (has_pair(h, v, z) ? 4u : 0u) | ((pxy && has_pair(h, x, y)) ? 8u : 0u) |
           ((pxz && has_pair(h, x, z)) ? 16u : 0u) | ((pyz && has_pair(h, y, z)) ? 32u : 0u) |
           ((pxy && has_triple(h, v, x, y)) ? 64u : 0u) |
           ((pxz && has_triple(h, v, x, z)) ? 128u : 0u) |
           ((pyz && has_triple(h, v, y, z)) ? 256u : 0u) |
           ((all && has_triple(h, x, y, z)) ? 512u : 0u) |
           ((all && has_quad(h, v, x, y, z)) ? 1024u : 0u);
    return true;
  }
};

// k = 4, a path x - u - v - y or a 4-cycle: centre pair (u, v) of the projection.
struct BaseP {
  static constexpr const char* kName = "baseline_P";
  static constexpr bool kDirect = false;
  DevGraph h;
  __device__ int32_t graph_node(const DevGraph& g, int64_t p) const {
    return (int32_t)(g.e2[p] >> 32);
  }
  using State = FamP::State;
  __device__ void begin(const DevGraph& g, int64_t p, uint64_t r, State& s) const {
    FamP{}.begin(g, p, r, s);
  }
  __device__ void next(State& s) const { FamP{}.next(s); }
  __device__ bool item(const DevGraph& g, int64_t, State& s, uint32_t& mask,
                       int32_t (&nd)[4]) const {
    const int32_t u = s.u, v = s.v;
    const int32_t x = g.adj2[s.ou + s.i2 + (s.i2 >= s.pu ? 1 : 0)];  // N(u) \ {v}
    const int32_t y = g.adj2[s.ov + s.j2 + (s.j2 >= s.pv ? 1 : 0)];  // N(v) \ {u}
    nd[0] = u;
    nd[1] = v;
    nd[2] = x;
    nd[3] = y;
    if (x == y) return false;
    if (has_pair(g, u, y) || has_pair(g, v, x)) return false;  // a degree-3 node: BaseS
    const bool pxy = has_pair(g, x, y);
    if (pxy) {  // 4-cycle: kept at its smallest pair
      const uint64_t kuv = pair_key(u, v);
      if (pair_key(u, x) < kuv || pair_key(v, y) < kuv || pair_key(x, y) < kuv) return false;
    }
    // positions u = 0, v = 1, x = 2, y = 3. u - y and v - x are not projection
    // pairs, so no 3- or 4-hyperedge lies inside: only pairs can be present
    mask = (has_pair(h, u, v) ? 1u : 0u) | (has_pair(h, u, x) ? 2u : 0u) |
           (has_pair(h, v, y) ? 16u : 0u) | ((pxy && has_pair(h, x, y)) ? 32u : 0u);
    return true;
  }
};

}  // namespace base
}  // namespace hm
