// CPU oracle for higher-order motif counting in hypergraphs.
//
// TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
// CPU-baseline leg load this library. It shares no code with the CUDA path
// and is deliberately plain: every step follows the definitions of the paper
// ("Exact and sampling methods for mining higher-order motifs in large
// hypergraphs", Lotito et al.), with the section each step comes from.
//
// What it computes
//   * normalisation: a hyperedge is a set of nodes (Def. 1, Sec. 3); repeated
//     members collapse, singletons are ignored (Sec. 4.3 skips the empty set
//     and singletons), duplicate hyperedges collapse because E is a set.
//   * exact census (problem statement, Sec. 3): for order k, hist[c] is the
//     number of k-node sets V' whose induced sub-hypergraph H[V'] (Def. 2) is
//     connected and belongs to isomorphism class c (Def. 3). The enumeration
//     follows Alg. 1 (Sec. 4.1): ESU over a projection, fill-in of the
//     candidate (Sec. 4.3), connectivity check, class by brute force over the
//     k! relabelings (Sec. 4.3), count. The projection only uses hyperedges of
//     size 2..k: a larger hyperedge never lies inside a k-node set, so it
//     cannot make H[V'] connected (the failure case of Fig. 2).
//   * sampling estimator (Alg. 4, Sec. 5): stratified draws with replacement,
//     enumeration of the connected k-node sets containing the drawn hyperedge,
//     the max-cardinality filter, and the correction factor.
//   * per-hyperedge contributions: for each counted set, credit each of its
//     maximum-cardinality hyperedges (the quantity whose sampling Alg. 4
//     estimates, Sec. 5).
//   * stub-shuffling null model (configuration-model stand-in, Sec. 6.3).
//   * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
//     as easy as 1, 2, 3", SC'11), written from the published definition.
//
// Mask layout (shared by specification with the CUDA path, not by code):
// subsets of the k sorted positions with size 2..k, ordered by size and then
// lexicographically; k=3: {01,02,12,012}; k=4: {01,02,03,12,13,23,012,013,
// 023,123,0123}. Class id = rank of the canonical mask (minimum over all k!
// relabelings) among the connected classes, ascending.

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Tuple = std::array<int32_t, 4>;  // sorted members, unused slots = -1

struct TupleHash {
  size_t operator()(const Tuple& t) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 4; ++i) {
      h ^= (uint32_t)t[i];
      h *= 1099511628211ull;
    }
    return (size_t)h;
  }
};

Tuple make_tuple(const int32_t* sorted_nodes, int s) {
  Tuple t;
  for (int i = 0; i < 4; ++i) t[i] = i < s ? sorted_nodes[i] : -1;
  return t;
}

// ---------------------------------------------------------------- classes
struct Classes {
  int k = 0;
  int nsub = 0;
  uint32_t sub[11];   // node bitmask of subset b
  int sub_size[11];
  std::vector<uint32_t> canon;  // canonical masks of connected classes, ascending
  std::vector<int> maxcard, countmax;
};

int subset_index(const Classes& C, uint32_t nodes) {
  for (int b = 0; b < C.nsub; ++b)
    if (C.sub[b] == nodes) return b;
  return -1;
}

uint32_t relabel(const Classes& C, uint32_t mask, const int* perm) {
  uint32_t out = 0;
  for (int b = 0; b < C.nsub; ++b) {
    if (!((mask >> b) & 1u)) continue;
    uint32_t mapped = 0;
    for (int i = 0; i < C.k; ++i)
      if ((C.sub[b] >> i) & 1u) mapped |= 1u << perm[i];
    out |= 1u << subset_index(C, mapped);
  }
  return out;
}

uint32_t canonical(const Classes& C, uint32_t mask) {
  int perm[4] = {0, 1, 2, 3};
  uint32_t best = mask;
  do {
    uint32_t r = relabel(C, mask, perm);
    if (r < best) best = r;
  } while (std::next_permutation(perm, perm + C.k));
  return best;
}

// H[V'] connected: the nodes are joined by the hyperedges present (Sec. 3).
bool connected(const Classes& C, uint32_t mask) {
  int parent[4] = {0, 1, 2, 3};
  auto find = [&](int x) {
    while (parent[x] != x) x = parent[x];
    return x;
  };
  for (int b = 0; b < C.nsub; ++b) {
    if (!((mask >> b) & 1u)) continue;
    int first = -1;
    for (int i = 0; i < C.k; ++i) {
      if (!((C.sub[b] >> i) & 1u)) continue;
      if (first < 0) {
        first = i;
      } else {
        int a = find(first), c = find(i);
        if (a != c) parent[c] = a;
      }
    }
  }
  int r0 = find(0);
  for (int i = 1; i < C.k; ++i)
    if (find(i) != r0) return false;
  return true;
}

void mask_maxcard(const Classes& C, uint32_t mask, int* maxcard, int* countmax) {
  int mc = 0, cm = 0;
  for (int b = 0; b < C.nsub; ++b) {
    if (!((mask >> b) & 1u)) continue;
    if (C.sub_size[b] > mc) {
      mc = C.sub_size[b];
      cm = 1;
    } else if (C.sub_size[b] == mc) {
      ++cm;
    }
  }
  *maxcard = mc;
  *countmax = cm;
}

Classes build_classes(int k) {
  Classes C;
  C.k = k;
  // subsets of {0..k-1} of size 2..k, by size, then lexicographic
  for (int s = 2; s <= k; ++s) {
    std::vector<int> sel(k, 0);
    std::fill(sel.begin(), sel.begin() + s, 1);
    // prev_permutation on a 1..10..0 vector walks the s-combinations
    // in lexicographic order of the chosen positions
    do {
      uint32_t m = 0;
      for (int i = 0; i < k; ++i)
        if (sel[i]) m |= 1u << i;
      C.sub[C.nsub] = m;
      C.sub_size[C.nsub] = s;
      ++C.nsub;
    } while (std::prev_permutation(sel.begin(), sel.end()));
  }
  std::set<uint32_t> canon;
  for (uint32_t mask = 0; mask < (1u << C.nsub); ++mask)
    if (connected(C, mask)) canon.insert(canonical(C, mask));
  C.canon.assign(canon.begin(), canon.end());
  for (uint32_t cm : C.canon) {
    int a, b;
    mask_maxcard(C, cm, &a, &b);
    C.maxcard.push_back(a);
    C.countmax.push_back(b);
  }
  return C;
}

const Classes& classes(int k) {
  static const Classes c3 = build_classes(3);
  static const Classes c4 = build_classes(4);
  return k == 3 ? c3 : c4;
}

int class_of(const Classes& C, uint32_t mask) {
  if (!connected(C, mask)) return -1;
  uint32_t cm = canonical(C, mask);
  auto it = std::lower_bound(C.canon.begin(), C.canon.end(), cm);
  return (int)(it - C.canon.begin());
}

// ---------------------------------------------------------------- graph
struct Graph {
  int32_t n = 0;
  int kmax = 0;
  std::vector<std::vector<Tuple>> E;  // E[s]: distinct hyperedges of size s, ascending
  int64_t big = 0;                    // input hyperedges whose distinct size > kmax
  std::unordered_map<Tuple, int64_t, TupleHash> index;  // tuple -> position in E[s]
};

Graph* build_graph(const int32_t* members, const int64_t* offsets, int64_t m, int32_t n,
                   int kmax) {
  Graph* g = new Graph;
  g->n = n;
  g->kmax = kmax;
  g->E.resize(kmax + 1);
  std::vector<std::set<Tuple>> sets(kmax + 1);
  std::vector<int32_t> buf;
  for (int64_t j = 0; j < m; ++j) {
    buf.assign(members + offsets[j], members + offsets[j + 1]);
    std::sort(buf.begin(), buf.end());
    buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
    int s = (int)buf.size();
    if (s < 2) continue;
    if (s > kmax) {
      ++g->big;
      continue;
    }
    sets[s].insert(make_tuple(buf.data(), s));
  }
  for (int s = 2; s <= kmax; ++s) {
    g->E[s].assign(sets[s].begin(), sets[s].end());
    for (size_t i = 0; i < g->E[s].size(); ++i) g->index[g->E[s][i]] = (int64_t)i;
  }
  return g;
}

bool has_edge(const Graph& g, const int32_t* sorted_nodes, int s) {
  if (s > g.kmax) return false;
  return g.index.count(make_tuple(sorted_nodes, s)) != 0;
}

// Projection (Def. 4, Sec. 4.1) restricted to hyperedges of size 2..k.
std::vector<std::vector<int32_t>> projection(const Graph& g, int k) {
  std::vector<std::vector<int32_t>> adj(g.n);
  for (int s = 2; s <= k && s <= g.kmax; ++s)
    for (const Tuple& t : g.E[s])
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b)
          if (a != b) adj[t[a]].push_back(t[b]);
  for (auto& l : adj) {
    std::sort(l.begin(), l.end());
    l.erase(std::unique(l.begin(), l.end()), l.end());
  }
  return adj;
}

bool adjacent(const std::vector<std::vector<int32_t>>& adj, int32_t a, int32_t b) {
  return std::binary_search(adj[a].begin(), adj[a].end(), b);
}

// Fill-in (Sec. 4.3): probe every subset of size 2..k of the candidate set.
uint32_t fill_in(const Graph& g, const Classes& C, const int32_t* sorted_nodes) {
  uint32_t mask = 0;
  for (int b = 0; b < C.nsub; ++b) {
    int32_t t[4];
    int s = 0;
    for (int i = 0; i < C.k; ++i)
      if ((C.sub[b] >> i) & 1u) t[s++] = sorted_nodes[i];
    if (has_edge(g, t, s)) mask |= 1u << b;
  }
  return mask;
}

// ESU (Wernicke 2006): every connected k-node set of the graph exactly once,
// rooted at its smallest node.
template <class Visit>
void esu_extend(const std::vector<std::vector<int32_t>>& adj, int k, std::vector<int32_t>& sub,
                std::vector<int32_t> ext, int32_t root, Visit& visit) {
  if ((int)sub.size() == k) {
    visit(sub);
    return;
  }
  while (!ext.empty()) {
    int32_t w = ext.back();
    ext.pop_back();
    std::vector<int32_t> ext2 = ext;
    for (int32_t u : adj[w]) {
      if (u <= root) continue;
      bool exclusive = true;
      for (int32_t x : sub)
        if (u == x || adjacent(adj, x, u)) {
          exclusive = false;
          break;
        }
      if (exclusive) ext2.push_back(u);
    }
    sub.push_back(w);
    esu_extend(adj, k, sub, ext2, root, visit);
    sub.pop_back();
  }
}

template <class MakeVisitor>
void esu_parallel(const Graph& g, int k, int nthreads, int64_t root_lo, int64_t root_hi,
                  MakeVisitor make_visitor) {
  auto adj = projection(g, k);
  if (root_hi > g.n) root_hi = g.n;
  if (root_lo < 0) root_lo = 0;
  std::atomic<int64_t> next(root_lo);
  auto work = [&](int tid) {
    auto visit = make_visitor(tid);
    std::vector<int32_t> sub;
    for (;;) {
      int64_t v = next.fetch_add(1);
      if (v >= root_hi) break;
      std::vector<int32_t> ext;
      for (int32_t u : adj[v])
        if (u > v) ext.push_back(u);
      sub.assign(1, (int32_t)v);
      esu_extend(adj, k, sub, ext, (int32_t)v, visit);
    }
  };
  if (nthreads <= 1) {
    work(0);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t) th.emplace_back(work, t);
  for (auto& t : th) t.join();
}

// ---------------------------------------------------------------- philox
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

uint64_t draw64(uint64_t seed, uint64_t index, uint32_t lane, uint32_t tag) {
  uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32), lane, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  philox4x32_10(ctr, key, o);
  return ((uint64_t)o[0] << 32) | o[1];
}

uint64_t mulhi64(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
}

const uint32_t TAG_SAMPLE = 0x53414D50u;  // "SAMP"
const uint32_t TAG_NULL = 0x4E554C4Cu;    // "NULL"

// Index drawn for sample t of stratum s: uniform over E_s, or proportional to
// the weights q (exclusive prefix sums P, total P[len]).
int64_t draw_index(uint64_t seed, int s, uint64_t t, int64_t len, const uint64_t* P) {
  uint64_t d = draw64(seed, t, (uint32_t)s, TAG_SAMPLE);
  if (!P) return (int64_t)mulhi64(d, (uint64_t)len);
  uint64_t r = mulhi64(d, P[len]);
  const uint64_t* it = std::upper_bound(P, P + len + 1, r);
  return (int64_t)(it - P) - 1;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

uint64_t orc_draw64(uint64_t seed, uint64_t index, uint32_t lane, uint32_t tag) {
  return draw64(seed, index, lane, tag);
}

int orc_num_classes(int k) {
  if (k != 3 && k != 4) return -1;
  return (int)classes(k).canon.size();
}

// canonical mask, maxcard and countmax of every class of order k
void orc_class_info(int k, uint32_t* canon, int32_t* maxcard, int32_t* countmax) {
  const Classes& C = classes(k);
  for (size_t c = 0; c < C.canon.size(); ++c) {
    canon[c] = C.canon[c];
    maxcard[c] = C.maxcard[c];
    countmax[c] = C.countmax[c];
  }
}

// class id of a labelled mask, -1 when the pattern is not connected
int orc_class_of(int k, uint32_t mask) { return class_of(classes(k), mask); }
uint32_t orc_canonical(int k, uint32_t mask) { return canonical(classes(k), mask); }
int orc_connected(int k, uint32_t mask) { return connected(classes(k), mask) ? 1 : 0; }

void* orc_graph_new(const int32_t* members, const int64_t* offsets, int64_t m, int32_t n,
                    int kmax) {
  return build_graph(members, offsets, m, n, kmax);
}

void orc_graph_free(void* g) { delete (Graph*)g; }

// s in 2..kmax: distinct hyperedges of size s; s == kmax+1: input hyperedges
// whose distinct size exceeds kmax
int64_t orc_graph_count(void* gp, int s) {
  const Graph& g = *(Graph*)gp;
  if (s == g.kmax + 1) return g.big;
  if (s < 2 || s > g.kmax) return 0;
  return (int64_t)g.E[s].size();
}

// E_s in ascending order, s members per row
void orc_graph_edges(void* gp, int s, int32_t* out) {
  const Graph& g = *(Graph*)gp;
  for (size_t i = 0; i < g.E[s].size(); ++i)
    for (int a = 0; a < s; ++a) out[i * s + a] = g.E[s][i][a];
}

// labelled mask of a k-node set (nodes given in any order)
uint32_t orc_fill_in(void* gp, int k, const int32_t* nodes) {
  int32_t s[4];
  std::copy(nodes, nodes + k, s);
  std::sort(s, s + k);
  return fill_in(*(Graph*)gp, classes(k), s);
}

// Exact census (problem statement, Sec. 3; enumeration as in Alg. 1) over the
// ESU roots in [root_lo, root_hi). hist has orc_num_classes(k) entries.
// Returns the number of connected candidate sets ESU produced.
int64_t orc_census(void* gp, int k, int nthreads, int64_t root_lo, int64_t root_hi,
                   uint64_t* hist) {
  const Graph& g = *(Graph*)gp;
  const Classes& C = classes(k);
  int nt = nthreads < 1 ? 1 : nthreads;
  std::vector<std::vector<uint64_t>> part(nt, std::vector<uint64_t>(C.canon.size(), 0));
  std::vector<int64_t> cand(nt, 0);
  esu_parallel(g, k, nt, root_lo, root_hi, [&](int tid) {
    return [&, tid](const std::vector<int32_t>& sub) {
      int32_t s[4];
      std::copy(sub.begin(), sub.end(), s);
      std::sort(s, s + k);
      ++cand[tid];
      int c = class_of(C, fill_in(g, C, s));
      if (c >= 0) ++part[tid][c];
    };
  });
  int64_t total = 0;
  for (size_t c = 0; c < C.canon.size(); ++c) {
    uint64_t v = 0;
    for (int t = 0; t < nt; ++t) v += part[t][c];
    hist[c] = v;
  }
  for (int t = 0; t < nt; ++t) total += cand[t];
  return total;
}

// Per-hyperedge contributions: contrib[row * ncls + c] counts the connected
// k-node sets of class c in which hyperedge `row` is one of the hyperedges of
// maximum cardinality. Rows: E_2, then E_3, ..., E_k (ascending within each).
// Returns 0, or 1 if a uint32 counter saturated.
int orc_contributions(void* gp, int k, int nthreads, uint32_t* contrib) {
  const Graph& g = *(Graph*)gp;
  const Classes& C = classes(k);
  const int ncls = (int)C.canon.size();
  std::vector<int64_t> base(k + 2, 0);
  for (int s = 2; s <= k; ++s) base[s + 1] = base[s] + (int64_t)g.E[s].size();
  std::atomic<int> saturated(0);
  esu_parallel(g, k, nthreads < 1 ? 1 : nthreads, 0, g.n, [&](int) {
    return [&](const std::vector<int32_t>& sub) {
      int32_t s[4];
      std::copy(sub.begin(), sub.end(), s);
      std::sort(s, s + k);
      uint32_t mask = fill_in(g, C, s);
      int c = class_of(C, mask);
      if (c < 0) return;
      int mc, cm;
      mask_maxcard(C, mask, &mc, &cm);
      for (int b = 0; b < C.nsub; ++b) {
        if (!((mask >> b) & 1u) || C.sub_size[b] != mc) continue;
        int32_t t[4];
        int sz = 0;
        for (int i = 0; i < k; ++i)
          if ((C.sub[b] >> i) & 1u) t[sz++] = s[i];
        int64_t row = base[sz] + g.index.at(make_tuple(t, sz));
        uint32_t old = __atomic_fetch_add(&contrib[row * ncls + c], 1u, __ATOMIC_RELAXED);
        if (old == 0xFFFFFFFFu) saturated = 1;
      }
    };
  });
  return saturated.load();
}

// Drawn hyperedge indices (position within E_s) for stratum s, samples
// [0, count). q: weights of E_s (NULL = uniform), each >= 1.
void orc_sample_indices(void* gp, int s, uint64_t count, uint64_t seed, const uint32_t* q,
                        int64_t* out) {
  const Graph& g = *(Graph*)gp;
  int64_t len = (int64_t)g.E[s].size();
  std::vector<uint64_t> P;
  if (q) {
    P.assign(len + 1, 0);
    for (int64_t i = 0; i < len; ++i) P[i + 1] = P[i] + q[i];
  }
  for (uint64_t t = 0; t < count; ++t) out[t] = draw_index(seed, s, t, len, q ? P.data() : nullptr);
}

// Alg. 4 (Sec. 5), for order k in {3,4}.
//   samples[s], s = 0..k: S_s (entries 0 and 1 ignored).
//   q: NULL (uniform within each stratum) or the weights of E_2, E_3, ..., E_k
//      concatenated (each >= 1); draws are then proportional to q and every
//      counted set is reweighted by floor(2^63 / q_e) (Hansen-Hurwitz).
//   raw: 2 * ncls uint64. Uniform: raw[2c] = count, raw[2c+1] = 0.
//        Weighted: (raw[2c+1], raw[2c]) = high and low words of the 128-bit sum.
//   est: ncls doubles, the corrected estimate of Alg. 4's last loop.
// Returns the number of (sample, set) pairs enumerated before the filter.
int64_t orc_sample(void* gp, int k, const uint64_t* samples, uint64_t seed, const uint32_t* q,
                   uint64_t* raw, double* est) {
  const Graph& g = *(Graph*)gp;
  const Classes& C = classes(k);
  const int ncls = (int)C.canon.size();
  auto adj = projection(g, k);
  std::vector<unsigned __int128> acc(ncls, 0);
  std::vector<uint64_t> Q(k + 1, 0);
  int64_t enumerated = 0;
  int64_t qoff = 0;
  for (int s = 2; s <= k; ++s) {
    int64_t len = (int64_t)g.E[s].size();
    std::vector<uint64_t> P;
    if (q) {
      P.assign(len + 1, 0);
      for (int64_t i = 0; i < len; ++i) P[i + 1] = P[i] + q[qoff + i];
      Q[s] = P[len];
    } else {
      Q[s] = (uint64_t)len;
    }
    if (len == 0) {
      qoff += len;
      continue;
    }
    for (uint64_t t = 0; t < samples[s]; ++t) {
      int64_t idx = draw_index(seed, s, t, len, q ? P.data() : nullptr);
      const Tuple& e = g.E[s][idx];
      uint64_t weight = q ? ((uint64_t)1 << 63) / q[qoff + idx] : 1;
      // connected supersets of e with k nodes, grown one neighbour at a time
      std::set<Tuple> cur;
      cur.insert(e);
      for (int size = s; size < k; ++size) {
        std::set<Tuple> next;
        for (const Tuple& X : cur) {
          for (int a = 0; a < size; ++a)
            for (int32_t u : adj[X[a]]) {
              if (std::find(X.begin(), X.begin() + size, u) != X.begin() + size) continue;
              int32_t y[4];
              std::copy(X.begin(), X.begin() + size, y);
              y[size] = u;
              std::sort(y, y + size + 1);
              next.insert(make_tuple(y, size + 1));
            }
        }
        cur.swap(next);
      }
      for (const Tuple& V : cur) {
        ++enumerated;
        uint32_t mask = fill_in(g, C, V.data());
        int c = class_of(C, mask);
        if (c < 0) continue;
        int mc, cm;
        mask_maxcard(C, mask, &mc, &cm);
        if (mc > s) continue;  // contains a hyperedge larger than e
        acc[c] += weight;
      }
    }
    qoff += len;
  }
  for (int c = 0; c < ncls; ++c) {
    raw[2 * c] = (uint64_t)acc[c];
    raw[2 * c + 1] = (uint64_t)(acc[c] >> 64);
    int m = C.maxcard[c];
    double Sm = (double)samples[m];
    double denom = Sm * (double)C.countmax[c];
    if (samples[m] == 0 || g.E[m].empty()) {
      est[c] = 0.0;
      continue;
    }
    double a;
    if (q) {
      double hi = (double)raw[2 * c + 1];
      double lo = (double)raw[2 * c];
      a = hi * 18446744073709551616.0 + lo;
      a = a * 0x1p-63;
    } else {
      a = (double)raw[2 * c];
    }
    est[c] = (a * (double)Q[m]) / denom;
  }
  return enumerated;
}

// Stub-shuffling null model (configuration-model stand-in, Sec. 6.3): the
// stubs (members in input order) are reordered by the keys
// (draw64(seed, i, model, TAG_NULL) >> 6, i) and cut again into the input
// sizes. out_members has offsets[m] entries; the offsets stay the same.
void orc_stub_shuffle(const int32_t* members, const int64_t* offsets, int64_t m, uint64_t seed,
                      uint32_t model, int32_t* out_members) {
  int64_t M = offsets[m];
  std::vector<std::pair<uint64_t, int64_t>> key(M);
  for (int64_t i = 0; i < M; ++i) key[i] = {draw64(seed, (uint64_t)i, model, TAG_NULL) >> 6, i};
  std::sort(key.begin(), key.end());
  for (int64_t i = 0; i < M; ++i) out_members[i] = members[key[i].second];
}

// Configuration model of hypergraphs (the null model Sec. 6.3 cites, by
// Chodrow), sampled by its pairwise-reshuffle Markov chain: two hyperedges e,
// f keep their intersection and deal the remaining members of both out again
// at random, |e| - |e n f| to e and the rest to f, which keeps every degree
// and size. Round r (of `sweeps`) pairs the hyperedges by a random matching:
// hyperedge i gets the key draw64(seed, (r << 32) | i, model << 8, TAG_MCMC)
// >> 6, the hyperedges are sorted by (key, i), and positions 2k and 2k + 1
// form pair k (an odd one out stays). In pair k the re-dealt members are S =
// e's members outside f (in order) then f's outside e, with their slots;
// Fisher-Yates steps q = 0, 1, ... while q < |e \ f| and q < |S| - 1 swap S[q]
// with S[q + mulhi64(draw64(seed, (r << 32) | k, (model << 8) | (q + 1),
// TAG_MCMC), |S| - q)], and S goes back to the slots in order. Pairs whose S
// has more than 255 members, fewer than 2, or lies wholly in e or in f stay
// as they are. out_members has offsets[m] entries; the offsets stay the same.
void orc_config_mcmc(const int32_t* members, const int64_t* offsets, int64_t m, uint64_t seed,
                     uint32_t model, int sweeps, int32_t* out_members) {
  const uint32_t TAG_MCMC = 0x4D434D43u;  // "MCMC"
  const int64_t M = offsets[m];
  for (int64_t i = 0; i < M; ++i) out_members[i] = members[i];
  for (int r = 0; r < sweeps; ++r) {
    std::vector<std::pair<uint64_t, int64_t>> key(m);
    for (int64_t i = 0; i < m; ++i)
      key[i] = {draw64(seed, ((uint64_t)r << 32) | (uint64_t)i, model << 8, TAG_MCMC) >> 6, i};
    std::sort(key.begin(), key.end());
    for (int64_t k = 0; 2 * k + 1 < m; ++k) {
      const int64_t e = key[2 * k].second, f = key[2 * k + 1].second;
      std::vector<int32_t> S;
      std::vector<int64_t> slot;
      auto in = [&](int64_t h, int32_t v) {
        for (int64_t j = offsets[h]; j < offsets[h + 1]; ++j)
          if (out_members[j] == v) return true;
        return false;
      };
      for (int64_t j = offsets[e]; j < offsets[e + 1]; ++j)
        if (!in(f, out_members[j])) {
          S.push_back(out_members[j]);
          slot.push_back(j);
        }
      const int ae = (int)S.size();
      for (int64_t j = offsets[f]; j < offsets[f + 1]; ++j)
        if (!in(e, out_members[j])) {
          S.push_back(out_members[j]);
          slot.push_back(j);
        }
      const int ns = (int)S.size();
      if (ns > 255 || ns < 2 || ae == 0 || ae == ns) continue;
      for (int q = 0; q < ae && q < ns - 1; ++q) {
        const uint64_t v =
            draw64(seed, ((uint64_t)r << 32) | (uint64_t)k, (model << 8) | (uint32_t)(q + 1), TAG_MCMC);
        const int j = q + (int)mulhi64(v, (uint64_t)(ns - q));
        std::swap(S[q], S[j]);
      }
      for (int q = 0; q < ns; ++q) out_members[slot[q]] = S[q];
    }
  }
}


// ---------------------------------------------------------------- order 5 (Sec. 6.4)
// Alg. 4 at order 5. A 5-node pattern is a 26-bit mask over the subsets of
// its 5 sorted positions with 2..5 members (by size, then lexicographic: bits
// 0-9 pairs 01..34, 10-19 triples 012..234, 20-24 quads 0123..1234, 25 the
// five). There is no class table: a class is its canonical mask, the minimum
// over the 120 relabelings. For a drawn hyperedge e, the sets counted are the
// 5-node V' containing e whose H[V'] is connected and whose largest
// hyperedges have |e| members; every such V' is connected in the projection
// of the hyperedges of size <= |e| (the only hyperedges inside it), so it can
// be grown from e by adding projection neighbours one at a time, and the
// oracle tries every set grown that way. Draw t of stratum s is hyperedge
// mulhi64(draw64(seed, t, s, "SAMP"), |E_s|) of E_s (ascending tuples).
namespace o5 {

struct Sub5 {
  uint32_t nodes[26];  // node bitmask of subset b
  int size[26];
  int index_of[32];    // node bitmask -> subset index, -1 for size < 2
  std::vector<std::array<uint8_t, 26>> perm_map;  // per relabeling: b -> image subset
};

const Sub5& sub5() {
  static Sub5 S = [] {
    Sub5 t;
    for (int i = 0; i < 32; ++i) t.index_of[i] = -1;
    int b = 0;
    // combinations of each size in lexicographic order
    for (int sz = 2; sz <= 5; ++sz) {
      std::vector<int> c(sz);
      for (int i = 0; i < sz; ++i) c[i] = i;
      while (true) {
        uint32_t m = 0;
        for (int i = 0; i < sz; ++i) m |= 1u << c[i];
        t.nodes[b] = m;
        t.size[b] = sz;
        t.index_of[m] = b;
        ++b;
        int i = sz - 1;
        while (i >= 0 && c[i] == 5 - sz + i) --i;
        if (i < 0) break;
        ++c[i];
        for (int j = i + 1; j < sz; ++j) c[j] = c[j - 1] + 1;
      }
    }
    int perm[5] = {0, 1, 2, 3, 4};
    do {
      std::array<uint8_t, 26> pm;
      for (int q = 0; q < 26; ++q) {
        uint32_t img = 0;
        for (int i = 0; i < 5; ++i)
          if ((t.nodes[q] >> i) & 1u) img |= 1u << perm[i];
        pm[q] = (uint8_t)t.index_of[img];
      }
      t.perm_map.push_back(pm);
    } while (std::next_permutation(perm, perm + 5));
    return t;
  }();
  return S;
}

uint32_t canonical5(uint32_t mask) {
  const Sub5& S = sub5();
  uint32_t best = mask;
  for (const auto& pm : S.perm_map) {
    uint32_t r = 0;
    for (int q = 0; q < 26; ++q)
      if ((mask >> q) & 1u) r |= 1u << pm[q];
    best = std::min(best, r);
  }
  return best;
}

bool connected5(uint32_t mask) {
  const Sub5& S = sub5();
  int parent[5] = {0, 1, 2, 3, 4};
  auto find = [&](int x) {
    while (parent[x] != x) x = parent[x];
    return x;
  };
  for (int q = 0; q < 26; ++q) {
    if (!((mask >> q) & 1u)) continue;
    int first = -1;
    for (int i = 0; i < 5; ++i) {
      if (!((S.nodes[q] >> i) & 1u)) continue;
      if (first < 0) first = i;
      else parent[find(i)] = find(first);
    }
  }
  const int r = find(0);
  for (int i = 1; i < 5; ++i)
    if (find(i) != r) return false;
  return true;
}

// (largest hyperedge size, how many hyperedges of that size) of a mask
void maxcard5(uint32_t mask, int* mc, int* cm) {
  const Sub5& S = sub5();
  *mc = 0;
  *cm = 0;
  for (int q = 0; q < 26; ++q) {
    if (!((mask >> q) & 1u)) continue;
    if (S.size[q] > *mc) {
      *mc = S.size[q];
      *cm = 1;
    } else if (S.size[q] == *mc) {
      ++*cm;
    }
  }
}

struct Graph5 {
  int32_t n = 0;
  std::vector<std::vector<int32_t>> E[6];  // distinct sorted hyperedges of size s, ascending
  std::set<std::vector<int32_t>> all;      // every distinct hyperedge of size 2..5
  std::vector<std::vector<int32_t>> adj[6];  // adj[s]: projection of sizes 2..s, sorted
};

Graph5 make_graph5(const int32_t* members, const int64_t* offsets, int64_t m, int32_t n) {
  Graph5 g;
  g.n = n;
  std::set<std::vector<int32_t>> bysize[6];
  for (int64_t j = 0; j < m; ++j) {
    std::vector<int32_t> e(members + offsets[j], members + offsets[j + 1]);
    std::sort(e.begin(), e.end());
    e.erase(std::unique(e.begin(), e.end()), e.end());
    if (e.size() < 2 || e.size() > 5) continue;
    bysize[e.size()].insert(e);
    g.all.insert(e);
  }
  for (int s = 2; s <= 5; ++s) g.E[s].assign(bysize[s].begin(), bysize[s].end());
  for (int s = 2; s <= 5; ++s) {
    std::vector<std::set<int32_t>> nb(n);
    for (int t = 2; t <= s; ++t)
      for (const auto& e : g.E[t])
        for (int32_t a : e)
          for (int32_t b : e)
            if (a != b) nb[a].insert(b);
    g.adj[s].resize(n);
    for (int v = 0; v < n; ++v) g.adj[s][v].assign(nb[v].begin(), nb[v].end());
  }
  return g;
}

// mask of the 5-node set (sorted nodes v[0..4])
uint32_t fill5(const Graph5& g, const int32_t* v) {
  const Sub5& S = sub5();
  uint32_t mask = 0;
  for (int q = 0; q < 26; ++q) {
    std::vector<int32_t> t;
    for (int i = 0; i < 5; ++i)
      if ((S.nodes[q] >> i) & 1u) t.push_back(v[i]);
    if (g.all.count(t)) mask |= 1u << q;
  }
  return mask;
}

// every counted set through hyperedge e: adds 1 to counts[canonical mask].
// The candidate 5-sets are grown from e one node at a time, each new node a
// projection neighbour (sizes <= |e|) of the set so far; distinct sets are
// kept at every size, so each candidate is tried once.
void sets_through(const Graph5& g, const std::vector<int32_t>& e,
                  std::map<uint32_t, uint64_t>& counts) {
  const int s = (int)e.size();
  std::set<std::vector<int32_t>> level = {e};
  for (int size = s; size < 5; ++size) {
    std::set<std::vector<int32_t>> next;
    for (const auto& cur : level)
      for (int32_t x : cur)
        for (int32_t y : g.adj[s][x]) {
          if (std::binary_search(cur.begin(), cur.end(), y)) continue;
          std::vector<int32_t> grown = cur;
          grown.insert(std::upper_bound(grown.begin(), grown.end(), y), y);
          next.insert(grown);
        }
    level.swap(next);
  }
  for (const auto& v : level) {
    const uint32_t mask = fill5(g, v.data());
    int mc, cm;
    maxcard5(mask, &mc, &cm);
    if (mc != s || !connected5(mask)) continue;
    ++counts[canonical5(mask)];
  }
}

int64_t write_out(const std::map<uint32_t, uint64_t>& counts, int64_t cap, uint32_t* masks,
                  uint64_t* vals) {
  int64_t i = 0;
  for (const auto& kv : counts) {
    if (i < cap) {
      masks[i] = kv.first;
      vals[i] = kv.second;
    }
    ++i;
  }
  return i;
}

}  // namespace o5

// Alg. 4 at order 5 (uniform draws). S: draws per stratum, S[s] for s = 2..5.
// Writes up to cap classes in ascending canonical mask: masks, raw counts n_c,
// estimates (n_c |E_m|) / (S_m countmax_c) in IEEE double, m = the class's
// largest hyperedge size. Returns the number of classes met.
int64_t orc_sample5(const int32_t* members, const int64_t* offsets, int64_t m, int32_t n,
                    const uint64_t* S, uint64_t seed, int64_t cap, uint32_t* masks, uint64_t* raw,
                    double* est) {
  const o5::Graph5 g = o5::make_graph5(members, offsets, m, n);
  std::map<uint32_t, uint64_t> counts;
  for (int s = 2; s <= 5; ++s) {
    const uint64_t len = g.E[s].size();
    if (len == 0) continue;
    for (uint64_t t = 0; t < S[s]; ++t) {
      const uint64_t idx = mulhi64(draw64(seed, t, (uint32_t)s, TAG_SAMPLE), len);
      o5::sets_through(g, g.E[s][idx], counts);
    }
  }
  const int64_t nc = o5::write_out(counts, cap, masks, raw);
  int64_t i = 0;
  for (const auto& kv : counts) {
    if (i >= cap) break;
    int mc, cm;
    o5::maxcard5(kv.first, &mc, &cm);
    const double denom = (double)S[mc] * (double)cm;
    est[i] = S[mc] ? ((double)kv.second * (double)g.E[mc].size()) / denom : 0.0;
    ++i;
  }
  return nc;
}

// Every hyperedge of size 2..5 taken once (no sampling): sum over e of the
// counted sets through e, per canonical mask. Equals countmax_c times the
// exact order-5 count of class c (each set is counted once per hyperedge of
// maximum cardinality it holds).
int64_t orc_sweep5(const int32_t* members, const int64_t* offsets, int64_t m, int32_t n,
                   int64_t cap, uint32_t* masks, uint64_t* sums) {
  const o5::Graph5 g = o5::make_graph5(members, offsets, m, n);
  std::map<uint32_t, uint64_t> counts;
  for (int s = 2; s <= 5; ++s)
    for (const auto& e : g.E[s]) o5::sets_through(g, e, counts);
  return o5::write_out(counts, cap, masks, sums);
}

uint32_t orc_canonical5(uint32_t mask) { return o5::canonical5(mask); }
int orc_connected5(uint32_t mask) { return o5::connected5(mask) ? 1 : 0; }
}  // extern "C"
