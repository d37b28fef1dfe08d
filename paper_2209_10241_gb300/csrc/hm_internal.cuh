// Internal definitions of the CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "hm.h"

namespace hm {

// ------------------------------------------------------------------ errors
struct Error : std::runtime_error {
  hm_status code;
  Error(hm_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

#define HM_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw ::hm::Error(e_ == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA,         \
                        std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

// Kernels launched by the library (all devices, all threads).
uint64_t launch_count_add(uint64_t n);

// check a kernel launch and count it
#define HM_KCHECK()                                   \
  do {                                                \
    ::hm::launch_count_add(1);                        \
    HM_CUDA(cudaGetLastError());                      \
  } while (0)

#define HM_CHECK(cond, code, msg)                       \
  do {                                                  \
    if (!(cond)) throw ::hm::Error((code), (msg));      \
  } while (0)

// Run an entry point body, converting exceptions into a status code.
template <class F>
hm_status guarded(F&& f) {
  try {
    f();
    set_last_error("");
    return HM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return HM_ENOMEM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return HM_ECUDA;
  }
}

// Stream-ordered device buffer (freed on the stream it was allocated on).
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(size_t count, cudaStream_t st) { alloc(count, st); }
  void alloc(size_t count, cudaStream_t st) {
    release();
    s = st;
    n = count;
    if (count) HM_CUDA(cudaMallocAsync((void**)&p, count * sizeof(T), st));
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  T* release_ownership() {
    T* q = p;
    p = nullptr;
    n = 0;
    return q;
  }
  ~DBuf() { release(); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
};

// Device memory owned by a graph: taken from the device's stream-ordered
// pool on the building stream, returned to it by hm_free.
void keep_pool_memory();
template <class T>
T* dalloc(size_t count, cudaStream_t s) {
  T* p = nullptr;
  if (count) HM_CUDA(cudaMallocAsync((void**)&p, count * sizeof(T), s));
  return p;
}

// Pinned host words of the calling thread (512, allocated once and kept):
// small results are read back into them, because a copy into pageable
// memory makes the host wait for the device at every copy. Slots: [0, 64)
// hm_build, [64, 72) work-space totals, [80] device wait timeouts.
uint64_t* pinned_words();

// Fork-join concurrency inside one call: up to kSide streams of this device
// (created once per device, non-blocking) start after everything already
// queued on `main`, and join() makes `main` wait for all of them. Buffers the
// side streams use must be allocated on `main` before the fork and released
// on it after the join; a Fork destroyed without join() (an error unwinds)
// still joins.
struct Fork {
  static constexpr int kSide = 3;
  cudaStream_t main;
  cudaStream_t side[kSide] = {};
  int width;  // side streams in use, 1..kSide (each costs two runtime calls per fork-join)
  bool joined = false;
  explicit Fork(cudaStream_t s, int width = kSide);
  cudaStream_t operator[](int i) const { return side[i]; }
  void join();
  ~Fork();
  Fork(const Fork&) = delete;
  Fork& operator=(const Fork&) = delete;
};

// ------------------------------------------------------------------ primitives (prims.cu)
// Exclusive scan: out[0..n] with out[n] = total. in and out may alias only if
// in == out is not required (they must not alias).
void scan_exclusive_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s);
void scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s);
// The same scan, allocating nothing: temporaries come from `scratch`, which
// must hold scan_scratch_elems(n) elements.
void scan_exclusive_u64_in(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t s,
                           uint64_t* scratch, size_t scratch_elems);
size_t scan_scratch_elems(int64_t n);
// Device-side bounded waits that gave up (see radix sort): enqueue a copy of
// the count to host memory on s; after s is synchronised, check it (throws
// HM_ETIMEOUT and clears the count when it is not zero).
void wait_timeouts_async(unsigned* h_count, cudaStream_t s);
void wait_timeouts_check(unsigned count, cudaStream_t s);
// One array for sort_batch (sort.cu): keys are the words a (and b, when
// b_is_key) -- or a with values b -- sorted stably by the listed 8-bit digit
// passes (arr 0 = a, 1 = b; shift), in place unless `unique`. With unique, the
// distinct keys go to `out` (and out_b) in the layout `unpack` names and
// their count to *d_kept (device); a and b are then left in an unspecified
// order. PAIR: key (u << member_bits) | v -> uint64 (u << 32) | v. TRIPLE /
// QUAD: 3 / 4 members of member_bits bits each, most significant first, in
// (b, a) as one 128-bit key -> int4 (pad -1).
struct SortJob {
  enum Unpack { RAW = 0, PAIR = 1, TRIPLE = 2, QUAD = 3 };
  uint64_t* a = nullptr;
  uint64_t* b = nullptr;
  int64_t n = 0;
  int passes = 0;
  int8_t arr[16] = {};
  int8_t shift[16] = {};
  int b_is_key = 0;
  int unique = 0;
  int unpack = RAW;
  int member_bits = 0;
  void* out = nullptr;
  uint64_t* out_b = nullptr;
  uint32_t* d_kept = nullptr;
};
// Sorts 1-4 independent arrays together (one temporary allocation, one
// launch per pass index for all of them).
// With `scratch` (device, sort_batch_scratch bytes, 256-byte aligned) nothing
// is allocated; `zeroed`: its first *zero_bytes bytes are already zero.
void sort_batch(const SortJob* jobs, int njobs, cudaStream_t s, unsigned char* scratch = nullptr,
                bool zeroed = false);
size_t sort_batch_scratch(const SortJob* jobs, int njobs, size_t* zero_bytes);
// Exclusive scans of 1-8 arrays in place, in one launch: a[0..n) becomes the
// prefix sums of its inputs and a[n] (which must exist) the total, also
// written to *total (device, may be NULL).
struct ScanJob {
  uint64_t* a = nullptr;
  int64_t n = 0;
  uint64_t* total = nullptr;
};
void scan_batch_inplace(const ScanJob* jobs, int njobs, cudaStream_t s,
                        unsigned char* scratch = nullptr, bool zeroed = false);
// Bytes of `scratch` a batch needs (256-byte aligned, all of it zeroed unless
// `zeroed`); 0 when every array fits one tile and no scratch is used.
size_t scan_batch_scratch(const ScanJob* jobs, int njobs);
// Stable LSD radix sort of n keys on bits [lo_bit, lo_bit + bits); vals
// (nullable) are permuted alongside. Keys equal on those bits keep their input
// order.
void radix_sort_u64(uint64_t* keys, uint64_t* vals, int64_t n, int bits, cudaStream_t s,
                    int lo_bit = 0);
// Stable LSD radix sort of 128-bit keys (hi, lo) lexicographically, on the low
// lo_bits of lo and the low hi_bits of hi.
void radix_sort_u128(uint64_t* hi, uint64_t* lo, int64_t n, int hi_bits, int lo_bits,
                     cudaStream_t s);

// ------------------------------------------------------------------ hashing
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  // SplitMix64 finaliser (Steele, Lea, Flood 2014)
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

__host__ __device__ __forceinline__ uint64_t pair_key(int32_t a, int32_t b) {
  // sorted pair packed as (min << 32) | max
  uint32_t x = (uint32_t)(a < b ? a : b), y = (uint32_t)(a < b ? b : a);
  return ((uint64_t)x << 32) | y;
}

__host__ __device__ __forceinline__ uint64_t hash_pair(uint64_t key) { return mix64(key); }

__host__ __device__ __forceinline__ uint64_t hash_tuple(int32_t a, int32_t b, int32_t c,
                                                        int32_t d) {
  uint64_t x = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
  uint64_t y = ((uint64_t)(uint32_t)c << 32) | (uint32_t)d;
  return mix64(x ^ mix64(y + 0x9E3779B97F4A7C15ull));
}

constexpr uint64_t EMPTY64 = ~0ull;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter c (in/out),
// key (k0, k1); ten rounds, the key bumped by the Weyl constants between them.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// 64-bit draw (r0 << 32) | r1 for counter (index lo, index hi, lane, tag), key = seed
__device__ __forceinline__ uint64_t philox_draw64(uint64_t seed, uint64_t index, uint32_t lane,
                                                  uint32_t tag) {
  uint32_t c[4] = {(uint32_t)index, (uint32_t)(index >> 32), lane, tag};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((uint64_t)c[0] << 32) | c[1];
}

// ------------------------------------------------------------------ graph
// Read-only view handed to kernels by value.
struct DevGraph {
  int32_t n;
  // distinct hyperedges in ascending order
  const uint64_t* e2;  // (u << 32) | v, u < v
  const int4* e3;      // (a, b, c, -1), a < b < c
  const int4* e4;      // (a, b, c, d), a < b < c < d
  int64_t m2, m3, m4;
  // open-addressing hash sets (linear probing), capacity mask + 1 (power of 2)
  const uint64_t* h2;
  uint64_t h2_mask;
  const int4* h3;
  uint64_t h3_mask;
  const int4* h4;
  uint64_t h4_mask;
  // node -> pair neighbours (sorted), node -> triples containing it (ascending index)
  const int64_t* off2;
  const int32_t* adj2;
  const int64_t* off3;
  const int32_t* inc3;
  // per pair p = (u, v): position of v in N2(u) and of u in N2(v)
  const int2* pairpos;
  // optional dense bitmaps, row u holding bwords 32-bit words: bits2 = pair
  // adjacency; bits3 / bits4 = u and v lie together in some 3- / 4-hyperedge
  // (a filter: a 3-hyperedge {a,b,c} can only exist if all its pairs are set)
  const uint32_t* bits2;
  const uint32_t* bits3;
  const uint32_t* bits4;
  // optional exact 3-hyperedge rows (one graph, small n): the row of the
  // ordered pair (a, b) starts at word (a * n + b) * bwords and has bit c set
  // iff {a, b, c} is a 3-hyperedge
  const uint32_t* tri3;
  int32_t bwords;
  // graphs without pair bitmaps: per node three 64-bit signatures (Bloom
  // words, bit sig_bit(v) for every v): [0, n) its pair neighbours, [n, 2n)
  // its co-members in 3-hyperedges, [2n, 3n) in 4-hyperedges. A clear bit
  // proves that the pair / triple / quad is absent, before any probe.
  const uint64_t* sig;
  // 0 for one graph. Otherwise the graph is a disjoint union of graphs whose
  // node ids occupy consecutive blocks of `block` ids (graph of node v =
  // v / block, computed as mulhi(v, block_inv) with block_inv = ceil(2^64 /
  // block), exact for v < 2^31); bitmap rows then span one block.
  int32_t block;
  uint64_t block_inv;
};

// Copies a class LUT (nmask bytes, a multiple of 16, from a 16-byte aligned
// device copy) into 16-byte aligned shared memory with 16-byte loads: one
// round trip to memory instead of nmask / blockDim.x dependent byte loads.
__device__ __forceinline__ void load_lut(uint8_t* lut_s, const uint8_t* lut_g, int nmask) {
  for (int i = threadIdx.x; i < nmask / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(lut_s)[i] = __ldg(reinterpret_cast<const uint4*>(lut_g) + i);
}

__device__ __forceinline__ int32_t graph_of(const DevGraph& g, int32_t v) {
  return g.block ? (int32_t)__umul64hi((uint64_t)(uint32_t)v, g.block_inv) : 0;
}
__device__ __forceinline__ int32_t graph_base(const DevGraph& g, int32_t v) {
  return g.block ? graph_of(g, v) * g.block : 0;
}

// The signature bit of node v (one of 64, by a multiplicative hash).
__device__ __forceinline__ uint64_t sig_bit(int32_t v) {
  return 1ull << (((uint64_t)(uint32_t)v * 0x9E3779B97F4A7C15ull) >> 58);
}

__device__ __forceinline__ bool has_pair(const DevGraph& g, int32_t a, int32_t b) {
  if (g.bits2) {
    const int32_t c = b - graph_base(g, a);
    uint32_t w = __ldg(g.bits2 + (size_t)a * g.bwords + (c >> 5));
    return (w >> (c & 31)) & 1u;
  }
  if (g.m2 == 0) return false;
  uint64_t key = pair_key(a, b);
  uint64_t slot = hash_pair(key) & g.h2_mask;
  for (uint64_t it = 0; it <= g.h2_mask; ++it) {
    uint64_t v = __ldg(g.h2 + slot);
    if (v == key) return true;
    if (v == EMPTY64) return false;
    slot = (slot + 1) & g.h2_mask;
  }
  return false;
}

__device__ __forceinline__ void sort3(int32_t& a, int32_t& b, int32_t& c) {
  int32_t t;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
}

__device__ __forceinline__ void sort4(int32_t& a, int32_t& b, int32_t& c, int32_t& d) {
  int32_t t;
  if (a > b) { t = a; a = b; b = t; }
  if (c > d) { t = c; c = d; d = t; }
  if (a > c) { t = a; a = c; c = t; }
  if (b > d) { t = b; b = d; d = t; }
  if (b > c) { t = b; b = c; c = t; }
}

__device__ __forceinline__ bool probe_tuple(const int4* table, uint64_t mask, int32_t a, int32_t b,
                                            int32_t c, int32_t d) {
  uint64_t slot = hash_tuple(a, b, c, d) & mask;
  for (uint64_t it = 0; it <= mask; ++it) {
    int4 v = __ldg(table + slot);
    if (v.x == a && v.y == b && v.z == c && v.w == d) return true;
    if (v.x == -1) return false;
    slot = (slot + 1) & mask;
  }
  return false;
}

// existence of the 3-hyperedge {a, b, c} (any order)
__device__ __forceinline__ bool has_triple(const DevGraph& g, int32_t a, int32_t b, int32_t c) {
  if (g.m3 == 0) return false;
  if (g.tri3) {  // exact rows: one load instead of a probe chain
    const uint32_t w = __ldg(g.tri3 + ((size_t)a * g.n + b) * g.bwords + (c >> 5));
    return (w >> (c & 31)) & 1u;
  }
  sort3(a, b, c);
  return probe_tuple(g.h3, g.h3_mask, a, b, c, -1);
}

// existence of the 4-hyperedge {a, b, c, d} (any order)
__device__ __forceinline__ bool has_quad(const DevGraph& g, int32_t a, int32_t b, int32_t c,
                                         int32_t d) {
  if (g.m4 == 0) return false;
  sort4(a, b, c, d);
  return probe_tuple(g.h4, g.h4_mask, a, b, c, d);
}

// ------------------------------------------------------------------ tracing (trace.cu)
// Whether spans named `name` are traced now: tracing is on and no filter
// (hm_trace_only) excludes the name.
bool trace_on(const char* name);
void trace_begin(cudaStream_t s, cudaEvent_t* a);
void trace_end(const char* name, cudaStream_t s, cudaEvent_t a);

// A named span of stream work (several launches) for the trace; end() records
// it, an abandoned span (an error was thrown) only releases its event.
struct TraceSpan {
  const char* name;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  TraceSpan(const char* n, cudaStream_t st) : name(n), s(st) {
    if (trace_on(name)) trace_begin(s, &a);
  }
  void end() {
    if (a) {
      cudaEvent_t e = a;
      a = nullptr;
      trace_end(name, s, e);
    }
  }
  ~TraceSpan() {
    if (a) cudaEventDestroy(a);
  }
  TraceSpan(const TraceSpan&) = delete;
  TraceSpan& operator=(const TraceSpan&) = delete;
};

// ------------------------------------------------------------------ classes (classes.cu)
struct ClassTables {
  int k;
  int ncls;
  std::vector<uint8_t> lut;       // labelled mask -> class id, 0xFF if disconnected
  std::vector<uint32_t> canon;    // class id -> canonical mask
  std::vector<int32_t> maxcard, countmax;
};
const ClassTables& class_tables(int k);
// device copy of the LUT of order k for the current device
const uint8_t* device_lut(int k);

}  // namespace hm

struct hm_graph;
namespace hm {
// build.cu
// block > 0: the input is a disjoint union of graphs of `block` node ids each
void build_graph(hm_graph* g, const int32_t* d_members, const int64_t* d_offsets, int64_t m,
                 int32_t n, int kmax, cudaStream_t s, int32_t block = 0);
void free_graph(hm_graph* g);
// census.cu
void prepare_census(hm_graph* g, int order, cudaStream_t s);
// graphlet.cu: the pairs-only 4-node sets of a graph with pair bitmaps, by
// pattern, into hist (the Q and TX launches must subtract their sets):
// prepare (zeroed scratch), then edges and pairs (independent of each other),
// then finish.
struct GraphletScratch {
  DBuf<unsigned char> buf;
  uint32_t* tnode = nullptr;
  unsigned long long* agg = nullptr;
  uint32_t* tslot = nullptr;  // graphs without pair bitmaps: triangles per pair-set slot
  int ngraphs = 1;
  int32_t per = 0;
  // graphs without pair bitmaps: per-warp lists of common neighbours (cap
  // entries each); the heavy tier's tables (2 C4.total slots), or with
  // HM_C4_SORT=1 its path keys (C4.total)
  int32_t* lists = nullptr;
  int64_t cap = 0;
  uint64_t* c4_keys = nullptr;
};
void graphlet_prepare(const hm_graph* g, GraphletScratch& G, cudaStream_t s);
// Per node of a graph without pair bitmaps, the 4-cycle paths of the heavy
// tier: its path bound when above the warp tier's, else 0; the warp tier's
// bounds go to g->c4_light. The bound in force is kept in the graph (the
// census splits the nodes by it).
void c4_bounds(hm_graph* g, uint64_t* out, cudaStream_t s);
// census.cu: the out-lists of a graph with node signatures (g->out_deg,
// g->out_adj) and, per node, C(out_deg, 2) into out.
void out_lists(hm_graph* g, uint64_t* out, cudaStream_t s);
void graphlet_edges(const hm_graph* g, GraphletScratch& G, cudaStream_t s);
void graphlet_pairs(const hm_graph* g, GraphletScratch& G, cudaStream_t s);
void graphlet_finish(const hm_graph* g, GraphletScratch& G, unsigned long long* hist,
                     cudaStream_t s);
double graphlet_cost(const hm_graph* g);
// hist holds hm_num_classes(order) counters per graph of the union (one graph: one row)
void launch_census(const hm_graph* g, int order, unsigned long long* hist, cudaStream_t s);
}  // namespace hm

// ------------------------------------------------------------------ graph object
struct hm_graph {
  int device = 0;
  int32_t n = 0;
  int kmax = 0;
  int64_t m_in = 0;
  int64_t counts[8] = {0};
  int bits = 1;  // bits per node id in packed sort keys
  // owned device arrays (cudaMalloc)
  uint64_t* e2 = nullptr;
  int4* e3 = nullptr;
  int4* e4 = nullptr;
  uint64_t* h2 = nullptr;
  uint64_t h2_mask = 0;
  int4* h3 = nullptr;
  uint64_t h3_mask = 0;
  int4* h4 = nullptr;
  uint64_t h4_mask = 0;
  int64_t* off2 = nullptr;
  int32_t* adj2 = nullptr;
  int64_t* off3 = nullptr;
  int32_t* inc3 = nullptr;
  int2* pairpos = nullptr;
  uint32_t* bits2 = nullptr;
  uint32_t* bits3 = nullptr;
  uint32_t* bits4 = nullptr;
  uint32_t* tri3 = nullptr;
  uint64_t* sig = nullptr;  // graphs without pair bitmaps: 3 n node signatures
  int32_t bwords = 0;
  int32_t block = 0;  // see DevGraph::block
  int32_t max_d2 = 0;
  // cached work spaces (prefix sums over anchors), per family
  struct Space {
    uint64_t* ws = nullptr;  // [anchors + 1]
    int64_t anchors = 0;
    uint64_t total = 0;
    bool ready = false;
  };
  Space W, S, P, TX;
  // bit-sliced variants of W, S, P (dense graphs): items are (anchor, first
  // neighbour[s]) and the last node runs over bitmap words
  Space Wb, Sb, Pb;
  // bit-sliced TX: items are (3-hyperedge, 4-word group of the rows)
  Space TXb;
  // graphs without pair bitmaps: per node, the 4-cycle paths of the heavy
  // tier (its path bound when above the warp tier's bound c4_warp_ub, else 0)
  Space C4;
  uint32_t c4_warp_ub = 0;
  // per node, its path bound when in [2, c4_warp_ub] (the warp tier's nodes), else 0
  uint16_t* c4_light = nullptr;
  // graphs with node signatures (one graph): per node v its pair neighbours
  // of higher rank (rank = (degree, id)), out_deg[v] of them, in any order at
  // out_adj[off2[v] ...]; TXO: per node C(out_deg, 2), the pairs of its
  // out-list, the index space of the sparse TX pass's wedge records
  Space TXO;
  int32_t* out_deg = nullptr;
  int32_t* out_adj = nullptr;
  // node -> 4-hyperedges containing it (indices into e4, any order); built
  // by the sampler on first use at order 4
  int64_t* off4 = nullptr;
  int32_t* inc4 = nullptr;
  bool useWb = false, useSb = false, usePb = false, useTXb = false;
  // order 4: pairs-only sets from graphlet identities instead of S and P
  bool useGL = false;
  // candidates per lane of the per-candidate families (0 = fill the GPU)
  int chunkW = 0, chunkS = 0, chunkP = 0, chunkTX = 0;
  bool tuned[5] = {false, false, false, false, false};  // by order
  std::vector<void*> owned;  // everything above, for hm_free

  hm::DevGraph view() const {
    hm::DevGraph g;
    g.n = n;
    g.e2 = e2;
    g.e3 = e3;
    g.e4 = e4;
    g.m2 = counts[2];
    g.m3 = kmax >= 3 ? counts[3] : 0;
    g.m4 = kmax >= 4 ? counts[4] : 0;
    g.h2 = h2;
    g.h2_mask = h2_mask;
    g.h3 = h3;
    g.h3_mask = h3_mask;
    g.h4 = h4;
    g.h4_mask = h4_mask;
    g.off2 = off2;
    g.adj2 = adj2;
    g.off3 = off3;
    g.inc3 = inc3;
    g.pairpos = pairpos;
    g.bits2 = bits2;
    g.bits3 = bits3;
    g.bits4 = bits4;
    g.tri3 = tri3;
    g.bwords = bwords;
    g.sig = sig;
    g.block = block;
    g.block_inv = block > 1 ? (uint64_t)((((unsigned __int128)1 << 64) + block - 1) / block) : 0;
    return g;
  }
};

namespace hm {
// Work spaces enqueued without a synchronisation (hm_build prepares those of
// its max_order this way, before its own final synchronisation).
struct PendingSpaces {
  hm_graph* g = nullptr;
  std::vector<std::pair<hm_graph::Space*, char>> need;
  std::vector<uint64_t*> made;  // allocations, owned by the graph once finished
  uint64_t* ws[8] = {};
  uint64_t* h = nullptr;  // the totals, in the calling thread's pinned words
};
std::vector<std::pair<hm_graph::Space*, char>> census_spaces(hm_graph* g, int order);
void spaces_enqueue(hm_graph* g, const std::vector<std::pair<hm_graph::Space*, char>>& todo,
                    cudaStream_t s, PendingSpaces& P);
void spaces_finish(PendingSpaces& P);
void choose_variants(hm_graph* g, int order);
}  // namespace hm
