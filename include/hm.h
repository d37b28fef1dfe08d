/*
 * hm.h -- C ABI of the GB300 higher-order motif library.
 *
 * Implements the counting step of "Exact and sampling methods for mining
 * higher-order motifs in large hypergraphs" (Lotito, Musciotto, Battiston,
 * Montresor): given a hypergraph H and an order k in {3, 4}, the frequency of
 * every higher-order motif of order k (problem statement, Sec. 3), exactly
 * (Sec. 4) or by stratified hyperedge sampling (Alg. 4, Sec. 5), plus the
 * counting of randomised null-model hypergraphs (Sec. 6.3).
 *
 * Conventions for every entry point
 *   - Pointers named d_* are CUDA device pointers; h_* are host pointers.
 *     The caller owns them; the library keeps no reference after the call's
 *     stream work completes.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is enqueued on it; entry points documented as
 *     "synchronous" also wait for it.
 *   - Node ids are int32 in [0, num_nodes). Counts are uint64.
 *   - Every entry point returns an hm_status; on failure hm_last_error()
 *     returns a message for the calling thread. No entry point aborts the
 *     process.
 *
 * Motif classes. A k-node pattern is encoded as a mask over the subsets of
 * its k positions with 2..k members, ordered by size, then lexicographically:
 *   k=3: bit 0 {0,1}, bit 1 {0,2}, bit 2 {1,2}, bit 3 {0,1,2};
 *   k=4: bits 0-5 {01,02,03,12,13,23}, bits 6-9 {012,013,023,123},
 *        bit 10 {0123}.
 * The canonical mask of a pattern is the minimum over its k! relabelings
 * (isomorphism, Def. 3). Class ids number the connected canonical masks in
 * ascending order: 6 classes for k=3, 171 for k=4.
 */
#ifndef HM_H_
#define HM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_graph hm_graph;
typedef struct hm_proposal hm_proposal;
typedef int hm_status;

enum {
  HM_OK = 0,
  HM_EINVAL = 1,       /* bad argument or input (message says which)            */
  HM_ENOMEM = 2,       /* a device or host allocation failed                      */
  HM_ECUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
  HM_ETABLEFULL = 4,   /* a hash insertion exceeded its probe bound               */
  HM_ETIMEOUT = 5,     /* a bounded device-side wait gave up                      */
  HM_EUNSUPPORTED = 6  /* valid request this graph was not built for              */
};

/* Message describing the last failure on the calling thread ("" if none). */
const char* hm_last_error(void);

/* Library version string. */
const char* hm_version(void);

/* Number of motif classes of order k (6 for k=3, 171 for k=4), -1 otherwise. */
int hm_num_classes(int order);

/*
 * Class metadata (Sec. 4.3 isomorphism classes; Alg. 4 needs maxcard and
 * countmax). For class `cls` of order `order`: its canonical mask, the size of
 * its largest hyperedge (maxcard) and how many hyperedges of that size it has
 * (countmax). Any output pointer may be NULL. HM_EINVAL on a bad order/cls.
 */
hm_status hm_class_info(int order, int cls, uint32_t* canonical_mask, int32_t* maxcard,
                        int32_t* countmax);

/*
 * Class id of a labelled mask of order k (any labelling), or -1 when the
 * pattern is not connected. HM_EINVAL on a bad order or mask.
 */
hm_status hm_class_of_mask(int order, uint32_t mask, int32_t* cls);

/*
 * Build the device representation of a hypergraph (Def. 1, Sec. 3, with the
 * hash of every hyperedge used for fill-in, Sec. 4.3).
 *   d_members  int32[d_offsets[num_hyperedges]]: members, hyperedge by hyperedge
 *   d_offsets  int64[num_hyperedges + 1]: hyperedge j is
 *              d_members[d_offsets[j] .. d_offsets[j+1]), offsets[0] == 0,
 *              non-decreasing (the host reads the last entry)
 *   num_nodes  node ids must lie in [0, num_nodes), 1 <= num_nodes < 2^31
 *   max_order  3 or 4: the largest order this graph will be counted at
 * Normalisation, not errors: repeated members collapse, hyperedges with fewer
 * than two distinct members are dropped, duplicate hyperedges collapse (E is a
 * set). Hyperedges with more than max_order distinct members cannot lie in a
 * max_order-node set (Def. 2), so they are only counted (hm_graph_info).
 * Synchronous on `stream`. Besides what the graph keeps, the build takes
 * temporaries of about 40 bytes per input hyperedge (sort keys sized for every
 * hyperedge, so that one pass normalises). Errors: HM_EINVAL (bad sizes, a
 * member outside [0, num_nodes), offsets not monotone), HM_ENOMEM, HM_ECUDA,
 * HM_EUNSUPPORTED (2^31 or more distinct pairs), HM_ETABLEFULL (a
 * hash set could not hold its keys: only when the HM_TABLE_CAP test hook
 * forces tables smaller than their key sets), HM_ETIMEOUT (a bounded wait of
 * the sort gave up). On success *out owns device memory until hm_free.
 */
hm_status hm_build(const int32_t* d_members, const int64_t* d_offsets, int64_t num_hyperedges,
                   int32_t num_nodes, int max_order, void* stream, hm_graph** out);

/*
 * Sizes of a built graph. counts (host, 8 entries):
 *   counts[0] = num_nodes, counts[1] = input hyperedges,
 *   counts[s] for s = 2..max_order = distinct hyperedges of size s (|E_s|),
 *   counts[max_order+1] = input hyperedges with more than max_order distinct
 *   members (not deduplicated), remaining entries 0.
 */
hm_status hm_graph_info(const hm_graph* g, int64_t* counts);

/*
 * Copy E_s (distinct hyperedges of size s, ascending lexicographic order of
 * their sorted members; the order the sampler indexes) to d_out, an int32
 * device buffer of s * |E_s| entries. Enqueued on `stream`.
 */
hm_status hm_graph_edges(const hm_graph* g, int s, int32_t* d_out, void* stream);

/*
 * Exact census (problem statement, Sec. 3; exact algorithms, Sec. 4.2):
 * d_hist[c] = number of `order`-node sets V' whose induced sub-hypergraph
 * H[V'] (Def. 2) is connected and of class c.
 *   d_hist  uint64[hm_num_classes(order)], device, overwritten.
 * Enqueued on `stream` (the first call per order also builds and caches
 * per-graph work spaces, which synchronises). HM_EINVAL if order is not 3 or
 * 4, HM_EUNSUPPORTED if order > the graph's max_order.
 */
hm_status hm_count_exact(hm_graph* g, int order, uint64_t* d_hist, void* stream);

/*
 * Stratified hyperedge-sampling estimator (Alg. 4, Sec. 5; budgets as in
 * Appendix A).
 *   samples_per_size  host uint64[order+1]; entry s (2..order) is S_s, the
 *                     number of draws (with replacement) from E_s. NULL: split
 *                     total_samples as S_2 = floor(S/6), S_4 = floor(S/3),
 *                     S_3 = S - S_2 - S_4 for order 4 (S_3 = 3 S_2, S_4 = 2 S_2,
 *                     Appendix A), and S_2 = floor(S/4), S_3 = S - S_2 for
 *                     order 3.
 *   seed              Philox4x32-10 key; draw t of stratum s uses counter
 *                     (t lo, t hi, s, 0x53414D50) and the 64-bit value
 *                     (r0 << 32) | r1; the index is mulhi64(value, |E_s|)
 *                     (uniform) or the inverse CDF of d_q at
 *                     mulhi64(value, Q_s) (weighted).
 *   d_q               NULL for uniform draws, else uint32 weights (each >= 1) of
 *                     E_2, E_3, ..., E_order concatenated (device); each counted
 *                     set is then weighted by floor(2^63 / q_e).
 *   d_est             double[ncls] (device): the corrected estimate of class c,
 *                     (n_c * |E_m|) / (S_m * countmax_c) uniform, or
 *                     (A_c * 2^-63 * Q_m) / (S_m * countmax_c) weighted,
 *                     with m = maxcard(c), evaluated in IEEE double in this order.
 *   d_raw             uint64[2 * ncls] (device) or NULL: (raw[2c], raw[2c+1]) =
 *                     low and high words of the integer accumulator of class c
 *                     (the plain count n_c for uniform draws).
 * Runs on `stream`, which it synchronises between stages to size them. At
 * order 4 the first call with S_2 > 0 builds the graph's node -> 4-hyperedge
 * lists (kept with the graph, 4 bytes per incidence). HM_EINVAL on a bad
 * order, or when a stratum with |E_s| > 0 gets S_s == 0 (its classes could
 * not be estimated); an empty stratum contributes an exact 0.
 * HM_EUNSUPPORTED if order > max_order.
 */
hm_status hm_count_sampled(hm_graph* g, int order, const uint64_t* samples_per_size,
                           uint64_t total_samples, uint64_t seed, const uint32_t* d_q,
                           double* d_est, uint64_t* d_raw, void* stream);

/*
 * Sizes of the index spaces hm_count_exact walks, written to host
 * totals[10] (d2 = pair degree, t3 = number of 3-hyperedges through a node):
 *   order 3: {T3 = |E_3|, W = sum_v C(d2(v), 2), Wb = sum_{v: d2>=2} d2(v),
 *             1 if the bit-sliced W variant is used}
 *   order 4: {Q = |E_4|, TX = sum_{e in E_3} sum_{x in e} (d2(x) + t3(x)),
 *             S = sum_v C(d2(v), 3), P = sum_{(u,v) in E_2} (d2(u)-1)(d2(v)-1),
 *             Sb = sum_v C(d2(v), 2), Pb = sum_{(u<v), d2(v)>1} (d2(u)-1),
 *             1 if bit-sliced S is used, 1 if bit-sliced P is used,
 *             TXb = |E_3| * (4-word groups per bitmap row), 1 if bit-sliced
 *             TX is used}
 * W, S, P, TX count candidate node sets; Wb, Sb, Pb, TXb count the items of
 * the bit-sliced variants (each item scans bitmap words of one row). The
 * bit-sliced sizes are 0 when the graph has no dense bitmaps. Synchronous.
 */
hm_status hm_work_totals(hm_graph* g, int order, uint64_t* totals, void* stream);

/*
 * End-to-end exact census from HOST buffers: copies the hyperedge list to the
 * device, builds the graph with max_order = order, counts (as hm_count_exact)
 * and copies the histogram back, all on `stream`; synchronous. Device memory
 * is taken and released inside the call.
 *   h_members, h_offsets  host arrays laid out as for hm_build
 *   h_hist                host uint64[hm_num_classes(order)], overwritten
 * Errors as hm_build and hm_count_exact.
 */
hm_status hm_count_exact_host(const int32_t* h_members, const int64_t* h_offsets,
                              int64_t num_hyperedges, int32_t num_nodes, int order,
                              uint64_t* h_hist, void* stream);

/*
 * The baseline of Sec. 4.1 (Alg. 1), for comparison with hm_count_exact
 * (Table 2): the hypergraph is projected onto a graph (two nodes joined when
 * they share a hyperedge of ANY size), every connected `order`-node subgraph
 * of the projection is enumerated once (wedges and triangles; stars, paths
 * and 4-cycles, by the canonical rules of simple graphs), filled in against
 * the hypergraph (Sec. 4.3) and counted by class when the sub-hypergraph it
 * induces is connected (Fig. 2 shows why it may not be). d_hist equals
 * hm_count_exact's; the extra work is the point of the comparison.
 *   d_members, d_offsets  as for hm_build (device)
 *   d_hist                device uint64[hm_num_classes(order)], overwritten
 *   h_info                host uint64[2] or NULL: {candidate sets generated
 *                         (sum_v C(d(v), 2) for order 3, sum_v C(d(v), 3) +
 *                         sum_{uv} (d(u) - 1)(d(v) - 1) for order 4, d the
 *                         projection degree), distinct projection pairs}
 * Builds the hypergraph and the projection inside the call, synchronous.
 * Errors as hm_build; HM_EINVAL if the projection has 2^31 pairs or more.
 */
hm_status hm_count_exact_baseline(const int32_t* d_members, const int64_t* d_offsets,
                                  int64_t num_hyperedges, int32_t num_nodes, int order,
                                  uint64_t* d_hist, uint64_t* h_info, void* stream);

/*
 * Kernel timing trace (no counterpart in the paper; instrumentation). While
 * enabled, every census kernel launch, and each phase of hm_build's ingest
 * (entries named "ingest_*", several launches each), is bracketed by CUDA
 * events recorded on its launching stream. hm_trace_read waits for the recorded events, writes
 * up to max_entries (name, milliseconds) pairs -- names as NUL-terminated
 * strings in rows of name_len bytes of `names` (may be NULL), times in `ms`
 * (may be NULL) -- sets *count, and clears the trace.
 */
hm_status hm_trace_enable(int on);
/* Restricts the trace to spans named `name` (NULL or "" = every span), so
 * that a timed run pays for the events of one kernel only. */
hm_status hm_trace_only(const char* name);
/*
 * Debug check of canonical generation (no counterpart in the paper; the
 * paper dedupes with a visited set, this library by rules that accept each
 * connected set in exactly one family and anchor). Runs the per-candidate
 * families (T3 and W at order 3; Q, TX, S and P at order 4) over the whole
 * graph, emits every connected set they accept as its sorted nodes packed
 * into one 64-bit key, radix-sorts the keys and counts repeats: h_out (host
 * uint64[2]) = {sets emitted, keys equal to their predecessor}. A correct
 * census has 0 repeats and as many sets as hm_count_exact's total. Needs
 * order * (bits per node id) <= 64 (HM_EUNSUPPORTED otherwise) and 8 bytes per
 * set of device memory. Synchronous.
 */
hm_status hm_debug_canonical_check(hm_graph* g, int order, uint64_t* h_out, void* stream);

/*
 * Self-test of the bounded device-side waits (no counterpart in the paper;
 * instrumentation). Runs the radix sort's decoupled look-back, in both its
 * thread and warp forms, against a status word that no tile ever publishes:
 * each wait gives up after its poll limit (2^20 polls, about a second), and
 * the call returns HM_ETIMEOUT through the same path as any entry point whose
 * wait gave up, with the device left usable. Returns HM_EINVAL if no wait
 * gave up. Synchronous.
 */
hm_status hm_selftest_wait(void* stream);

/*
 * Instrumentation (no counterpart in the paper): while on != 0, work that
 * the library would run concurrently on side streams (the census launches of
 * one graph, the ingest's structure chains) runs in order on the calling
 * stream instead, so that traced spans time one kernel each, as a profiler's
 * serialised launch list does. Results are the same either way. Process-wide.
 */
hm_status hm_serialize_launches(int on);

/* Number of kernels the library has launched in this process (instrumentation). */
uint64_t hm_launch_count(void);

/*
 * L2 read bandwidth of this GPU (no counterpart in the paper; instrumentation
 * for the roofline of kernels whose working set stays in L2). Allocates a
 * device buffer of `bytes` (a multiple of 16, at most 64 MiB so that it stays
 * resident in L2), fills it, reads it once untimed and then `reps` times with
 * 16-byte loads that bypass L1 (every SM's resident blocks, each block its
 * slice), and writes the bytes read per second / 1e9 to *gbs (host). The
 * time comes from CUDA events on `stream`. Synchronous; HM_EINVAL for a size
 * outside (0, 64 MiB], not a multiple of 16, or reps < 1.
 */
hm_status hm_l2_read_bandwidth(size_t bytes, int reps, double* gbs, void* stream);
hm_status hm_trace_read(int max_entries, char* names, int name_len, float* ms, int* count);

/* ---------------------------------------------------------------- learned proposal
 * An extension of Alg. 4 (Sec. 5), which samples uniformly within each
 * stratum: a small MLP maps per-hyperedge features to importance weights q
 * for hm_count_sampled (whose Hansen-Hurwitz reweighting keeps the estimate
 * unbiased for any q >= 1). Rows are E_2, E_3, ..., E_order in the order of
 * hm_graph_edges.
 */

/*
 * Per-hyperedge exact contributions: d_contrib[row * ncls + c] (device
 * uint32, overwritten) = the number of connected order-node sets of class c
 * in which hyperedge `row` is one of the hyperedges of maximum cardinality --
 * the count a draw of that hyperedge adds in Alg. 4 (max-cardinality rule,
 * Sec. 5). Summed over rows: countmax_c * hm_count_exact's count. Counters
 * wrap at 2^32. Synchronous only if the census work spaces are not yet built.
 */
hm_status hm_contributions(hm_graph* g, int order, uint32_t* d_contrib, void* stream);

/*
 * Per-hyperedge features, device float32[rows][16]: 1, |e|/4,
 * log1p(min, mean, max pair degree of the members), log1p(min, mean, max
 * number of 3-hyperedges through the members), log1p(member pairs that are
 * hyperedges), log1p(sets a draw of e enumerates at this order), log1p(sum
 * of pair degrees), log1p(sum of 3-hyperedge counts), then 4 zeros.
 */
hm_status hm_features(hm_graph* g, int order, float* d_feat, void* stream);

/*
 * The MLP 16 -> 64 -> 64 -> 1 (ReLU) on BF16 tensor cores with FP32
 * accumulation. Parameters: device float32[hm_mlp_num_params()] packed as
 * W1[16][64] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3 (W[in][out]).
 * bf16 rounding is applied to the inputs, the weights, both hidden
 * activations and the back-propagated dz2, dz1 entering matrix products.
 *   hm_mlp_forward  y[i] = f(x[i]) for n rows of 16 floats.
 *   hm_mlp_backward d_grad (overwritten) = gradient of mean_i (y_i - t_i)^2;
 *                   *d_loss_sum (may be NULL) = sum_i (y_i - t_i)^2;
 *                   d_scratch: device buffer of hm_mlp_scratch_bytes(n)
 *                   bytes, 16-byte aligned. Every sum is taken in a fixed
 *                   order, so the gradient is the same bit for bit on
 *                   every call with the same inputs.
 *   hm_mlp_adam     one Adam step (beta 0.9 / 0.999, eps 1e-8, bias
 *                   correction for `step` >= 1) on params, moments m and v.
 *   hm_mlp_train    `epochs` passes of minibatch Adam (batch rows, learning
 *                   rate lr) over the rows shuffled once with Philox(seed);
 *                   h_loss (host, may be NULL) receives each epoch's mean
 *                   loss. Synchronous.
 */
int hm_mlp_num_params(void);
size_t hm_mlp_scratch_bytes(int64_t n);
hm_status hm_mlp_forward(const float* d_params, const float* d_x, int64_t n, float* d_y,
                         void* stream);
hm_status hm_mlp_backward(const float* d_params, const float* d_x, const float* d_target,
                          int64_t n, float* d_grad, float* d_loss_sum, void* d_scratch,
                          void* stream);
hm_status hm_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int step,
                      float lr, void* stream);
hm_status hm_mlp_train(float* d_params, const float* d_x, const float* d_target, int64_t n,
                       int epochs, int64_t batch, float lr, uint64_t seed, float* h_loss,
                       void* stream);

/*
 * Training targets: d_target[row] = log(sqrt(sum_c (n_{e,c} / countmax_c /
 * T_c)^2) + eps) over classes with T_c > 0, from hm_contributions' output and
 * the exact counts d_exact_hist (uint64[ncls]); sqrt(sum ...) is the
 * per-hyperedge importance that minimises sum_c Var(T^_c) / T_c^2 for
 * with-replacement Hansen-Hurwitz sampling. Synchronous.
 */
hm_status hm_proposal_targets(hm_graph* g, int order, const uint32_t* d_contrib,
                              const uint64_t* d_exact_hist, float eps, float* d_target,
                              void* stream);

/*
 * Integer proposal for hm_count_sampled from explicit MLP parameters: within
 * stratum s, with z_e = f(x_e) - beta * log1p(cost_e), cost_e = the number of
 * sets a draw of e enumerates (feature 9), w_e = exp(z_e - max_s z),
 * p_e = (1 - lambda) w_e / sum_s w + lambda / |E_s| (0 < lambda <= 1 keeps
 * every p_e > 0), and d_q[row] = min(2^32 - 1, 1 + floor(p_e * |E_s| * 1024))
 * (device uint32). beta in [0, 1]: 0 minimises the variance per draw, 1/2
 * the variance per unit of enumeration work (draw probability proportional
 * to t_e / sqrt(cost_e)). Reductions run in a fixed order: q is
 * reproducible. Synchronous.
 */
hm_status hm_proposal_weights_params(hm_graph* g, int order, const float* d_params,
                                     float lambda, float beta, uint32_t* d_q, void* stream);

/*
 * He-uniform initial MLP parameters (device float[hm_mlp_num_params()]):
 * weight i = (2u - 1) * sqrt(6 / fan_in) with u = (v >> 11) * 2^-53 and v the
 * 64-bit Philox4x32-10 value of key = seed, counter (i, 0, 0, 0x494E4954),
 * computed in double and rounded to float; biases 0. Enqueued on `stream`.
 */
hm_status hm_mlp_init(float* d_params, uint64_t seed, void* stream);

/*
 * Train the learned proposal of Alg. 4's sampler on `train` (typically a
 * subsample of, or a graph shaped like, the hypergraph to be sampled), all
 * on the device: exact per-hyperedge contributions (hm_contributions) and
 * the exact census (hm_count_exact) give the targets (hm_proposal_targets,
 * eps = 1e-9), hm_features gives the inputs, the parameters start from
 * hm_mlp_init(seed) and train by hm_mlp_train(epochs, batch, lr, seed).
 * Bit for bit the same as that chain of calls. h_loss: host float[epochs]
 * (may be NULL), each epoch's mean loss. Synchronous. On success *out owns a
 * small device buffer until hm_proposal_free. Errors: HM_EINVAL (bad
 * arguments), HM_EUNSUPPORTED (order > the graph's max_order), HM_ENOMEM,
 * HM_ECUDA, HM_ETIMEOUT.
 */
hm_status hm_proposal_train(hm_graph* train, int order, uint64_t seed, int epochs, int64_t batch,
                            float lr, float* h_loss, void* stream, hm_proposal** out);

/* Copy a trained proposal's MLP parameters to d_params (device
 * float[hm_mlp_num_params()]); enqueued on `stream`. */
hm_status hm_proposal_params(const hm_proposal* p, float* d_params, void* stream);

/* Order a proposal was trained at (-1 for NULL). */
int hm_proposal_order(const hm_proposal* p);

/*
 * Integer proposal q for hm_count_sampled on graph g (any graph built with
 * max_order >= the proposal's order), as hm_proposal_weights_params with the
 * proposal's trained parameters and order. Synchronous.
 */
hm_status hm_proposal_weights(const hm_proposal* p, hm_graph* g, float lambda, float beta,
                              uint32_t* d_q, void* stream);

/* Release a proposal. NULL is allowed. */
void hm_proposal_free(hm_proposal* p);

/*
 * Null-model batch: the counting step repeated on randomised hypergraphs
 * (Sec. 6.3 compares observed frequencies with those of configuration-model
 * draws; the model is realised here as stub shuffling). For base b in
 * [0, num_bases) and j in [0, models_per_base), model t = b*models_per_base+j
 * is base b's stubs (its members in input order) reordered by the keys
 * (v >> 6, i), v = (r0 << 32) | r1 of Philox4x32-10 with key = seed and
 * counter (i lo, i hi, t, 0x4E554C4C), cut again into the base's hyperedge
 * sizes, normalised as by hm_build, and counted exactly at `order` as by
 * hm_count_exact.
 *   d_members, d_offsets  every base's hyperedges in one CSR (device; offsets
 *                         index d_members globally)
 *   h_base_edges          host int64[num_bases + 1]: base b owns hyperedges
 *                         [h_base_edges[b], h_base_edges[b+1])
 *   h_num_nodes           host int32[num_nodes]: base b's ids lie in [0, n_b)
 *   d_hists               device uint64[num_bases * models_per_base *
 *                         hm_num_classes(order)]; row t = model t
 * Up to 64 models are counted together as one disjoint union (model t's node
 * v becomes t * max(n_b) + v): one ingest and one persistent launch per
 * candidate family for the whole group, whatever the models' sizes.
 * Synchronous. Errors: HM_EINVAL (bad ranges, max(n_b) * 64 >= 2^31, a member
 * outside its base's [0, n_b)), HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_count_null_batch(int num_bases, const int32_t* d_members, const int64_t* d_offsets,
                              const int64_t* h_base_edges, const int32_t* h_num_nodes, int order,
                              int models_per_base, uint64_t seed, uint64_t* d_hists,
                              void* stream);

/* ---------------------------------------------------------------- order 5
 * Alg. 4 at order 5 (Sec. 6.4). A 5-node pattern is a 26-bit mask over the
 * subsets of its five sorted positions with 2..5 members, by size and then
 * lexicographically: bits 0-9 {01,02,03,04,12,13,14,23,24,34}, bits 10-19
 * the triples {012,...,234}, bits 20-24 the quads {0123,...,1234}, bit 25
 * {01234}. A class is its canonical mask: the minimum over the 120
 * relabelings (Def. 3); there is no class table.
 *
 * Draw t of stratum s (s = 2..5) is hyperedge mulhi64(v, |E_s|) of E_s
 * (distinct hyperedges with s distinct members, ascending), v the 64-bit
 * Philox4x32-10 value of key = seed, counter (t lo, t hi, s, 0x53414D50). The
 * sets counted for it are the 5-node V' containing it whose H[V'] is
 * connected and whose largest hyperedges have s members; n_c counts them
 * over all draws, and the estimate of class c is
 * (n_c * |E_m|) / (S_m * countmax_c) in IEEE double in this order, m and
 * countmax_c the size and number of c's largest hyperedges.
 *   samples_per_size  host uint64[6], entry s = S_s (s = 2..5); NULL: split
 *                     total_samples as S_2 = floor(S/8), S_3 = floor(3S/8),
 *                     S_4 = floor(S/4), S_5 = S - S_2 - S_3 - S_4
 *   d_masks, d_raw, d_est  device uint32 / uint64 / double[capacity]: the
 *                     classes met, ascending by canonical mask (the first
 *                     `capacity` of them), with n_c and the estimate
 *   *h_num_classes    the number of classes met (may exceed capacity)
 * Builds its structures from the hyperedge list inside the call (uniform
 * draws only), uses a 512 MiB histogram, synchronous. Errors: HM_EINVAL (bad
 * sizes, a stratum with |E_s| > 0 and S_s == 0), HM_EUNSUPPORTED (node ids of
 * 2^25 or more), HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_count_sampled5(const int32_t* d_members, const int64_t* d_offsets,
                            int64_t num_hyperedges, int32_t num_nodes,
                            const uint64_t* samples_per_size, uint64_t total_samples,
                            uint64_t seed, uint32_t* d_masks, uint64_t* d_raw, double* d_est,
                            int64_t capacity, int64_t* h_num_classes, void* stream);

/* ---------------------------------------------------------------- motif profiles
 * Sec. 6.3 judges estimated counts by the motif profiles they give against a
 * configuration-model null, next to the profiles of the exact counts (rho,
 * MaxAE and MAE, Table 3). The profile is the one of the prior work the
 * paper cites: for class c, with N_c the observed count and <N_c> its mean
 * over the null models,
 *   D_c  = (N_c - <N_c>) / (N_c + <N_c> + eps)      (eps = 4 there),
 *   SP_c = D_c / sqrt(sum_k D_k^2)                  (zeros when D = 0).
 * All arithmetic is IEEE double with sums in a fixed order (reproducible).
 */

/*
 * Significance profile of one hypergraph.
 *   d_observed   device double[num_classes]: observed counts (exact counts
 *                through hm_counts_to_double, or hm_count_sampled estimates)
 *   d_null_rows  device uint64[num_models * num_classes]: the null models'
 *                exact counts, row t = model t (hm_count_null_batch layout)
 *   d_profile    device double[num_classes]: SP, overwritten
 *   d_abundance  device double[num_classes] or NULL: D, overwritten
 * Enqueued on `stream`. HM_EINVAL on sizes < 1, NULL buffers or eps < 0.
 */
hm_status hm_significance_profile(int num_classes, const double* d_observed,
                                  const uint64_t* d_null_rows, int num_models, double eps,
                                  double* d_profile, double* d_abundance, void* stream);

/*
 * Agreement of an estimated profile p with the exact one q (Table 3):
 * d_out (device double[3]) = {Pearson's rho of p and q (0 when either is
 * constant), max_c |p_c - q_c| (MaxAE), mean_c |p_c - q_c| (MAE)}. Enqueued
 * on `stream`.
 */
hm_status hm_profile_compare(int num_classes, const double* d_estimated, const double* d_exact,
                             double* d_out, void* stream);

/* d_out[i] = (double)d_counts[i] for i < n (exact below 2^53); enqueued. */
hm_status hm_counts_to_double(const uint64_t* d_counts, int64_t n, double* d_out, void* stream);

/* ---------------------------------------------------------------- configuration model
 * The null model Sec. 6.3 samples is Chodrow's configuration model of
 * hypergraphs. It is sampled here by its pairwise-reshuffle Markov chain: two
 * hyperedges e, f keep their intersection and deal the rest of their
 * members out again at random, |e| - |e n f| to e and the remainder to f.
 * Degrees and sizes are kept, no hyperedge gets a repeated member, and the
 * move is symmetric, so the stationary distribution is uniform over the
 * hyperedge-labelled hypergraphs with those degrees and sizes (duplicate
 * hyperedges allowed; the census collapses them, as for any input).
 * Round r of `sweeps` pairs the hyperedges of a model by a random matching:
 * hyperedge i gets the key v >> 6, v the 64-bit Philox4x32-10 value of key =
 * seed and counter ((r << 32) | i, model << 8, 0x4D434D43), the hyperedges
 * are sorted by (key, i) and positions 2k, 2k + 1 form pair k (an odd one
 * out stays). In pair k, S = e's members outside f (in order), then f's
 * outside e; step q of a partial Fisher-Yates shuffle (q < |e \ f| and
 * q < |S| - 1) swaps S[q] with S[q + mulhi64(v_q, |S| - q)], v_q the value of
 * counter ((r << 32) | k, (model << 8) | (q + 1), 0x4D434D43), and S returns
 * to the same slots in order (e's first). Pairs with |S| > 255, |S| < 2 or S
 * within one of them stay as they are. Every pair of a round moves at once
 * (disjoint moves commute). Hyperedges must not repeat a member (HM_EINVAL).
 */

/*
 * One configuration-model draw: d_out (device int32[d_offsets[m]]) gets the
 * members of model `model` (< 2^24) after `sweeps` rounds started from the
 * input (offsets unchanged). Synchronous. Errors: HM_EINVAL (bad sizes, a
 * member outside [0, num_nodes), a repeated member), HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_configuration_model(const int32_t* d_members, const int64_t* d_offsets,
                                 int64_t num_hyperedges, int32_t num_nodes, uint32_t model,
                                 int sweeps, uint64_t seed, int32_t* d_out, void* stream);

/*
 * hm_count_null_batch with configuration-model draws instead of stub
 * shuffles: model t = b * models_per_base + j starts from base b and takes
 * `sweeps` rounds of pairwise reshuffles (as hm_configuration_model with
 * model = t), then is counted at `order` as by hm_count_exact. The models of
 * a 64-model group are reshuffled together, each round one sort and one
 * launch for the group. Same layout and errors as hm_count_null_batch, plus
 * HM_EINVAL for a repeated member or 2^24 models or more.
 */
hm_status hm_count_null_batch_mcmc(int num_bases, const int32_t* d_members,
                                   const int64_t* d_offsets, const int64_t* h_base_edges,
                                   const int32_t* h_num_nodes, int order, int models_per_base,
                                   int sweeps, uint64_t seed, uint64_t* d_hists, void* stream);

/*
 * hm_count_sampled without any device allocation (the paper has no
 * counterpart). It serves callers that cannot allocate device memory while
 * they count: applications that reserve the GPU's memory up front (a serving
 * process with a fixed budget, or one where another framework's caching
 * allocator holds the rest), and latency-critical loops where
 * cudaMalloc/cudaFree may block or synchronise the device. Same arguments,
 * results and errors as hm_count_sampled, bit for bit.
 *   - Every temporary lives in one static device array of 32 MiB inside
 *     libhm.so, which each GPU that loads the library holds until the
 *     process exits. Requests whose temporaries cannot fit are rejected with
 *     HM_EINVAL and a message naming the limit: with weights d_q, each
 *     stratum needs about 16 * |E_s| bytes; at order 4 one draw of a pair
 *     needs about 64 * (max pair degree) bytes. Larger sample counts are
 *     taken in several batches.
 *   - The first call on a device (with that device current) resolves the
 *     array's device address and copies the class tables; make that first
 *     call before any stream capture.
 *   - All calls on a device share the array: calls that overlap on the GPU
 *     (other streams, other host threads) race and must be serialised by the
 *     caller.
 *   - The call synchronises `stream` and reads sizes back to the host
 *     between sample batches, so it is made from ordinary host code; it
 *     cannot be called from a stream callback (host function), where CUDA
 *     calls are not allowed.
 *   - The graph must have been built by hm_build (which allocates).
 */
hm_status hm_count_sampled_noalloc(hm_graph* g, int order, const uint64_t* samples_per_size,
                                   uint64_t total_samples, uint64_t seed, const uint32_t* d_q,
                                   double* d_est, uint64_t* d_raw, void* stream);

/* Release a graph and its device memory. NULL is allowed. */
void hm_free(hm_graph* g);

#ifdef __cplusplus
}
#endif

#endif /* HM_H_ */
