// Learned importance proposal for the sampler (an extension of Alg. 4,
// Sec. 5: the paper samples uniformly within each stratum).
//
// Target. With with-replacement draws from probabilities p_e and the
// Hansen-Hurwitz reweighting the sampler applies, the proposal minimising
// sum_c Var(T^_c) / T_c^2 draws e with probability proportional to
// t_e = sqrt(sum_c (y_{e,c} / T_c)^2), y_{e,c} = n_{e,c} / countmax_c (the
// per-hyperedge contributions of contrib.cu, T_c the exact counts). The MLP
// regresses log(t_e + eps) on the hyperedge's features.
//
// Proposal. Within stratum s, with z_e = f(x_e) - beta log1p(cost_e) (cost_e =
// the number of sets a draw of e enumerates; beta = 1/2 makes the draw
// probability proportional to t_e / sqrt(cost_e), the optimum when the
// budget is GPU time rather than draws): w_e = exp(z_e - max_s z),
// p_e = (1 - lambda) w_e / sum_s w + lambda / |E_s| (a defensive mixture, so
// p_e > 0 everywhere and the estimator stays unbiased), and the integer
// weight the sampler consumes is q_e = min(2^32 - 1, 1 + floor(p_e |E_s| 2^10)).
// Reductions run in a fixed order, so q is reproducible bit for bit.
#include <cmath>
#include <vector>

#include "hm_internal.cuh"

namespace hm {

void features(const hm_graph* g, int order, float* d_feat, cudaStream_t s);
void contributions(hm_graph* g, int order, uint32_t* d_contrib, cudaStream_t s);
void prepare_census(hm_graph* g, int order, cudaStream_t s);
void launch_census(const hm_graph* g, int order, unsigned long long* hist, cudaStream_t s);
void mlp_forward(const float* params, const float* X, int64_t n, float* y, cudaStream_t s);
void mlp_backward(const float* params, const float* X, const float* target, int64_t n,
                  float* grad, float* loss_sum, void* scratch, cudaStream_t s);
void mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
              cudaStream_t s);
int mlp_num_params();
size_t mlp_scratch_bytes(int64_t n);

namespace {

constexpr int RED_BLOCKS = 256;

unsigned grid_n(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

__global__ void k_targets(const uint32_t* __restrict__ contrib, int64_t rows, int ncls,
                          const unsigned long long* __restrict__ exact,
                          const int8_t* __restrict__ countmax, float eps, float* __restrict__ out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < ncls; ++c) {
      const uint32_t v = contrib[r * ncls + c];
      if (v == 0 || exact[c] == 0) continue;
      const double y = (double)v / (double)countmax[c] / (double)exact[c];
      acc += y * y;
    }
    out[r] = (float)log(sqrt(acc) + (double)eps);
  }
}

// per-block maxima / sums of one stratum, combined by one thread in block order
__global__ void k_block_max(const float* __restrict__ y, int64_t n, float* __restrict__ part) {
  __shared__ float sm[256];
  float m = -3.4e38f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, y[i]);
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmaxf(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_block_expsum(const float* __restrict__ y, int64_t n,
                               const float* __restrict__ mx, double* __restrict__ part) {
  __shared__ double sm[256];
  double a = 0.0;
  const float m = *mx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a += (double)expf(y[i] - m);
  sm[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_combine_max(const float* __restrict__ part, int nb, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float m = -3.4e38f;
    for (int i = 0; i < nb; ++i) m = fmaxf(m, part[i]);
    *out = m;
  }
}

__global__ void k_combine_sum(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < nb; ++i) a += part[i];
    *out = a;
  }
}

// z_e = f(x_e) - beta * log1p(work_e): feature 9 is log1p of the number of
// sets a draw of e enumerates, the cost of the draw
__global__ void k_cost_adjust(float* __restrict__ y, const float* __restrict__ feat, int64_t n,
                              float beta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] -= beta * feat[i * 16 + 9];
}

__global__ void k_quantise(const float* __restrict__ y, int64_t n, const float* __restrict__ mx,
                           const double* __restrict__ sum, float lambda,
                           uint32_t* __restrict__ q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double w = (double)expf(y[i] - *mx);
    const double p = (1.0 - (double)lambda) * w / *sum + (double)lambda / (double)n;
    const double v = 1.0 + floor(p * (double)n * 1024.0);
    q[i] = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
  }
}

__global__ void k_shuffle_keys(int64_t n, uint64_t seed, uint64_t* __restrict__ keys,
                               uint64_t* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = philox_draw64(seed, (uint64_t)i, 0u, 0x4D4C5031u);  // "MLP1"
    idx[i] = (uint64_t)i;
  }
}

__global__ void k_gather_rows(const float* __restrict__ X, const float* __restrict__ t,
                              const uint64_t* __restrict__ idx, int64_t n,
                              float* __restrict__ Xo, float* __restrict__ to) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = (int64_t)idx[i];
    const float4* src = reinterpret_cast<const float4*>(X + j * 16);
    float4* dst = reinterpret_cast<float4*>(Xo + i * 16);
    dst[0] = src[0];
    dst[1] = src[1];
    dst[2] = src[2];
    dst[3] = src[3];
    to[i] = t[j];
  }
}

// He-uniform initial weights from Philox4x32-10 (key = seed, counter =
// (parameter index, 0, 0, "INIT")): u = (value >> 11) 2^-53 in [0, 1), and
// weight = (2u - 1) sqrt(6 / fan_in) in double, rounded once to float; the
// biases start at 0. Layout as in mlp.cu: W1[16][64] | b1[64] | W2[64][64] |
// b2[64] | w3[64] | b3.
__global__ void k_mlp_init(float* __restrict__ p, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 5313) return;
  double fan = 0.0;
  if (i < 1024) fan = 16.0;
  else if (i >= 1088 && i < 5184) fan = 64.0;
  else if (i >= 5248 && i < 5312) fan = 64.0;
  if (fan == 0.0) {
    p[i] = 0.f;
    return;
  }
  const uint64_t v = philox_draw64(seed, (uint64_t)i, 0u, 0x494E4954u);  // "INIT"
  const double u = (double)(v >> 11) * 0x1.0p-53;
  p[i] = (float)((2.0 * u - 1.0) * sqrt(6.0 / fan));
}

}  // namespace

void mlp_init(float* params, uint64_t seed, cudaStream_t s) {
  HM_CHECK(mlp_num_params() == 5313, HM_EINVAL, "parameter layout changed");
  k_mlp_init<<<(5313 + 255) / 256, 256, 0, s>>>(params, seed);
  HM_KCHECK();
}

void proposal_targets(const hm_graph* g, int order, const uint32_t* contrib,
                      const uint64_t* exact_hist, float eps, float* out, cudaStream_t s) {
  int64_t rows = 0;
  for (int k = 2; k <= order; ++k) rows += g->counts[k];
  if (rows == 0) return;
  const ClassTables& T = class_tables(order);
  DBuf<int8_t> cm(T.ncls, s);
  std::vector<int8_t> h(T.ncls);
  for (int c = 0; c < T.ncls; ++c) h[c] = (int8_t)T.countmax[c];
  HM_CUDA(cudaMemcpyAsync(cm.p, h.data(), T.ncls, cudaMemcpyHostToDevice, s));
  k_targets<<<grid_n(rows), 256, 0, s>>>(contrib, rows, T.ncls,
                                         (const unsigned long long*)exact_hist, cm.p, eps, out);
  HM_KCHECK();
  HM_CUDA(cudaStreamSynchronize(s));
}

void proposal_weights(const hm_graph* g, int order, const float* params, float lambda,
                      float beta, uint32_t* q, cudaStream_t s) {
  int64_t rows = 0;
  for (int k = 2; k <= order; ++k) rows += g->counts[k];
  if (rows == 0) return;
  DBuf<float> feat(rows * 16, s), y(rows, s), part(RED_BLOCKS, s), mx(1, s);
  DBuf<double> dpart(RED_BLOCKS, s), sum(1, s);
  features(g, order, feat.p, s);
  mlp_forward(params, feat.p, rows, y.p, s);
  if (beta != 0.f) {
    k_cost_adjust<<<grid_n(rows), 256, 0, s>>>(y.p, feat.p, rows, beta);
    HM_KCHECK();
  }
  int64_t off = 0;
  for (int k = 2; k <= order; ++k) {
    const int64_t n = g->counts[k];
    if (n > 0) {
      k_block_max<<<RED_BLOCKS, 256, 0, s>>>(y.p + off, n, part.p);
      HM_KCHECK();
      k_combine_max<<<1, 32, 0, s>>>(part.p, RED_BLOCKS, mx.p);
      HM_KCHECK();
      k_block_expsum<<<RED_BLOCKS, 256, 0, s>>>(y.p + off, n, mx.p, dpart.p);
      HM_KCHECK();
      k_combine_sum<<<1, 32, 0, s>>>(dpart.p, RED_BLOCKS, sum.p);
      HM_KCHECK();
      k_quantise<<<grid_n(n), 256, 0, s>>>(y.p + off, n, mx.p, sum.p, lambda, q + off);
      HM_KCHECK();
    }
    off += n;
  }
  HM_CUDA(cudaStreamSynchronize(s));
}

void mlp_train(float* params, const float* X, const float* target, int64_t n, int epochs,
               int64_t batch, float lr, uint64_t seed, float* h_loss, cudaStream_t s) {
  const int np = mlp_num_params();
  DBuf<float> m(np, s), v(np, s), grad(np, s), loss(1, s);
  HM_CUDA(cudaMemsetAsync(m.p, 0, np * sizeof(float), s));
  HM_CUDA(cudaMemsetAsync(v.p, 0, np * sizeof(float), s));
  if (n == 0) return;
  if (batch <= 0 || batch > n) batch = n;
  DBuf<unsigned char> scratch(mlp_scratch_bytes(batch), s);
  DBuf<float> Xs(n * 16, s), ts(n, s);
  {
    DBuf<uint64_t> keys(n, s), idx(n, s);
    k_shuffle_keys<<<grid_n(n), 256, 0, s>>>(n, seed, keys.p, idx.p);
    HM_KCHECK();
    radix_sort_u64(keys.p, idx.p, n, 64, s);
    k_gather_rows<<<grid_n(n), 256, 0, s>>>(X, target, idx.p, n, Xs.p, ts.p);
    HM_KCHECK();
  }
  int step = 0;
  for (int e = 0; e < epochs; ++e) {
    double eloss = 0.0;
    for (int64_t b0 = 0; b0 < n; b0 += batch) {
      const int64_t nb = std::min<int64_t>(batch, n - b0);
      mlp_backward(params, Xs.p + b0 * 16, ts.p + b0, nb, grad.p, loss.p, scratch.p, s);
      mlp_adam(params, grad.p, m.p, v.p, ++step, lr, s);
      if (h_loss) {
        float l = 0.f;
        HM_CUDA(cudaMemcpyAsync(&l, loss.p, sizeof l, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        eloss += l;
      }
    }
    if (h_loss) h_loss[e] = (float)(eloss / (double)n);
  }
  unsigned timeouts = 0;
  wait_timeouts_async(&timeouts, s);
  HM_CUDA(cudaStreamSynchronize(s));
  wait_timeouts_check(timeouts, s);
}

}  // namespace hm

// A trained proposal: the MLP parameters and the order it was trained at.
struct hm_proposal {
  int device = 0;
  int order = 4;
  float* params = nullptr;  // device float[5313]
};

namespace hm {

// Alg. 4's proposal trained inside the library: exact per-hyperedge
// contributions and the exact census of the training graph give the targets,
// the features are the inputs, the weights start from mlp_init(seed) and train
// with mlp_train(seed).
void proposal_train(hm_graph* g, int order, uint64_t seed, int epochs, int64_t batch, float lr,
                    float* h_loss, cudaStream_t s, hm_proposal* p) {
  int64_t rows = 0;
  for (int k = 2; k <= order; ++k) rows += g->counts[k];
  const ClassTables& T = class_tables(order);
  mlp_init(p->params, seed, s);
  if (rows == 0) {
    for (int e = 0; h_loss && e < epochs; ++e) h_loss[e] = 0.f;
    HM_CUDA(cudaStreamSynchronize(s));
    return;
  }
  DBuf<float> feat(rows * 16, s), tgt(rows, s);
  {
    DBuf<uint32_t> contrib((size_t)rows * T.ncls, s);
    DBuf<unsigned long long> exact(T.ncls, s);
    contributions(g, order, contrib.p, s);
    prepare_census(g, order, s);
    HM_CUDA(cudaMemsetAsync(exact.p, 0, sizeof(unsigned long long) * T.ncls, s));
    launch_census(g, order, exact.p, s);
    proposal_targets(g, order, contrib.p, (const uint64_t*)exact.p, 1e-9f, tgt.p, s);
  }
  features(g, order, feat.p, s);
  mlp_train(p->params, feat.p, tgt.p, rows, epochs, batch, lr, seed, h_loss, s);
}

}  // namespace hm

extern "C" {

hm_status hm_mlp_init(float* d_params, uint64_t seed, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(d_params != nullptr, HM_EINVAL, "NULL parameters");
    hm::mlp_init(d_params, seed, (cudaStream_t)stream);
  });
}

hm_status hm_proposal_train(hm_graph* train, int order, uint64_t seed, int epochs, int64_t batch,
                            float lr, float* h_loss, void* stream, hm_proposal** out) {
  hm_proposal* p = nullptr;
  hm_status st = hm::guarded([&] {
    HM_CHECK(train != nullptr && out != nullptr, HM_EINVAL, "NULL argument");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= train->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    HM_CHECK(epochs >= 1 && batch >= 1, HM_EINVAL, "epochs and batch must be >= 1");
    HM_CHECK(lr > 0.f, HM_EINVAL, "learning rate must be > 0");
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CHECK(dev == train->device, HM_EINVAL, "graph was built on another device");
    cudaStream_t s = (cudaStream_t)stream;
    p = new hm_proposal();
    p->device = dev;
    p->order = order;
    HM_CUDA(cudaMalloc((void**)&p->params, sizeof(float) * hm::mlp_num_params()));
    hm::proposal_train(train, order, seed, epochs, batch, lr, h_loss, s, p);
  });
  if (st != HM_OK) {
    if (p) {
      if (p->params) cudaFree(p->params);
      delete p;
    }
    return st;
  }
  *out = p;
  return HM_OK;
}

hm_status hm_proposal_params(const hm_proposal* p, float* d_params, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(p && d_params, HM_EINVAL, "NULL argument");
    HM_CUDA(cudaMemcpyAsync(d_params, p->params, sizeof(float) * hm::mlp_num_params(),
                            cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  });
}

int hm_proposal_order(const hm_proposal* p) { return p ? p->order : -1; }

hm_status hm_proposal_weights(const hm_proposal* p, hm_graph* g, float lambda, float beta,
                              uint32_t* d_q, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(p && g && d_q, HM_EINVAL, "NULL argument");
    HM_CHECK(p->order <= g->kmax, HM_EUNSUPPORTED, "proposal order exceeds the graph's max_order");
    HM_CHECK(lambda > 0.f && lambda <= 1.f, HM_EINVAL, "lambda must be in (0, 1]");
    HM_CHECK(beta >= 0.f && beta <= 1.f, HM_EINVAL, "beta must be in [0, 1]");
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CHECK(dev == g->device && dev == p->device, HM_EINVAL,
             "graph or proposal lives on another device");
    hm::proposal_weights(g, p->order, p->params, lambda, beta, d_q, (cudaStream_t)stream);
  });
}

void hm_proposal_free(hm_proposal* p) {
  if (!p) return;
  if (p->params) cudaFree(p->params);
  delete p;
}

hm_status hm_proposal_targets(hm_graph* g, int order, const uint32_t* d_contrib,
                              const uint64_t* d_exact_hist, float eps, float* d_target,
                              void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g && d_contrib && d_exact_hist && d_target, HM_EINVAL, "NULL argument");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= g->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    HM_CHECK(eps > 0.f, HM_EINVAL, "eps must be > 0");
    hm::proposal_targets(g, order, d_contrib, d_exact_hist, eps, d_target, (cudaStream_t)stream);
  });
}

hm_status hm_proposal_weights_params(hm_graph* g, int order, const float* d_params,
                                     float lambda, float beta, uint32_t* d_q, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(g && d_params && d_q, HM_EINVAL, "NULL argument");
    HM_CHECK(order == 3 || order == 4, HM_EINVAL, "order must be 3 or 4");
    HM_CHECK(order <= g->kmax, HM_EUNSUPPORTED, "order exceeds the graph's max_order");
    HM_CHECK(lambda > 0.f && lambda <= 1.f, HM_EINVAL, "lambda must be in (0, 1]");
    HM_CHECK(beta >= 0.f && beta <= 1.f, HM_EINVAL, "beta must be in [0, 1]");
    hm::proposal_weights(g, order, d_params, lambda, beta, d_q, (cudaStream_t)stream);
  });
}

hm_status hm_mlp_train(float* d_params, const float* d_x, const float* d_target, int64_t n,
                       int epochs, int64_t batch, float lr, uint64_t seed, float* h_loss,
                       void* stream) {
  return hm::guarded([&] {
    HM_CHECK(d_params && n >= 0 && epochs >= 0, HM_EINVAL, "bad arguments");
    HM_CHECK(n == 0 || (d_x && d_target), HM_EINVAL, "NULL data");
    hm::mlp_train(d_params, d_x, d_target, n, epochs, batch, lr, seed, h_loss,
                  (cudaStream_t)stream);
  });
}

}  // extern "C"
