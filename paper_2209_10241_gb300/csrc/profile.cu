// Motif significance profiles and their comparison (Sec. 6.3, Table 3).
//
// The paper judges sampled counts by the motif profiles they give against a
// configuration-model null, next to the profiles of the exact counts, with
// Pearson's rho, the maximum and the mean absolute error. The profile is the
// one of the cited prior work on higher-order motifs:
//   D_c  = (N_c - <N_c>) / (N_c + <N_c> + eps)   (eps = 4 there),
//   SP_c = D_c / sqrt(sum_k D_k^2)               (all zeros when D = 0),
// N_c the observed count (exact or estimated), <N_c> the mean over the null
// models. Everything runs in IEEE double in one block, with every sum taken
// in a fixed order (a thread per class sums the models in order; class sums
// go through a fixed shared-memory tree), so results are reproducible.
#include <algorithm>
#include <cmath>

#include "hm_internal.cuh"

namespace hm {
namespace {

constexpr int PROF_THREADS = 256;

// Fixed-order block sum of one double per thread (every thread gets it).
__device__ double block_sum(double v, double* sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int o = PROF_THREADS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sm[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(PROF_THREADS)
    k_profile(const double* __restrict__ obs, const uint64_t* __restrict__ rows, int M, int C,
              double eps, double* __restrict__ prof, double* __restrict__ abund) {
  __shared__ double sm[PROF_THREADS];
  double sq = 0.0;
  for (int c = threadIdx.x; c < C; c += PROF_THREADS) {
    double s = 0.0;
    for (int t = 0; t < M; ++t) s += (double)rows[(int64_t)t * C + c];
    const double mean = s / (double)M;
    const double d = (obs[c] - mean) / (obs[c] + mean + eps);
    prof[c] = d;
    if (abund) abund[c] = d;
    sq += d * d;
  }
  const double norm = sqrt(block_sum(sq, sm));
  for (int c = threadIdx.x; c < C; c += PROF_THREADS) prof[c] = norm > 0.0 ? prof[c] / norm : 0.0;
}

__global__ void __launch_bounds__(PROF_THREADS)
    k_compare(const double* __restrict__ p, const double* __restrict__ q, int C,
              double* __restrict__ out) {
  __shared__ double sm[PROF_THREADS];
  double sp = 0.0, sq = 0.0, mx = 0.0, sa = 0.0;
  for (int c = threadIdx.x; c < C; c += PROF_THREADS) {
    sp += p[c];
    sq += q[c];
    const double e = fabs(p[c] - q[c]);
    sa += e;
    mx = fmax(mx, e);
  }
  const double mp = block_sum(sp, sm) / (double)C;
  const double mq = block_sum(sq, sm) / (double)C;
  const double mae = block_sum(sa, sm) / (double)C;
  // maximum through the same tree
  sm[threadIdx.x] = mx;
  __syncthreads();
  for (int o = PROF_THREADS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  const double maxae = sm[0];
  __syncthreads();
  double xy = 0.0, xx = 0.0, yy = 0.0;
  for (int c = threadIdx.x; c < C; c += PROF_THREADS) {
    const double dp = p[c] - mp, dq = q[c] - mq;
    xy += dp * dq;
    xx += dp * dp;
    yy += dq * dq;
  }
  const double sxy = block_sum(xy, sm), sxx = block_sum(xx, sm), syy = block_sum(yy, sm);
  if (threadIdx.x == 0) {
    const double den = sqrt(sxx * syy);
    out[0] = den > 0.0 ? sxy / den : 0.0;
    out[1] = maxae;
    out[2] = mae;
  }
}

__global__ void k_u64_to_f64(const uint64_t* __restrict__ in, int64_t n, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

}  // namespace
}  // namespace hm

extern "C" {

hm_status hm_significance_profile(int num_classes, const double* d_observed,
                                  const uint64_t* d_null_rows, int num_models, double eps,
                                  double* d_profile, double* d_abundance, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(num_classes >= 1 && num_models >= 1, HM_EINVAL,
             "num_classes and num_models must be >= 1");
    HM_CHECK(d_observed && d_null_rows && d_profile, HM_EINVAL, "NULL argument");
    HM_CHECK(eps >= 0.0, HM_EINVAL, "eps must be >= 0");
    hm::k_profile<<<1, hm::PROF_THREADS, 0, (cudaStream_t)stream>>>(
        d_observed, d_null_rows, num_models, num_classes, eps, d_profile, d_abundance);
    HM_KCHECK();
  });
}

hm_status hm_profile_compare(int num_classes, const double* d_estimated, const double* d_exact,
                             double* d_out, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(num_classes >= 1, HM_EINVAL, "num_classes must be >= 1");
    HM_CHECK(d_estimated && d_exact && d_out, HM_EINVAL, "NULL argument");
    hm::k_compare<<<1, hm::PROF_THREADS, 0, (cudaStream_t)stream>>>(d_estimated, d_exact,
                                                                    num_classes, d_out);
    HM_KCHECK();
  });
}

hm_status hm_counts_to_double(const uint64_t* d_counts, int64_t n, double* d_out, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(n >= 0, HM_EINVAL, "n must be >= 0");
    if (n == 0) return;
    HM_CHECK(d_counts && d_out, HM_EINVAL, "NULL argument");
    const int64_t b = std::min<int64_t>((n + 255) / 256, 152 * 8);
    hm::k_u64_to_f64<<<(unsigned)b, 256, 0, (cudaStream_t)stream>>>(d_counts, n, d_out);
    HM_KCHECK();
  });
}

}  // extern "C"
