// Learned sampling proposal: a small MLP (16 -> 64 -> 64 -> 1, ReLU) mapping
// per-hyperedge features to a log-importance weight. BF16 operands on the
// tensor cores (mma.sync m16n8k16), FP32 accumulation, hand-written forward,
// backward and Adam kernels. The model is tiny (5,313 parameters); its cost
// is reading the features, so the forward keeps every activation in
// registers (the accumulator fragment of one layer is the operand fragment of
// the next) and the weight gradients are split-K GEMMs over the rows.
//
// Parameters (float32, packed): W1[16][64] | b1[64] | W2[64][64] | b2[64] |
// w3[64] | b3, W[in][out]. Rounding points (the CPU reference follows them):
// x, W1, W2, w3 -> bf16; z1 = x W1 + b1 (fp32), h1 = bf16(relu(z1));
// z2 = h1 W2 + b2, h2 = bf16(relu(z2)); y = h2 . w3 + b3 (fp32).
// Backward of L = mean (y - t)^2: dy = 2 (y - t) / N; db3 = sum dy;
// dw3 = sum dy h2; dz2 = dy w3 [z2 > 0]; db2 = sum dz2;
// dW2 = h1^T bf16(dz2); dh1 = bf16(dz2) W2^T; dz1 = dh1 [z1 > 0];
// db1 = sum dz1; dW1 = x^T bf16(dz1).
#include <cuda_bf16.h>

#include "hm_internal.cuh"

namespace hm {
namespace {

constexpr int IN = 16, HID = 64;
constexpr int P_W1 = 0, P_B1 = 1024, P_W2 = 1088, P_B2 = 5184, P_W3 = 5248, P_B3 = 5312;
constexpr int NPARAM = 5313;
constexpr int MLP_THREADS = 256;
constexpr int BWD_PART = 3 * 64 + 2;  // per-block backward partial: db1 | db2 | dw3 | db3 | loss

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Weights staged in shared memory, bf16, in the layouts the fragments read:
// w1t[out][in] and w2t[out][in] (B operands of the forward), w2[in][out] (B
// operand of dh1 = dz2 W2^T), w3[out].
struct Smem {
  __nv_bfloat16 w1t[HID * IN];
  __nv_bfloat16 w2t[HID * HID];
  __nv_bfloat16 w2[HID * HID];
  float b1[HID], b2[HID], w3[HID];
  float b3;
};

__device__ void stage_params(Smem& s, const float* __restrict__ p) {
  for (int i = threadIdx.x; i < IN * HID; i += blockDim.x) {
    const int in = i / HID, out = i % HID;
    s.w1t[out * IN + in] = __float2bfloat16_rn(p[P_W1 + i]);
  }
  for (int i = threadIdx.x; i < HID * HID; i += blockDim.x) {
    const int in = i / HID, out = i % HID;
    const __nv_bfloat16 v = __float2bfloat16_rn(p[P_W2 + i]);
    s.w2t[out * HID + in] = v;
    s.w2[i] = v;
  }
  for (int i = threadIdx.x; i < HID; i += blockDim.x) {
    s.b1[i] = p[P_B1 + i];
    s.b2[i] = p[P_B2 + i];
    s.w3[i] = bf16r(p[P_W3 + i]);
  }
  if (threadIdx.x == 0) s.b3 = p[P_B3];
  __syncthreads();
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// Forward of one 16-row tile. Fragment coordinates: g = lane / 4 (rows g and
// g + 8), t = lane % 4 (columns 8j + 2t, 8j + 2t + 1 of n-tile j).
struct Tile {
  float z1[8][4], z2[8][4];  // pre-activations (C fragments)
  float y[2];                // outputs of rows g, g + 8
};

__device__ __forceinline__ void forward_tile(const Smem& s, const float* __restrict__ X, int64_t n,
                                             int64_t r0, Tile& T) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t ra = r0 + g, rb = r0 + g + 8;
  float xa[4] = {0, 0, 0, 0}, xb[4] = {0, 0, 0, 0};
  if (ra < n) {
    const float* p = X + ra * IN;
    xa[0] = p[2 * t];
    xa[1] = p[2 * t + 1];
    xa[2] = p[2 * t + 8];
    xa[3] = p[2 * t + 9];
  }
  if (rb < n) {
    const float* p = X + rb * IN;
    xb[0] = p[2 * t];
    xb[1] = p[2 * t + 1];
    xb[2] = p[2 * t + 8];
    xb[3] = p[2 * t + 9];
  }
  const uint32_t a[4] = {pack_bf16(xa[0], xa[1]), pack_bf16(xb[0], xb[1]), pack_bf16(xa[2], xa[3]),
                         pack_bf16(xb[2], xb[3])};
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = 8 * j + 2 * t;
    T.z1[j][0] = s.b1[c];
    T.z1[j][1] = s.b1[c + 1];
    T.z1[j][2] = s.b1[c];
    T.z1[j][3] = s.b1[c + 1];
    const __nv_bfloat16* w = s.w1t + (8 * j + g) * IN + 2 * t;
    mma16816(T.z1[j], a, ld32(w), ld32(w + 8));
  }
  uint32_t a2[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float* d0 = T.z1[2 * k];
    const float* d1 = T.z1[2 * k + 1];
    a2[k][0] = pack_bf16(fmaxf(d0[0], 0.f), fmaxf(d0[1], 0.f));
    a2[k][1] = pack_bf16(fmaxf(d0[2], 0.f), fmaxf(d0[3], 0.f));
    a2[k][2] = pack_bf16(fmaxf(d1[0], 0.f), fmaxf(d1[1], 0.f));
    a2[k][3] = pack_bf16(fmaxf(d1[2], 0.f), fmaxf(d1[3], 0.f));
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = 8 * j + 2 * t;
    T.z2[j][0] = s.b2[c];
    T.z2[j][1] = s.b2[c + 1];
    T.z2[j][2] = s.b2[c];
    T.z2[j][3] = s.b2[c + 1];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __nv_bfloat16* w = s.w2t + (8 * j + g) * HID + 16 * k + 2 * t;
      mma16816(T.z2[j], a2[k], ld32(w), ld32(w + 8));
    }
  }
  float pa = 0.f, pb = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = 8 * j + 2 * t;
    pa += bf16r(fmaxf(T.z2[j][0], 0.f)) * s.w3[c] + bf16r(fmaxf(T.z2[j][1], 0.f)) * s.w3[c + 1];
    pb += bf16r(fmaxf(T.z2[j][2], 0.f)) * s.w3[c] + bf16r(fmaxf(T.z2[j][3], 0.f)) * s.w3[c + 1];
  }
  pa += __shfl_xor_sync(0xffffffffu, pa, 1);
  pa += __shfl_xor_sync(0xffffffffu, pa, 2);
  pb += __shfl_xor_sync(0xffffffffu, pb, 1);
  pb += __shfl_xor_sync(0xffffffffu, pb, 2);
  T.y[0] = pa + s.b3;
  T.y[1] = pb + s.b3;
}

__global__ void __launch_bounds__(MLP_THREADS)
    k_mlp_forward(const float* __restrict__ params, const float* __restrict__ X, int64_t n,
                  float* __restrict__ y) {
  __shared__ Smem s;
  stage_params(s, params);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t tiles = (n + 15) / 16;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t tile = warp; tile < tiles; tile += nwarps) {
    Tile T;
    forward_tile(s, X, n, tile * 16, T);
    if (t == 0) {
      const int64_t ra = tile * 16 + g, rb = ra + 8;
      if (ra < n) y[ra] = T.y[0];
      if (rb < n) y[rb] = T.y[1];
    }
  }
}

// Per-tile backward: bias and w3 gradients (fp32 atomics), and the bf16
// matrices the weight-gradient GEMMs contract over the rows:
// Xb[n][16], H1b[n][64], DZ2b[n][64], DZ1b[n][64].
__global__ void __launch_bounds__(MLP_THREADS)
    k_mlp_backward(const float* __restrict__ params, const float* __restrict__ X,
                   const float* __restrict__ target, int64_t n, float inv_n,
                   float* __restrict__ part, __nv_bfloat16* __restrict__ Xb,
                   __nv_bfloat16* __restrict__ H1b, __nv_bfloat16* __restrict__ DZ2b,
                   __nv_bfloat16* __restrict__ DZ1b) {
  __shared__ Smem s;
  __shared__ float gs[MLP_THREADS / 32][BWD_PART];  // per warp: db1 | db2 | dw3 | db3 | loss
  stage_params(s, params);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t tiles = (n + 15) / 16;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float db1[16], db2[16], dw3[16], db3 = 0.f, lsum = 0.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) db1[i] = db2[i] = dw3[i] = 0.f;
  for (int64_t tile = warp; tile < tiles; tile += nwarps) {
    Tile T;
    const int64_t r0 = tile * 16, ra = r0 + g, rb = r0 + g + 8;
    forward_tile(s, X, n, r0, T);
    const bool va = ra < n, vb = rb < n;
    const float ea = va ? T.y[0] - target[ra] : 0.f, eb = vb ? T.y[1] - target[rb] : 0.f;
    const float dya = 2.f * ea * inv_n, dyb = 2.f * eb * inv_n;
    if (t == 0) {
      db3 += dya + dyb;
      lsum += ea * ea + eb * eb;
    }
    // dz2 (C fragments) and its bf16 A fragments
    uint32_t adz[4][4];
    float dz2[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * j + 2 * t;
      const float h00 = bf16r(fmaxf(T.z2[j][0], 0.f)), h01 = bf16r(fmaxf(T.z2[j][1], 0.f));
      const float h10 = bf16r(fmaxf(T.z2[j][2], 0.f)), h11 = bf16r(fmaxf(T.z2[j][3], 0.f));
      dw3[2 * j] += dya * h00 + dyb * h10;
      dw3[2 * j + 1] += dya * h01 + dyb * h11;
      dz2[j][0] = T.z2[j][0] > 0.f ? dya * s.w3[c] : 0.f;
      dz2[j][1] = T.z2[j][1] > 0.f ? dya * s.w3[c + 1] : 0.f;
      dz2[j][2] = T.z2[j][2] > 0.f ? dyb * s.w3[c] : 0.f;
      dz2[j][3] = T.z2[j][3] > 0.f ? dyb * s.w3[c + 1] : 0.f;
      db2[2 * j] += dz2[j][0] + dz2[j][2];
      db2[2 * j + 1] += dz2[j][1] + dz2[j][3];
      if (va) {
        *reinterpret_cast<uint32_t*>(DZ2b + ra * HID + c) = pack_bf16(dz2[j][0], dz2[j][1]);
        *reinterpret_cast<uint32_t*>(H1b + ra * HID + c) =
            pack_bf16(fmaxf(T.z1[j][0], 0.f), fmaxf(T.z1[j][1], 0.f));
      }
      if (vb) {
        *reinterpret_cast<uint32_t*>(DZ2b + rb * HID + c) = pack_bf16(dz2[j][2], dz2[j][3]);
        *reinterpret_cast<uint32_t*>(H1b + rb * HID + c) =
            pack_bf16(fmaxf(T.z1[j][2], 0.f), fmaxf(T.z1[j][3], 0.f));
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      adz[k][0] = pack_bf16(dz2[2 * k][0], dz2[2 * k][1]);
      adz[k][1] = pack_bf16(dz2[2 * k][2], dz2[2 * k][3]);
      adz[k][2] = pack_bf16(dz2[2 * k + 1][0], dz2[2 * k + 1][1]);
      adz[k][3] = pack_bf16(dz2[2 * k + 1][2], dz2[2 * k + 1][3]);
    }
    // dh1 = bf16(dz2) W2^T: B[k = out c][n = in i] = W2[i][c], read from w2[i][c]
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float dh[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const __nv_bfloat16* w = s.w2 + (8 * j + g) * HID + 16 * k + 2 * t;
        mma16816(dh, adz[k], ld32(w), ld32(w + 8));
      }
      const int c = 8 * j + 2 * t;
      const float d00 = T.z1[j][0] > 0.f ? dh[0] : 0.f, d01 = T.z1[j][1] > 0.f ? dh[1] : 0.f;
      const float d10 = T.z1[j][2] > 0.f ? dh[2] : 0.f, d11 = T.z1[j][3] > 0.f ? dh[3] : 0.f;
      db1[2 * j] += d00 + d10;
      db1[2 * j + 1] += d01 + d11;
      if (va) *reinterpret_cast<uint32_t*>(DZ1b + ra * HID + c) = pack_bf16(d00, d01);
      if (vb) *reinterpret_cast<uint32_t*>(DZ1b + rb * HID + c) = pack_bf16(d10, d11);
    }
    // bf16 copy of the inputs for dW1
    if (va) {
      const float* p = X + ra * IN;
      *reinterpret_cast<uint32_t*>(Xb + ra * IN + 2 * t) = pack_bf16(p[2 * t], p[2 * t + 1]);
      *reinterpret_cast<uint32_t*>(Xb + ra * IN + 2 * t + 8) = pack_bf16(p[2 * t + 8], p[2 * t + 9]);
    }
    if (vb) {
      const float* p = X + rb * IN;
      *reinterpret_cast<uint32_t*>(Xb + rb * IN + 2 * t) = pack_bf16(p[2 * t], p[2 * t + 1]);
      *reinterpret_cast<uint32_t*>(Xb + rb * IN + 2 * t + 8) = pack_bf16(p[2 * t + 8], p[2 * t + 9]);
    }
  }
  // Fixed-order reductions (results do not depend on scheduling): over the 8
  // row groups of the warp by shuffles, over the warps of the block in warp
  // order, and over blocks by k_sum_partials in block order.
#pragma unroll
  for (int i = 0; i < 16; ++i) {
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      db1[i] += __shfl_xor_sync(0xffffffffu, db1[i], o);
      db2[i] += __shfl_xor_sync(0xffffffffu, db2[i], o);
      dw3[i] += __shfl_xor_sync(0xffffffffu, dw3[i], o);
    }
  }
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) {
    db3 += __shfl_xor_sync(0xffffffffu, db3, o);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  }
  const int wib = threadIdx.x >> 5;
  if (g == 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = 8 * j + 2 * t + e;
        gs[wib][c] = db1[2 * j + e];
        gs[wib][HID + c] = db2[2 * j + e];
        gs[wib][2 * HID + c] = dw3[2 * j + e];
      }
  }
  if (lane == 0) {
    gs[wib][3 * HID] = db3;
    gs[wib][3 * HID + 1] = lsum;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < BWD_PART; i += blockDim.x) {
    float a = 0.f;
#pragma unroll
    for (int w = 0; w < MLP_THREADS / 32; ++w) a += gs[w][i];
    part[(int64_t)blockIdx.x * BWD_PART + i] = a;
  }
}

// Sum over blocks b, in block order, of part[b * width + i], written to
// grad[grad_off + i]; grad_off < 0 selects the backward partial's layout
// (db1 | db2 | dw3 | db3 | loss sum), scattered to its parameters and *loss.
__global__ void k_sum_partials(const float* __restrict__ part, int nblocks, int width,
                               float* __restrict__ grad, int grad_off, float* __restrict__ loss) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < width; i += gridDim.x * blockDim.x) {
    float a = 0.f;
    for (int b = 0; b < nblocks; ++b) a += part[(int64_t)b * width + i];
    if (grad_off >= 0) {
      grad[grad_off + i] = a;
    } else {
      // backward layout: db1 | db2 | dw3 | db3 | loss
      if (i < HID) grad[P_B1 + i] = a;
      else if (i < 2 * HID) grad[P_B2 + i - HID] = a;
      else if (i < 3 * HID) grad[P_W3 + i - 2 * HID] = a;
      else if (i == 3 * HID) grad[P_B3] = a;
      else if (loss) *loss = a;
    }
  }
}

// Partial dW[ka][64] = A^T B over one block's rows, A: [n][ka] bf16, B: [n][64]
// bf16 (ka = 16 or 64), written to part[block]. Each block takes a contiguous
// range of rows in 16-row steps staged in shared memory; warp w owns output
// rows 16w..16w+15 (8 n-tiles in registers) and reads A^T / B fragments with
// ldmatrix.trans.
template <int KA>
__global__ void __launch_bounds__(KA * 2)
    k_mlp_wgrad(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
                int64_t n, int64_t rows_per_block, float* __restrict__ part) {
  constexpr int WARPS = KA / 16;
  constexpr int AS = KA + 8, BS = HID + 8;  // padded row strides (bank spread)
  __shared__ __align__(16) __nv_bfloat16 As[16 * AS];
  __shared__ __align__(16) __nv_bfloat16 Bs[16 * BS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  const int64_t lo = blockIdx.x * rows_per_block;
  const int64_t hi = min(n, lo + rows_per_block);
  for (int64_t r0 = lo; r0 < hi; r0 += 16) {
    __syncthreads();
    // stage 16 rows of A (KA cols) and B (64 cols) as 16-byte pieces, zero past n
    for (int i = threadIdx.x; i < 16 * (KA / 8); i += blockDim.x) {
      const int r = i / (KA / 8), c = (i % (KA / 8)) * 8;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (r0 + r < hi) v = *reinterpret_cast<const uint4*>(A + (r0 + r) * KA + c);
      *reinterpret_cast<uint4*>(As + r * AS + c) = v;
    }
    for (int i = threadIdx.x; i < 16 * (HID / 8); i += blockDim.x) {
      const int r = i / (HID / 8), c = (i % (HID / 8)) * 8;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (r0 + r < hi) v = *reinterpret_cast<const uint4*>(B + (r0 + r) * HID + c);
      *reinterpret_cast<uint4*>(Bs + r * BS + c) = v;
    }
    __syncthreads();
    if (warp < WARPS) {
      // A^T fragment: matrices (rows of A 0-7 | 8-15) x (cols 16w + 0-7 | 8-15)
      const int q = lane >> 3, rho = lane & 7;
      const int rb = (q >> 1) * 8, cb = 16 * warp + (q & 1) * 8;
      uint32_t a[4];
      const uint32_t pa = (uint32_t)__cvta_generic_to_shared(As + (rb + rho) * AS + cb);
      asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                   : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                   : "r"(pa));
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        // B fragments of n-tiles 2jj and 2jj+1: rows 0-7 / 8-15, cols 16jj + 0-7 / 8-15
        const int brow = (q & 1) * 8 + rho, bcol = 16 * jj + (q >> 1) * 8;
        const uint32_t pb = (uint32_t)__cvta_generic_to_shared(Bs + brow * BS + bcol);
        uint32_t b[4];
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                     : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
                     : "r"(pb));
        mma16816(acc[2 * jj], a, b[0], b[1]);
        mma16816(acc[2 * jj + 1], a, b[2], b[3]);
      }
    }
  }
  if (warp < WARPS) {
    const int g = lane >> 2, t = lane & 3;
    float* out = part + (int64_t)blockIdx.x * (KA * HID);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = 8 * j + 2 * t, ra = 16 * warp + g, rb = ra + 8;
      *reinterpret_cast<float2*>(out + ra * HID + c) = make_float2(acc[j][0], acc[j][1]);
      *reinterpret_cast<float2*>(out + rb * HID + c) = make_float2(acc[j][2], acc[j][3]);
    }
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

int mlp_blocks(int64_t n) {
  int64_t tiles = (n + 15) / 16;
  int64_t b = (tiles + (MLP_THREADS / 32) - 1) / (MLP_THREADS / 32);
  if (b > 152 * 4) b = 152 * 4;
  return (int)(b < 1 ? 1 : b);
}

// weight-gradient blocks: at least 128 rows each (a multiple of 16), at most
// 512 blocks, so that a minibatch of a few thousand rows still spreads over
// tens of SMs
int64_t wgrad_rows_per_block(int64_t n) {
  const int64_t r = (n + 511) / 512;
  return r < 128 ? 128 : ((r + 15) / 16) * 16;
}
int wgrad_blocks(int64_t n) {
  const int64_t b = (n + wgrad_rows_per_block(n) - 1) / wgrad_rows_per_block(n);
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int mlp_num_params() { return NPARAM; }

size_t mlp_scratch_bytes(int64_t n) {
  if (n <= 0) return 0;
  const size_t mats = (size_t)n * (IN + 3 * HID) * sizeof(__nv_bfloat16);
  const size_t parts = ((size_t)mlp_blocks(n) * BWD_PART +
                        (size_t)wgrad_blocks(n) * (HID * HID + IN * HID)) * sizeof(float);
  return ((mats + 255) / 256) * 256 + parts;
}

void mlp_forward(const float* params, const float* X, int64_t n, float* y, cudaStream_t s) {
  if (n == 0) return;
  k_mlp_forward<<<mlp_blocks(n), MLP_THREADS, 0, s>>>(params, X, n, y);
  HM_KCHECK();
}

// Gradient of L = mean over the n rows of (y - target)^2 into grad (zeroed
// here); scratch holds 2 * n * (16 + 3 * 64) bytes of bf16 matrices.
void mlp_backward(const float* params, const float* X, const float* target, int64_t n,
                  float* grad, float* loss_sum, void* scratch, cudaStream_t s) {
  if (n == 0) {
    HM_CUDA(cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), s));
    if (loss_sum) HM_CUDA(cudaMemsetAsync(loss_sum, 0, sizeof(float), s));
    return;
  }
  __nv_bfloat16* Xb = (__nv_bfloat16*)scratch;
  __nv_bfloat16* H1b = Xb + n * IN;
  __nv_bfloat16* DZ2b = H1b + n * HID;
  __nv_bfloat16* DZ1b = DZ2b + n * HID;
  const size_t mats = (size_t)n * (IN + 3 * HID) * sizeof(__nv_bfloat16);
  float* part_b = (float*)((char*)scratch + ((mats + 255) / 256) * 256);
  const int bb = mlp_blocks(n), wb = wgrad_blocks(n);
  float* part_w2 = part_b + (size_t)bb * BWD_PART;
  float* part_w1 = part_w2 + (size_t)wb * HID * HID;
  k_mlp_backward<<<bb, MLP_THREADS, 0, s>>>(params, X, target, n, 1.f / (float)n, part_b, Xb,
                                            H1b, DZ2b, DZ1b);
  HM_KCHECK();
  const int64_t rows = wgrad_rows_per_block(n);
  k_mlp_wgrad<HID><<<wb, HID * 2, 0, s>>>(H1b, DZ2b, n, rows, part_w2);
  HM_KCHECK();
  k_mlp_wgrad<IN><<<wb, IN * 2 < 32 ? 32 : IN * 2, 0, s>>>(Xb, DZ1b, n, rows, part_w1);
  HM_KCHECK();
  k_sum_partials<<<1, 256, 0, s>>>(part_b, bb, BWD_PART, grad, -1, loss_sum);
  HM_KCHECK();
  k_sum_partials<<<16, 256, 0, s>>>(part_w2, wb, HID * HID, grad, P_W2, nullptr);
  HM_KCHECK();
  k_sum_partials<<<4, 256, 0, s>>>(part_w1, wb, IN * HID, grad, P_W1, nullptr);
  HM_KCHECK();
}

void mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
              cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, grad, m, v, NPARAM, lr, b1, b2, 1e-8f, c1,
                                              c2);
  HM_KCHECK();
}

}  // namespace hm

extern "C" {

int hm_mlp_num_params(void) { return hm::mlp_num_params(); }

size_t hm_mlp_scratch_bytes(int64_t n) { return hm::mlp_scratch_bytes(n); }

hm_status hm_mlp_forward(const float* d_params, const float* d_x, int64_t n, float* d_y,
                         void* stream) {
  return hm::guarded([&] {
    HM_CHECK(n >= 0 && (n == 0 || (d_params && d_x && d_y)), HM_EINVAL, "bad arguments");
    hm::mlp_forward(d_params, d_x, n, d_y, (cudaStream_t)stream);
  });
}

hm_status hm_mlp_backward(const float* d_params, const float* d_x, const float* d_target,
                          int64_t n, float* d_grad, float* d_loss_sum, void* d_scratch,
                          void* stream) {
  return hm::guarded([&] {
    HM_CHECK(n >= 0 && d_params && d_grad, HM_EINVAL, "bad arguments");
    HM_CHECK(n == 0 || (d_x && d_target && d_scratch), HM_EINVAL, "bad arguments");
    hm::mlp_backward(d_params, d_x, d_target, n, d_grad, d_loss_sum, d_scratch,
                     (cudaStream_t)stream);
  });
}

hm_status hm_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int step,
                      float lr, void* stream) {
  return hm::guarded([&] {
    HM_CHECK(d_params && d_grad && d_m && d_v && step >= 1, HM_EINVAL, "bad arguments");
    hm::mlp_adam(d_params, d_grad, d_m, d_v, step, lr, (cudaStream_t)stream);
  });
}

}  // extern "C"
