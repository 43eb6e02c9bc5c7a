// lbm_mlp.cuh -- the learned first-layer correction: a 9-64-64-64-4 network
// (tanh hidden layers) evaluated per first-cell column, and its training.
//
// The paper has no learned component; this is the near-wall/canopy
// correction of the first cell: inputs are u_x, |S| and the leaf-area density
// of the three cells above the ground (x, y = 0..2, z), outputs are
// (du_x, du_z, dtau_x, dtau_z), applied by the next step as the extra
// acceleration a = (lam du_x - dtau_x, lam du_z - dtau_z) of cell (x, 0, z).
//
// Precision: weights and activations are BF16, products accumulate in FP32.
// Inference runs on the tensor cores (mma.sync m16n8k16, BF16 in, FP32
// accumulate): one warp pushes 16 columns through all four layers with the
// activations held in registers (an accumulator fragment of one layer is, laid
// side by side, the A fragment of the next).  Training (forward, backward,
// weight gradients, Adam) runs on the CUDA cores with the same rounding.
//
// Flat parameter vector (FP32), rows = outputs, row-major:
//   W1[64][9] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64] b4[4]
//   x_mean[9] x_std[9] y_mean[4] y_std[4]
#pragma once

#include "lbm_features.cuh"

namespace lbm {


__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// D += A B for one m16n8k16 tile (BF16 inputs, FP32 accumulators).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Weights staged in shared memory for the tensor-core pass: BF16, row-major
// [out][in]; the first layer's inputs are padded to 16, the last layer's
// outputs to 8 (padding zero).
struct MlpSmem {
  __nv_bfloat16 w1[64 * 16];
  __nv_bfloat16 w2[64 * 64];
  __nv_bfloat16 w3[64 * 64];
  __nv_bfloat16 w4[8 * 64];
  float b1[64], b2[64], b3[64], b4[8];
  float xm[16], xinv[16], ym[4], ys[4];
};

__device__ void mlp_stage(MlpSmem& s, const float* __restrict__ th) {
  for (int k = threadIdx.x; k < 64 * 16; k += blockDim.x) {
    const int o = k / 16, i = k % 16;
    s.w1[k] = __float2bfloat16_rn(i < MLP_IN ? th[OFF_W1 + o * MLP_IN + i] : 0.f);
  }
  for (int k = threadIdx.x; k < 64 * 64; k += blockDim.x) {
    s.w2[k] = __float2bfloat16_rn(th[OFF_W2 + k]);
    s.w3[k] = __float2bfloat16_rn(th[OFF_W3 + k]);
  }
  for (int k = threadIdx.x; k < 8 * 64; k += blockDim.x)
    s.w4[k] = __float2bfloat16_rn(k < 4 * 64 ? th[OFF_W4 + k] : 0.f);
  for (int k = threadIdx.x; k < 64; k += blockDim.x) {
    s.b1[k] = th[OFF_B1 + k];
    s.b2[k] = th[OFF_B2 + k];
    s.b3[k] = th[OFF_B3 + k];
  }
  for (int k = threadIdx.x; k < 16; k += blockDim.x) {
    s.xm[k] = k < MLP_IN ? th[OFF_XM + k] : 0.f;
    s.xinv[k] = k < MLP_IN ? 1.0f / th[OFF_XS + k] : 0.f;
    if (k < 8) s.b4[k] = k < 4 ? th[OFF_B4 + k] : 0.f;
    if (k < 4) {
      s.ym[k] = th[OFF_YM + k];
      s.ys[k] = th[OFF_YS + k];
    }
  }
}

// One hidden layer on the tensor cores: h (A fragments, KS k-slices of 16) ->
// tanh(W h + b) as the A fragments of the next layer (4 k-slices of 16).
template <int KS>
__device__ __forceinline__ void mlp_hidden(const uint32_t (&a)[KS][4], uint32_t (&out)[4][4],
                                           const __nv_bfloat16* w, const float* b, int lane) {
  const int g = lane >> 2, t = lane & 3;
  constexpr int K = KS * 16;
#pragma unroll
  for (int j = 0; j < 8; j++) {  // n-tiles of 8 outputs
    // accumulator layout: d0, d1 = (row g, cols 2t, 2t+1); d2, d3 = (row g+8, same cols)
    float d[4];
    d[0] = b[8 * j + 2 * t];
    d[1] = b[8 * j + 2 * t + 1];
    d[2] = d[0];
    d[3] = d[1];
    const __nv_bfloat16* wr = w + (8 * j + g) * K + 2 * t;  // W[n = 8j + g][k]
#pragma unroll
    for (int s = 0; s < KS; s++) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr + 16 * s);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 16 * s + 8);
      mma_bf16(d, a[s], b0, b1);
    }
    // n-tile j feeds k-slice j/2 of the next layer: even tiles the low 8 k
    // (registers 0, 1), odd tiles the high 8 k (registers 2, 3)
    const int ks = j >> 1, hi = (j & 1) * 2;
    out[ks][hi + 0] = pack_bf16(tanh_fast(d[0]), tanh_fast(d[1]));
    out[ks][hi + 1] = pack_bf16(tanh_fast(d[2]), tanh_fast(d[3]));
  }
}

// The network on 16 rows whose standardised inputs sit in `xin` (shared,
// [16][16] BF16, columns 9..15 zero); returns the raw outputs of rows g and
// g + 8 for columns 2t, 2t+1 (lanes with t < 2 hold the 4 real outputs).
__device__ __forceinline__ void mlp_rows16(const MlpSmem& s, const __nv_bfloat16* xin, int lane,
                                           float (&o)[4]) {
  const int g = lane >> 2, t = lane & 3;
  uint32_t a0[1][4];
  a0[0][0] = *reinterpret_cast<const uint32_t*>(xin + g * 16 + 2 * t);
  a0[0][1] = *reinterpret_cast<const uint32_t*>(xin + (g + 8) * 16 + 2 * t);
  a0[0][2] = *reinterpret_cast<const uint32_t*>(xin + g * 16 + 2 * t + 8);
  a0[0][3] = *reinterpret_cast<const uint32_t*>(xin + (g + 8) * 16 + 2 * t + 8);
  uint32_t h1[4][4], h2[4][4], h3[4][4];
  mlp_hidden<1>(a0, h1, s.w1, s.b1, lane);
  mlp_hidden<4>(h1, h2, s.w2, s.b2, lane);
  mlp_hidden<4>(h2, h3, s.w3, s.b3, lane);
  float d[4];
  d[0] = s.b4[2 * t];
  d[1] = s.b4[2 * t + 1];
  d[2] = d[0];
  d[3] = d[1];
  const __nv_bfloat16* wr = s.w4 + g * 64 + 2 * t;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wr + 16 * k);
    const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wr + 16 * k + 8);
    mma_bf16(d, h3[k], b0, b1);
  }
  o[0] = d[0];
  o[1] = d[1];
  o[2] = d[2];
  o[3] = d[3];
}

// Outputs of rows g, g+8 in physical units: y = y_mean + y_std * o; lanes
// with t = 0 end up with (y0, y1, y2, y3) of row g in r0 and of row g+8 in r1.
__device__ __forceinline__ void mlp_gather_outputs(const MlpSmem& s, const float (&o)[4], int lane,
                                                   float (&r0)[4], float (&r1)[4]) {
  const int t = lane & 3;
  const float c0 = t < 2 ? s.ym[2 * t] + s.ys[2 * t] * o[0] : 0.f;
  const float c1 = t < 2 ? s.ym[2 * t + 1] + s.ys[2 * t + 1] * o[1] : 0.f;
  const float c2 = t < 2 ? s.ym[2 * t] + s.ys[2 * t] * o[2] : 0.f;
  const float c3 = t < 2 ? s.ym[2 * t + 1] + s.ys[2 * t + 1] * o[3] : 0.f;
  // outputs 2, 3 live in the lane with t = 1 (lane + 1)
  const float u0 = __shfl_down_sync(0xffffffffu, c0, 1);
  const float u1 = __shfl_down_sync(0xffffffffu, c1, 1);
  const float u2 = __shfl_down_sync(0xffffffffu, c2, 1);
  const float u3 = __shfl_down_sync(0xffffffffu, c3, 1);
  r0[0] = c0; r0[1] = c1; r0[2] = u0; r0[3] = u1;
  r1[0] = c2; r1[1] = c3; r1[2] = u2; r1[3] = u3;
}

// Inference on rows of raw features X[n][9] -> Y[n][4] (tensor cores).
__global__ void __launch_bounds__(128) mlp_infer_kernel(const float* __restrict__ th,
                                                        const float* __restrict__ X, long long n,
                                                        float* __restrict__ Y) {
  __shared__ MlpSmem s;
  __shared__ __align__(16) __nv_bfloat16 xin[4][16 * 16];
  mlp_stage(s, th);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long tiles = (n + 15) / 16;
  for (long long tile = (long long)blockIdx.x * 4 + warp; tile < tiles; tile += (long long)gridDim.x * 4) {
    __syncwarp();
    if (lane < 16) {
      const long long r = tile * 16 + lane;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const float v = (r < n && k < MLP_IN) ? (X[r * MLP_IN + k] - s.xm[k]) * s.xinv[k] : 0.f;
        xin[warp][lane * 16 + k] = __float2bfloat16_rn(v);
      }
    }
    __syncwarp();
    float o[4], r0[4], r1[4];
    mlp_rows16(s, xin[warp], lane, o);
    mlp_gather_outputs(s, o, lane, r0, r1);
    if ((lane & 3) == 0) {
      const long long ra = tile * 16 + (lane >> 2), rb = ra + 8;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        if (ra < n) Y[ra * MLP_OUT + k] = r0[k];
        if (rb < n) Y[rb * MLP_OUT + k] = r1[k];
      }
    }
  }
}

// The network on feature rows X[n][9] (tensor cores), written as the layer-0
// acceleration a = (lam du_x - dtau_x, lam du_z - dtau_z) of each row.
__global__ void __launch_bounds__(128) mlp_accel_kernel(const float* __restrict__ th,
                                                        const float* __restrict__ X, long long n,
                                                        float lam, float2* __restrict__ accel) {
  __shared__ MlpSmem s;
  __shared__ __align__(16) __nv_bfloat16 xin[4][16 * 16];
  mlp_stage(s, th);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long tiles = (n + 15) / 16;
  for (long long tile = (long long)blockIdx.x * 4 + warp; tile < tiles; tile += (long long)gridDim.x * 4) {
    __syncwarp();
    if (lane < 16) {
      const long long r = tile * 16 + lane;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const float v = (r < n && k < MLP_IN) ? (X[r * MLP_IN + k] - s.xm[k]) * s.xinv[k] : 0.f;
        xin[warp][lane * 16 + k] = __float2bfloat16_rn(v);
      }
    }
    __syncwarp();
    float o[4], r0[4], r1[4];
    mlp_rows16(s, xin[warp], lane, o);
    mlp_gather_outputs(s, o, lane, r0, r1);
    if ((lane & 3) == 0) {
      const long long ra = tile * 16 + (lane >> 2), rb = ra + 8;
      if (ra < n) accel[ra] = make_float2(lam * r0[0] - r0[2], lam * r0[1] - r0[3]);
      if (rb < n) accel[rb] = make_float2(lam * r1[0] - r1[2], lam * r1[1] - r1[3]);
    }
  }
}

// ---- training (CUDA cores; same BF16 rounding of weights and activations) -------
// Weights staged as FP32 values already rounded to BF16.
struct MlpTrainSmem {
  float w1[64 * 9], w2[64 * 64], w3[64 * 64], w4[4 * 64];
  float b1[64], b2[64], b3[64], b4[4];
  float xm[9], xinv[9], ym[4], yinv[4];
};

__device__ void mlp_stage_train(MlpTrainSmem& s, const float* __restrict__ th) {
  for (int k = threadIdx.x; k < 64 * 64; k += blockDim.x) {
    s.w2[k] = bf16r(th[OFF_W2 + k]);
    s.w3[k] = bf16r(th[OFF_W3 + k]);
    if (k < 64 * 9) s.w1[k] = bf16r(th[OFF_W1 + k]);
    if (k < 4 * 64) s.w4[k] = bf16r(th[OFF_W4 + k]);
    if (k < 64) {
      s.b1[k] = th[OFF_B1 + k];
      s.b2[k] = th[OFF_B2 + k];
      s.b3[k] = th[OFF_B3 + k];
    }
    if (k < 9) {
      s.xm[k] = th[OFF_XM + k];
      s.xinv[k] = 1.0f / th[OFF_XS + k];
    }
    if (k < 4) {
      s.b4[k] = th[OFF_B4 + k];
      s.ym[k] = th[OFF_YM + k];
      s.yinv[k] = 1.0f / th[OFF_YS + k];
    }
  }
}

// Forward for training: one thread per sample of a batch of rows idx[0..n);
// stores the layer inputs H0 (standardised, [n][9]) and activations H1..H3
// ([n][64], BF16-rounded), and dL/do = 2 (o - t) / (4 n_total) in D4 ([n][4]);
// adds the sum of squared errors to *sse.
__global__ void __launch_bounds__(128) mlp_train_fwd(const float* __restrict__ th,
                                                     const float* __restrict__ X,
                                                     const float* __restrict__ Y,
                                                     const int* __restrict__ idx, int n,
                                                     float scale, float* __restrict__ H0,
                                                     float* __restrict__ H1, float* __restrict__ H2,
                                                     float* __restrict__ H3,
                                                     float* __restrict__ D4, float* sse) {
  __shared__ MlpTrainSmem s;
  mlp_stage_train(s, th);
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  float err = 0.f;
  if (r < n) {
    const long long row = idx ? idx[r] : r;
    float h0[9], ha[64], hb[64];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      h0[k] = bf16r((X[row * 9 + k] - s.xm[k]) * s.xinv[k]);
      H0[(long long)r * 9 + k] = h0[k];
    }
#pragma unroll
    for (int j = 0; j < 64; j++) {
      float a = s.b1[j];
#pragma unroll
      for (int k = 0; k < 9; k++) a = fmaf(s.w1[j * 9 + k], h0[k], a);
      ha[j] = bf16r(tanh_fast(a));
      H1[(long long)r * 64 + j] = ha[j];
    }
#pragma unroll
    for (int j = 0; j < 64; j++) {
      float a = s.b2[j];
#pragma unroll
      for (int k = 0; k < 64; k++) a = fmaf(s.w2[j * 64 + k], ha[k], a);
      hb[j] = bf16r(tanh_fast(a));
      H2[(long long)r * 64 + j] = hb[j];
    }
#pragma unroll
    for (int j = 0; j < 64; j++) {
      float a = s.b3[j];
#pragma unroll
      for (int k = 0; k < 64; k++) a = fmaf(s.w3[j * 64 + k], hb[k], a);
      ha[j] = bf16r(tanh_fast(a));
      H3[(long long)r * 64 + j] = ha[j];
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
      float a = s.b4[j];
#pragma unroll
      for (int k = 0; k < 64; k++) a = fmaf(s.w4[j * 64 + k], ha[k], a);
      const float tgt = (Y[row * 4 + j] - s.ym[j]) * s.yinv[j];
      const float e = a - tgt;
      err += e * e;
      D4[(long long)r * 4 + j] = scale * e;
    }
  }
  err = warp_sum(err);
  if ((threadIdx.x & 31) == 0 && err != 0.f) atomicAdd(sse, err);
}

// Backward for training: the deltas of the hidden layers (FP32), one thread
// per sample: D3 = (W4^T D4) (1 - H3^2), D2 = (W3^T D3) (1 - H2^2), D1 = ...
__global__ void __launch_bounds__(128) mlp_train_bwd(const float* __restrict__ th, int n,
                                                     const float* __restrict__ H1,
                                                     const float* __restrict__ H2,
                                                     const float* __restrict__ H3,
                                                     const float* __restrict__ D4,
                                                     float* __restrict__ D1, float* __restrict__ D2,
                                                     float* __restrict__ D3) {
  __shared__ MlpTrainSmem s;
  mlp_stage_train(s, th);
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float da[64], db[64], d4[4];
#pragma unroll
  for (int j = 0; j < 4; j++) d4[j] = D4[(long long)r * 4 + j];
#pragma unroll
  for (int k = 0; k < 64; k++) {
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < 4; j++) a = fmaf(s.w4[j * 64 + k], d4[j], a);
    const float h = H3[(long long)r * 64 + k];
    da[k] = a * (1.0f - h * h);
    D3[(long long)r * 64 + k] = da[k];
  }
#pragma unroll
  for (int k = 0; k < 64; k++) {
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < 64; j++) a = fmaf(s.w3[j * 64 + k], da[j], a);
    const float h = H2[(long long)r * 64 + k];
    db[k] = a * (1.0f - h * h);
    D2[(long long)r * 64 + k] = db[k];
  }
#pragma unroll
  for (int k = 0; k < 64; k++) {
    float a = 0.f;
#pragma unroll
    for (int j = 0; j < 64; j++) a = fmaf(s.w2[j * 64 + k], db[j], a);
    const float h = H1[(long long)r * 64 + k];
    D1[(long long)r * 64 + k] = a * (1.0f - h * h);
  }
}

// Weight and bias gradients of one layer, summed over the batch:
// dW[j][k] = sum_r D[r][j] Hin[r][k], db[j] = sum_r D[r][j].  Block: 256
// threads over (4 output rows) x (64 inputs); blockIdx.y = output-row group,
// blockIdx.x = slice of the batch (partial sums are added atomically).
__global__ void __launch_bounds__(256) mlp_train_wgrad(const float* __restrict__ D, int nout,
                                                       const float* __restrict__ Hin, int nin,
                                                       int n, int rows_per_slice,
                                                       float* __restrict__ gW, float* __restrict__ gb) {
  const int j = blockIdx.y * 4 + (threadIdx.x >> 6), k = threadIdx.x & 63;
  if (j >= nout) return;
  const int r0 = blockIdx.x * rows_per_slice, r1 = min(n, r0 + rows_per_slice);
  float aw = 0.f, ab = 0.f;
  for (int r = r0; r < r1; r++) {
    const float d = D[(long long)r * nout + j];
    if (k < nin) aw = fmaf(d, Hin[(long long)r * nin + k], aw);
    ab += d;
  }
  if (k < nin) atomicAdd(&gW[j * nin + k], aw);
  if (k == 0) atomicAdd(&gb[j], ab);
}

// Adam (Kingma & Ba 2015, Algorithm 1) on the trainable parameters.
__global__ void mlp_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                         float* __restrict__ v, int n, float lr, float c1, float c2) {
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = beta1 * m[k] + (1.0f - beta1) * gk;
    const float vk = beta2 * v[k] + (1.0f - beta2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    th[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);  // c1 = 1/(1-beta1^t), c2 = 1/(1-beta2^t)
  }
}

}  // namespace lbm
