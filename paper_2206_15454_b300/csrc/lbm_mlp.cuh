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

#include "lbm_mlp_net.cuh"

namespace lbm {


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
