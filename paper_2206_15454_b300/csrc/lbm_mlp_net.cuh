// lbm_mlp_net.cuh -- the correction network's forward pass on the tensor
// cores (device functions only, so the per-storage translation units that run
// it beside the column features can include it): weights staged in shared
// memory as BF16, mma.sync m16n8k16 with FP32 accumulators, one warp per 16
// rows with the activations kept in registers between layers.
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
// outputs to 8 (padding zero).  Rows are MLP_WPAD elements longer than their
// inputs, so the eight rows a warp's B fragments read (one per lane group)
// fall in different banks: with rows 128 bytes apart every fragment load was
// an 8-way bank conflict.
constexpr int MLP_WPAD = 8;
struct MlpSmem {
  __nv_bfloat16 w1[64 * (16 + MLP_WPAD)];
  __nv_bfloat16 w2[64 * (64 + MLP_WPAD)];
  __nv_bfloat16 w3[64 * (64 + MLP_WPAD)];
  __nv_bfloat16 w4[8 * (64 + MLP_WPAD)];
  float b1[64], b2[64], b3[64], b4[8];
  float xm[16], xinv[16], ym[4], ys[4];
};

__device__ __forceinline__ void mlp_stage(MlpSmem& s, const float* __restrict__ th) {
  constexpr int R1 = 16 + MLP_WPAD, R = 64 + MLP_WPAD;  // row strides
  for (int k = threadIdx.x; k < 64 * R1; k += blockDim.x) {
    const int o = k / R1, i = k % R1;
    s.w1[k] = __float2bfloat16_rn(i < MLP_IN ? th[OFF_W1 + o * MLP_IN + i] : 0.f);
  }
  for (int k = threadIdx.x; k < 64 * R; k += blockDim.x) {
    const int o = k / R, i = k % R;
    s.w2[k] = __float2bfloat16_rn(i < 64 ? th[OFF_W2 + o * 64 + i] : 0.f);
    s.w3[k] = __float2bfloat16_rn(i < 64 ? th[OFF_W3 + o * 64 + i] : 0.f);
  }
  for (int k = threadIdx.x; k < 8 * R; k += blockDim.x) {
    const int o = k / R, i = k % R;
    s.w4[k] = __float2bfloat16_rn(o < 4 && i < 64 ? th[OFF_W4 + o * 64 + i] : 0.f);
  }
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
    const __nv_bfloat16* wr = w + (8 * j + g) * (K + MLP_WPAD) + 2 * t;  // W[n = 8j + g][k]
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
  const __nv_bfloat16* wr = s.w4 + g * (64 + MLP_WPAD) + 2 * t;
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

}  // namespace lbm
