// lbm_features.cuh -- inputs of the learned first-layer correction: the
// column features of the domain state (templates over chunk width and
// storage; the network itself is in lbm_mlp.cuh).
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr int MLP_IN = 9, MLP_OUT = 4;  // network inputs and outputs per first-cell column
// Layout of the network's flat parameter vector (FP32, rows = outputs,
// row-major): W1[64][9] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64]
// b4[4], then x_mean[9] x_std[9] y_mean[4] y_std[4].
constexpr int MLP_H = 64;
constexpr int OFF_W1 = 0, OFF_B1 = 576, OFF_W2 = 640, OFF_B2 = 4736, OFF_W3 = 4800, OFF_B3 = 8896,
              OFF_W4 = 8960, OFF_B4 = 9216;
constexpr int MLP_NW = 9220;  // trainable parameters
constexpr int OFF_XM = 9220, OFF_XS = 9229, OFF_YM = 9238, OFF_YS = 9242;
constexpr int MLP_NP = 9246;  // with the normalisation

// Column features of the domain state (the inputs the correction sees):
// u_x, |S| and the leaf-area density at y = 0, 1, 2 of column (x, z).
template <int XT, int S>
__device__ __forceinline__ void column_features(const StepParams& p, float gx, int x, int z,
                                                float (&feat)[MLP_IN]) {
#pragma unroll
  for (int y = 0; y < 3; y++) {
    const int yy = min(y, p.ny - 1);
    float f[NQ];
    gather_cell<XT, S>(p, x, yy, z, f);
    const float k = drag_factor(p, x, yy);
    const Macro m = moments<true>(f, gx, p.g[1], p.g[2], k, p.drag_x_only);
    feat[y] = m.ux;
    feat[3 + y] = strain_rate(f, m, p.tau0, p.c18, p.edm, p.tau_rho2);
    feat[6 + y] = (p.lad != nullptr && x >= p.canopy_x0 && x < p.canopy_x1) ? p.lad[yy] : 0.f;
  }
}

// Column features of the whole first layer: X[c][9] for c = z * nx + x.
template <int XT, int S>
__global__ void __launch_bounds__(256) features_kernel(StepParams p, float* __restrict__ X) {
  const float gx = controlled_gx(p, threadIdx.x & 31);  // blockDim.x is a multiple of 32
  const long long ncol = (long long)p.nx * p.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncol;
       c += (long long)gridDim.x * blockDim.x) {
    float feat[MLP_IN];
    column_features<XT, S>(p, gx, (int)(c % p.nx), (int)(c / p.nx), feat);
#pragma unroll
    for (int k = 0; k < MLP_IN; k++) X[c * MLP_IN + k] = feat[k];
  }
}

}  // namespace lbm
