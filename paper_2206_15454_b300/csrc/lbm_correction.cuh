// lbm_correction.cuh -- the learned first-layer correction after a step, in
// one pass: the column features of the new state and the network on them.
// (The paper has no learned component; the correction and its inputs are
// described in lbm_mlp.cuh.)
#pragma once

#include "lbm_features.cuh"
#include "lbm_mlp_net.cuh"

namespace lbm {

// One warp per 16 first-cell columns (c = z nx + x): its lanes gather the 48
// cells (y = 0, 1, 2 of each column; one cell per lane and round) and compute
// their features (column_features' arithmetic) into shared memory, the
// standardised BF16 rows go to the warp's input tile, and the network writes
// the layer-0 acceleration a = (lam du_x - dtau_x, lam du_z - dtau_z) of each
// column.  The features never leave the SM: the network sees exactly the
// values features_kernel would have written (the same FP32 arithmetic), so
// the field equals that of the network on lbm_features' output.
template <int XT, int S>
__global__ void __launch_bounds__(128, 5) correction_kernel(StepParams p, const float* __restrict__ th,
                                                            float lam, float2* __restrict__ accel) {
  __shared__ MlpSmem s;
  __shared__ __align__(16) __nv_bfloat16 xin[4][16 * 16];
  __shared__ float feat[4][16][MLP_IN];
  mlp_stage(s, th);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float gx = controlled_gx(p, lane);
  const long long ncol = (long long)p.nx * p.nz;
  const long long tiles = (ncol + 15) / 16;
  for (long long tile = (long long)blockIdx.x * 4 + warp; tile < tiles; tile += (long long)gridDim.x * 4) {
    __syncwarp();
    for (int j = lane; j < 48; j += 32) {
      const int k = j & 15, y = j >> 4;
      const long long c = tile * 16 + k;
      if (c >= ncol) continue;
      const int x = (int)(c % p.nx), z = (int)(c / p.nx);
      const int yy = min(y, p.ny - 1);
      float f[NQ];
      gather_cell<XT, S>(p, x, yy, z, f);
      const Macro m = moments<true>(f, gx, p.g[1], p.g[2], drag_factor(p, x, yy), p.drag_x_only);
      feat[warp][k][y] = m.ux;
      feat[warp][k][3 + y] = strain_rate(f, m, p.tau0, p.c18, p.edm, p.tau_rho2);
      feat[warp][k][6 + y] = (p.lad != nullptr && x >= p.canopy_x0 && x < p.canopy_x1) ? p.lad[yy] : 0.f;
    }
    __syncwarp();
    if (lane < 16) {
      const long long r = tile * 16 + lane;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const float v = (r < ncol && k < MLP_IN) ? (feat[warp][lane][k] - s.xm[k]) * s.xinv[k] : 0.f;
        xin[warp][lane * 16 + k] = __float2bfloat16_rn(v);
      }
    }
    __syncwarp();
    float o[4], r0[4], r1[4];
    mlp_rows16(s, xin[warp], lane, o);
    mlp_gather_outputs(s, o, lane, r0, r1);
    if ((lane & 3) == 0) {
      const long long ra = tile * 16 + (lane >> 2), rb = ra + 8;
      if (ra < ncol) accel[ra] = make_float2(lam * r0[0] - r0[2], lam * r0[1] - r0[3]);
      if (rb < ncol) accel[rb] = make_float2(lam * r1[0] - r1[2], lam * r1[1] - r1[3]);
    }
  }
}

}  // namespace lbm
