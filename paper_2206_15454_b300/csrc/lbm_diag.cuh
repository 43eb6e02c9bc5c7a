// lbm_diag.cuh -- diagnostic read-outs computed from the macroscopic fields
// (not part of the time step).
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// ---- Q-criterion of the velocity field (diagnostic read-out) --------------------------
// Vortical structures are shown as iso-surfaces of Q (Sec. 4) = (|Omega|^2 - |S|^2) / 2,
// S and Omega the symmetric and antisymmetric parts of the velocity gradient
// G_ab = d u_a / d x_b; with both written out, Q = -(1/2) sum_ab G_ab G_ba.  G
// by central differences of the cell velocities (u: [3][z][y][x]), wrapping
// periodic directions, one-sided at the first and last cell of a bounded one,
// zero across a direction one cell wide.  One thread per cell.
struct Diff {
  int m, p;   // neighbours (cell indices along the direction)
  float s;    // 1/2 for a central difference, 1 for a one-sided one, 0 if none
};
__device__ __forceinline__ Diff diff_along(int i, int n, bool periodic) {
  if (n == 1) return {i, i, 0.f};
  if (periodic) return {i == 0 ? n - 1 : i - 1, i == n - 1 ? 0 : i + 1, 0.5f};
  if (i == 0) return {0, 1, 1.f};
  if (i == n - 1) return {n - 2, n - 1, 1.f};
  return {i - 1, i + 1, 0.5f};
}

__global__ void q_kernel(const float* __restrict__ u, float* __restrict__ q, int nx, int ny, int nz,
                         int x_periodic, int y_periodic) {
  const long long n = (long long)nx * ny * nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx);
    const long long r = c / nx;
    const int y = (int)(r % ny);
    const int z = (int)(r / ny);
    const Diff dx = diff_along(x, nx, x_periodic != 0), dy = diff_along(y, ny, y_periodic != 0),
               dz = diff_along(z, nz, true);
    const long long row = (long long)z * ny + y;
    const long long xm = row * nx + dx.m, xp = row * nx + dx.p;
    const long long ym = ((long long)z * ny + dy.m) * nx + x, yp = ((long long)z * ny + dy.p) * nx + x;
    const long long zm = ((long long)dz.m * ny + y) * nx + x, zp = ((long long)dz.p * ny + y) * nx + x;
    float G[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const float* ua = u + a * n;
      G[a][0] = (ua[xp] - ua[xm]) * dx.s;
      G[a][1] = (ua[yp] - ua[ym]) * dy.s;
      G[a][2] = (ua[zp] - ua[zm]) * dz.s;
    }
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) acc += G[a][b] * G[b][a];
    q[c] = -0.5f * acc;
  }
}

// Second pass of the global mass (lbm_mass): the per-block partial sums in a
// fixed order, plus the lattice-weight part of every cell (base = cells).
__global__ void mass_final_kernel(const double* partial, int n, double base, double* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < n; k++) s += partial[k];
    *out = base + s;
  }
}

// The pipelined statistics read-out (lbm_stats_begin): n16 16-byte words of
// the plane sums and health flags (adjacent in the workspace) into a slot of
// the context's pinned host buffer, through its mapped device address.  It
// runs as a programmatic dependent of the step before it and lets the next
// step's launch proceed from its start, so consecutive steps keep their
// programmatic overlap (an asynchronous copy between two steps broke it).
__global__ void readout_kernel(const uint4* __restrict__ src, uint4* dst, long long n16) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the step before has completed
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n16;
       k += (long long)gridDim.x * blockDim.x)
    dst[k] = src[k];
  __threadfence_system();
}

}  // namespace lbm
