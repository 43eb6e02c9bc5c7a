// lbm_device.cuh -- device side of the D3Q19 LBM-LES step for sm_103a.
//
// One thread updates one cell per tile; a persistent grid walks contiguous
// tile ranges.  Per cell (arxiv 2206.15454, Sec. 2 and Algorithm 1):
//   pull-stream 19 populations (boundaries fused into the source choice),
//   density and momentum (Eqs. density, momentum), the canopy drag
//   F = -C_D a(y) |u| u (Eq. forestForce) solved jointly with the half-force
//   velocity shift, equilibrium (Eq. local_eq), non-equilibrium flux
//   (Eq. tensor), Smagorinsky tau_total (Eqs. nu_t, strain, tau_total),
//   BGK relaxation (Eqs. lbe, bgk) plus Guo forcing (Eq. bodyforce), store.
// Populations live in HBM as offsets from the lattice weights, f_i - w_i, in
// the storage type; all arithmetic is FP32.  The path is HBM-bound (152 B or
// 76 B per lattice update); there is no contraction, so no tensor cores.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

// ---- D3Q19 lattice (public direction order, see include/lbm.h) -----------
constexpr int NQ = 19;
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
// opposite direction: the order pairs i (odd) with i + 1
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// direction with the y component flipped
__host__ __device__ constexpr int miry(int i) {
  return i == 3 ? 4 : i == 4 ? 3 : i == 7 ? 9 : i == 9 ? 7 : i == 8 ? 10 : i == 10 ? 8
       : i == 15 ? 18 : i == 18 ? 15 : i == 16 ? 17 : i == 17 ? 16 : i;
}
__host__ __device__ constexpr float wgt(int i) {
  return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr double wgt_d(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// ---- storage types ----------------------------------------------------------
template <int S> struct Store;
template <> struct Store<0> {
  using T = float;
  static __device__ __forceinline__ float ld(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(T* p, float v) { *p = v; }
  static __host__ __device__ __forceinline__ T from_double(double v) { return (float)v; }
};
template <> struct Store<1> {
  using T = __half;
  static __device__ __forceinline__ float ld(const T* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st(T* p, float v) { *p = __float2half_rn(v); }
  static __host__ __device__ __forceinline__ T from_double(double v) { return __double2half(v); }
};
template <> struct Store<2> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float ld(const T* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ void st(T* p, float v) { *p = __float2bfloat16_rn(v); }
  static __host__ __device__ __forceinline__ T from_double(double v) { return __double2bfloat16(v); }
};

// ---- device-resident controller / health state --------------------------------
struct DevState {
  unsigned int nan_flag;    // set when a cell produced a non-finite value
  unsigned int pad;
};

constexpr int MAX_BLOCKS = 4096;  // per-block bulk-velocity partials per slot

constexpr int MAX_XBINS = 64;

struct StepParams {
  const void* src;
  void* dst;
  int nx, ny, nz, pitch;
  long long plane;          // elements per population plane (ny*nz*pitch)
  long long qoff[NQ];       // q * plane: read from the parameter bank, not registers
  int x_io;                 // 1: inflow at x = 0, outflow at x = nx-1; 0: periodic
  int y_walls;              // 1: bounce-back bottom + `top` kind; 0: periodic
  int top;                  // 1 bounce-back, 2 free-slip, 3 equilibrium
  float tau0, c18;          // c18 = 18 sqrt(2) C_s^2
  float g[3];               // driving acceleration (g[0] replaced by the controller)
  int ctrl;                 // bulk-velocity controller on
  int have_prev;            // a previous step measured U_b
  double g0x, gain, u_target, inv_cells;
  double* ub_part;          // [2][MAX_BLOCKS] per-block sums of u_x, slot = step parity
  int slot_read, slot_write, nprev;  // nprev: blocks of the previous launch
  int canopy_x0, canopy_x1;
  const float* kdrag;       // ny values C_D a(y), or nullptr
  const float* feq_in;      // [ny][19] shifted f_eq(1, u_in(y)) (inflow), or nullptr
  float feq_top[NQ];        // shifted f_eq(1, u_top) (equilibrium top)
  // tiling: tile = (y, z-group, x-chunk); block = (tx, ry) threads
  int nxc, nzg;
  long long ntiles;
  // statistics
  double* stats;            // [9][nbins][ny] FP64 sums, or nullptr when off
  int nbins;
  DevState* state;
};

// Source coordinates of direction i for a cell at (x, y, z): the caller
// precomputes the per-axis neighbours once per cell.
struct Nbr {
  int xm, xp;   // source x for c_x = +1 (x-1) and c_x = -1 (x+1), after wrap/clamp
  int zm, zp;   // source z for c_z = +1 and -1 (periodic)
  int ym, yp;   // source y for c_y = +1 and -1 (periodic wrap or own row at walls)
  bool inflow;  // x == 0 with an inflow boundary
  bool lo_wall, hi_wall;
};

__device__ __forceinline__ Nbr neighbours(const StepParams& p, int x, int y, int z) {
  Nbr n;
  n.inflow = false;
  n.xm = x - 1;
  n.xp = x + 1;
  if (x == 0) {
    if (p.x_io) { n.xm = 0; n.inflow = true; } else { n.xm = p.nx - 1; }
  }
  if (x == p.nx - 1) n.xp = p.x_io ? p.nx - 1 : 0;   // outflow: zero-gradient copy
  n.zm = (z == 0) ? p.nz - 1 : z - 1;
  n.zp = (z == p.nz - 1) ? 0 : z + 1;
  n.ym = y - 1;
  n.yp = y + 1;
  n.lo_wall = n.hi_wall = false;
  if (y == 0) {
    if (p.y_walls) { n.ym = 0; n.lo_wall = true; } else { n.ym = p.ny - 1; }
  }
  if (y == p.ny - 1) {
    if (p.y_walls) { n.yp = y; n.hi_wall = true; } else { n.yp = 0; }
  }
  return n;
}

template <int I>
__device__ __forceinline__ int src_x(const Nbr& n, int x) { return cx(I) == 1 ? n.xm : cx(I) == -1 ? n.xp : x; }
template <int I>
__device__ __forceinline__ int src_y(const Nbr& n, int y) { return cy(I) == 1 ? n.ym : cy(I) == -1 ? n.yp : y; }
template <int I>
__device__ __forceinline__ int src_z(const Nbr& n, int z) { return cz(I) == 1 ? n.zm : cz(I) == -1 ? n.zp : z; }

template <int S, int I>
__device__ __forceinline__ float load_dir(const StepParams& p, const typename Store<S>::T* src,
                                          const Nbr& n, int x, int y, int z) {
  const int xs = src_x<I>(n, x), ys = src_y<I>(n, y), zs = src_z<I>(n, z);
  const long long idx = p.qoff[I] + (long long)((ys * p.nz + zs) * p.pitch + xs);
  return Store<S>::ld(src + idx);
}

template <int S, int I>
__device__ __forceinline__ void pull_one(const StepParams& p, const typename Store<S>::T* src,
                                         const Nbr& n, int x, int y, int z, float* f) {
  float v = load_dir<S, I>(p, src, n, x, y, z);
  // inflow: incoming populations at x = 0 are the inflow equilibrium
  if (cx(I) == 1 && n.inflow) v = p.feq_in[src_y<I>(n, y) * NQ + I];
  // bottom wall, halfway bounce-back: the population sent towards the wall returns
  if (cy(I) == 1 && n.lo_wall) {
    v = Store<S>::ld(src + p.qoff[opp(I)] + (long long)((y * p.nz + z) * p.pitch + x));
  }
  if (cy(I) == -1 && n.hi_wall) {
    if (p.top == 1) {
      v = Store<S>::ld(src + p.qoff[opp(I)] + (long long)((y * p.nz + z) * p.pitch + x));
    } else if (p.top == 2) {
      // free slip: the mirrored population of the upstream column in x and z
      constexpr int J = miry(I);
      const int xs = src_x<I>(n, x), zs = src_z<I>(n, z);
      v = Store<S>::ld(src + p.qoff[J] + (long long)((y * p.nz + zs) * p.pitch + xs));
      if (cx(I) == 1 && n.inflow) v = p.feq_in[y * NQ + J];
    } else {
      v = p.feq_top[I];
    }
  }
  f[I] = v;
}

template <int S, int I = 0>
__device__ __forceinline__ void pull_all(const StepParams& p, const typename Store<S>::T* src,
                                         const Nbr& n, int x, int y, int z, float* f) {
  if constexpr (I < NQ) {
    pull_one<S, I>(p, src, n, x, y, z, f);
    pull_all<S, I + 1>(p, src, n, x, y, z, f);
  }
}

// Moments, canopy-corrected velocity and total force density.
struct Macro {
  float drho, rho, ux, uy, uz, Fx, Fy, Fz;
};

__device__ __forceinline__ Macro moments(const float* f, float gx, float gy, float gz, float k) {
  Macro m;
  float drho = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
  for (int i = 0; i < NQ; i++) {
    drho += f[i];
    if (cx(i) == 1) mx += f[i];
    if (cx(i) == -1) mx -= f[i];
    if (cy(i) == 1) my += f[i];
    if (cy(i) == -1) my -= f[i];
    if (cz(i) == 1) mz += f[i];
    if (cz(i) == -1) mz -= f[i];
  }
  const float rho = 1.0f + drho;
  const float inv_rho = 1.0f / rho;
  // Eq. momentum: rho u = m + F/2 with the driving part of F ...
  float vx = (mx + 0.5f * rho * gx) * inv_rho;
  float vy = (my + 0.5f * rho * gy) * inv_rho;
  float vz = (mz + 0.5f * rho * gz) * inv_rho;
  float Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
  if (k > 0.f) {
    // ... and the canopy part g_c = -k |u| u: u = v + g_c/2 gives u parallel
    // to v with |u| the positive root of (k/2) s^2 + s = |v|.
    const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
    const float s = 2.0f / (1.0f + sqrtf(1.0f + 2.0f * k * vn));
    vx *= s; vy *= s; vz *= s;
    const float kun = k * s * vn;  // k |u|
    Fx -= rho * kun * vx;
    Fy -= rho * kun * vy;
    Fz -= rho * kun * vz;
  }
  m.drho = drho; m.rho = rho;
  m.ux = vx; m.uy = vy; m.uz = vz;
  m.Fx = Fx; m.Fy = Fy; m.Fz = Fz;
  return m;
}

// BGK-Smagorinsky collision with Guo forcing, in place on shifted populations.
// The equilibrium is evaluated twice (for Pi_neq, then for the relaxation)
// instead of being kept in 19 more registers.
__device__ __forceinline__ float feq_shifted(int i, const Macro& m, float uu) {
  const float cu = cx(i) * m.ux + cy(i) * m.uy + cz(i) * m.uz;
  // f_eq - w_i (Eq. local_eq with rho = 1 + drho)
  return wgt(i) * (m.drho + m.rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu));
}

__device__ __forceinline__ void collide(float* f, const Macro& m, float tau0, float c18) {
  const float ux = m.ux, uy = m.uy, uz = m.uz;
  const float uu = ux * ux + uy * uy + uz * uz;
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int i = 0; i < NQ; i++) {
    const float d = f[i] - feq_shifted(i, m, uu);
    if (cx(i) != 0) pxx += d;
    if (cy(i) != 0) pyy += d;
    if (cz(i) != 0) pzz += d;
    if (cx(i) * cy(i) == 1) pxy += d;
    if (cx(i) * cy(i) == -1) pxy -= d;
    if (cx(i) * cz(i) == 1) pxz += d;
    if (cx(i) * cz(i) == -1) pxz -= d;
    if (cy(i) * cz(i) == 1) pyz += d;
    if (cy(i) * cz(i) == -1) pyz -= d;
  }
  const float q2 = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
  const float tau = 0.5f * (tau0 + sqrtf(tau0 * tau0 + c18 * sqrtf(q2) / m.rho));
  const float om = 1.0f / tau;
  const float pre = 1.0f - 0.5f * om;
  const float uF = ux * m.Fx + uy * m.Fy + uz * m.Fz;
#pragma unroll
  for (int i = 0; i < NQ; i++) {
    const float cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
    const float cF = cx(i) * m.Fx + cy(i) * m.Fy + cz(i) * m.Fz;
    const float Fi = pre * wgt(i) * (3.0f * (cF - uF) + 9.0f * cu * cF);
    f[i] = f[i] - om * (f[i] - feq_shifted(i, m, uu)) + Fi;
  }
}

__device__ __forceinline__ float drag_factor(const StepParams& p, int x, int y) {
  if (p.kdrag == nullptr || x < p.canopy_x0 || x >= p.canopy_x1) return 0.f;
  return __ldg(p.kdrag + y);
}

// Controller input: the bulk velocity of the previous step, summed by one
// warp from that step's per-block partials in a fixed order (every block gets
// the same value, and reruns are bitwise reproducible).  Call with a full warp.
__device__ __forceinline__ double prev_bulk_velocity(const StepParams& p, int lane) {
  const double* part = p.ub_part + (long long)p.slot_read * MAX_BLOCKS;
  double s = 0.0;
  for (int k = lane; k < p.nprev; k += 32) s += part[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s * p.inv_cells;
}

__device__ __forceinline__ float controlled_gx(const StepParams& p, int lane) {
  if (!(p.ctrl && p.have_prev)) return p.g[0];
  return (float)(p.g0x + p.gain * (p.u_target - prev_bulk_velocity(p, lane)));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- the fused step -----------------------------------------------------------------
template <int S, bool STATS>
__global__ void __launch_bounds__(256) step_kernel(StepParams p) {
  using T = typename Store<S>::T;
  const T* __restrict__ src = static_cast<const T*>(p.src);
  T* __restrict__ dst = static_cast<T*>(p.dst);

  __shared__ float s_stats[9 * MAX_XBINS];
  __shared__ float s_ub[32];
  __shared__ float s_gx;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthreads = blockDim.x * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5;
  if (STATS) {
    for (int k = tid; k < 9 * p.nbins; k += nthreads) s_stats[k] = 0.f;
  }
  if (warp == 0) {
    const float v = controlled_gx(p, lane);
    if (lane == 0) s_gx = v;
  }
  __syncthreads();
  const float gx = s_gx, gy = p.g[1], gz = p.g[2];

  const long long t0 = (long long)blockIdx.x * p.ntiles / gridDim.x;
  const long long t1 = (long long)(blockIdx.x + 1) * p.ntiles / gridDim.x;
  // tile t -> (y, z-group, x-chunk), walked incrementally
  int xc = (int)(t0 % p.nxc);
  long long rest = t0 / p.nxc;
  int zg = (int)(rest % p.nzg);
  int y = (int)(rest / p.nzg);

  float ub_acc = 0.f;
  bool bad = false;

  for (long long t = t0; t < t1; t++) {
    const int x = xc * blockDim.x + threadIdx.x;
    const int z = zg * blockDim.y + threadIdx.y;
    const bool active = (x < p.nx) && (z < p.nz);
    float q[9];
    int bin = 0;
    if (active) {
      const Nbr n = neighbours(p, x, y, z);
      float f[NQ];
      pull_all<S>(p, src, n, x, y, z, f);
      const Macro m = moments(f, gx, gy, gz, drag_factor(p, x, y));
      collide(f, m, p.tau0, p.c18);
      const long long own = (long long)((y * p.nz + z) * p.pitch + x);
#pragma unroll
      for (int i = 0; i < NQ; i++) Store<S>::st(dst + p.qoff[i] + own, f[i]);
      ub_acc += m.ux;
      bad |= !(fabsf(m.drho) < 1e30f && fabsf(m.ux) + fabsf(m.uy) + fabsf(m.uz) < 1e30f);
      if (STATS) {
        q[0] = m.ux; q[1] = m.uy; q[2] = m.uz;
        q[3] = m.ux * m.ux; q[4] = m.uy * m.uy; q[5] = m.uz * m.uz;
        q[6] = m.ux * m.uy; q[7] = m.ux * m.uz; q[8] = m.uy * m.uz;
        bin = (int)(((long long)x * p.nbins) / p.nx);
      }
    } else if (STATS) {
#pragma unroll
      for (int k = 0; k < 9; k++) q[k] = 0.f;
      bin = -1;
    }
    if (STATS) {
      // warp-level reduction when the warp shares one x-bin, else per lane
      const unsigned act = __ballot_sync(0xffffffffu, bin >= 0);
      if (act) {
        const int b0 = __shfl_sync(0xffffffffu, bin, __ffs(act) - 1);
        const int key = bin >= 0 ? bin : b0;
        const unsigned same = __match_any_sync(0xffffffffu, key);
        if (same == 0xffffffffu) {
#pragma unroll
          for (int k = 0; k < 9; k++) {
            const float v = warp_sum(q[k]);
            if (lane == 0) atomicAdd(&s_stats[k * p.nbins + key], v);
          }
        } else if (bin >= 0) {
#pragma unroll
          for (int k = 0; k < 9; k++) atomicAdd(&s_stats[k * p.nbins + bin], q[k]);
        }
      }
    }
    // advance to the next tile; flush the plane statistics when y changes
    const int y_now = y;
    if (++xc == p.nxc) {
      xc = 0;
      if (++zg == p.nzg) { zg = 0; ++y; }
    }
    if (STATS && (y != y_now || t + 1 == t1)) {
      __syncthreads();
      for (int k = tid; k < 9 * p.nbins; k += nthreads) {
        const float v = s_stats[k];
        if (v != 0.f) {
          const int qk = k / p.nbins, b = k - qk * p.nbins;
          atomicAdd(&p.stats[((long long)qk * p.nbins + b) * p.ny + y_now], (double)v);
        }
        s_stats[k] = 0.f;
      }
      __syncthreads();
    }
  }

  if (bad) atomicOr(&p.state->nan_flag, 1u);
  // bulk velocity of this step (read by the controller of the next step)
  const float w = warp_sum(ub_acc);
  if (lane == 0) s_ub[warp] = w;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int k = 0; k < (nthreads + 31) / 32; k++) s += (double)s_ub[k];
    p.ub_part[(long long)p.slot_write * MAX_BLOCKS + blockIdx.x] = s;
  }
}

// ---- initialisation: f = f_eq(1, u0) with seeded perturbations ----------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
  // n-th output of SplitMix64 (Steele, Lea & Flood 2014) seeded with `seed`
  uint64_t z = seed + (n + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ double uniform_pm1(uint64_t seed, uint64_t n) {
  return 2.0 * ((double)(splitmix64(seed, n) >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

struct InitParams {
  void* f;
  int nx, ny, nz, pitch;
  long long plane;
  const double* u_prof;  // ny values or nullptr
  uint64_t seed;
  double amp;
};

template <int S>
__global__ void init_kernel(InitParams p) {
  using T = typename Store<S>::T;
  T* f = static_cast<T*>(p.f);
  const long long n = (long long)p.nx * p.ny * p.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % p.nx);
    const long long r = c / p.nx;
    const int y = (int)(r % p.ny);
    const int z = (int)(r / p.ny);
    double u[3] = {p.u_prof ? p.u_prof[y] : 0.0, 0.0, 0.0};
    for (int a = 0; a < 3; a++) u[a] += p.amp * uniform_pm1(p.seed, 3ull * (uint64_t)c + a);
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const long long own = (long long)((y * p.nz + z) * p.pitch + x);
#pragma unroll
    for (int i = 0; i < NQ; i++) {
      const double cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
      const double fs = wgt_d(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);  // f_eq(1,u) - w_i
      f[(long long)i * p.plane + own] = Store<S>::from_double(fs);
    }
  }
}

// ---- global mass: deterministic two-pass FP64 reduction ------------------------------
template <int S>
__global__ void mass_partial_kernel(const void* fv, int nx, int pitch, long long rows, long long plane,
                                    double* partial) {
  using T = typename Store<S>::T;
  const T* f = static_cast<const T*>(fv);
  double acc = 0.0;
  const long long per_plane = rows * nx;
  const long long total = per_plane * NQ;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long q = k / per_plane, rem = k - q * per_plane;
    const long long row = rem / nx, x = rem - row * nx;
    acc += (double)Store<S>::ld(f + q * plane + row * pitch + x);
  }
  __shared__ double s[256];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void mass_final_kernel(const double* partial, int n, double base, double* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < n; k++) s += partial[k];
    *out = base + s;
  }
}

// ---- macroscopic fields of the next step (pull + moments only) ------------------------
template <int S>
__global__ void macro_kernel(StepParams p, float* out) {
  using T = typename Store<S>::T;
  const T* src = static_cast<const T*>(p.src);
  const long long n = (long long)p.nx * p.ny * p.nz;
  const float gx = controlled_gx(p, threadIdx.x & 31);  // blockDim.x is a multiple of 32
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % p.nx);
    const long long r = c / p.nx;
    const int y = (int)(r % p.ny);
    const int z = (int)(r / p.ny);
    const Nbr nb = neighbours(p, x, y, z);
    float f[NQ];
    pull_all<S>(p, src, nb, x, y, z, f);
    const Macro m = moments(f, gx, p.g[1], p.g[2], drag_factor(p, x, y));
    out[c] = m.rho;
    out[n + c] = m.ux;
    out[2 * n + c] = m.uy;
    out[3 * n + c] = m.uz;
  }
}

}  // namespace lbm
