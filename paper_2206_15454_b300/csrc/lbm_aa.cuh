// lbm_aa.cuh -- AA-pattern in-place storage: one population set instead of
// the two of the pull scheme (the "double-population" storage of Sec. 3),
// with the same bytes moved per lattice update.
//
// The set has a ghost layer one cell wide on every side.  Let f*_i(x) be the
// post-collision population of direction i at cell x (the state of the pull
// scheme).  After an even number of steps the set holds it "swapped", in slot
// opp(i) of its own cell; after an odd number "streamed", in slot i of cell
// x + c_i (a ghost cell when x + c_i lies outside).  The two kinds of step
// alternate:
//   B (from swapped):  f_i(x) = slot opp(i) at x - c_i, collide, f*_i(x) -> slot i at x + c_i
//   A (from streamed): f_i(x) = slot i at x,            collide, f*_i(x) -> slot opp(i) at x
// Every location is read and written by the same thread, so the update is in
// place.  Neither step applies a boundary condition: before each step a fill
// kernel writes exactly the slots whose upstream cell x - c_i lies outside the
// domain (ghost slots before B, the cell's own slots before A) with the value
// the pull scheme's streaming gives (row_source / source_x: periodic wrap,
// bounce-back, free slip, equilibrium top, inflow, outflow).  (Reading those
// values in place inside the step was tried: the boundary cells' dependent
// loads made their rows, which a static split gives to few blocks, set the
// step's duration.)  The collision is the pull kernel's (moments_v / collide_v).
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// Element of direction q at cell (x, y, z), x in [-1, nx], y in [-1, ny],
// z in [-1, nz]: planes [q][z + 1][y + 1], rows of `aa_pitch` elements with
// cell x at row start + x; the left ghost of a row is the last element of the
// previous row (aa_pitch >= nx + 2), `aa_lead` elements precede row 0.
__host__ __device__ __forceinline__ long long aa_index(const StepParams& p, int q, int x, int y,
                                                       int z) {
  return p.aa_lead + (((long long)q * (p.nz + 2) + (z + 1)) * (p.ny + 2) + (y + 1)) * p.aa_pitch + x;
}

// The post-collision value f*_q at interior cell (x, y, z) in the current layout.
// (A plain, coherent load: the fill kernel writes the same set.)
template <int S>
__device__ __forceinline__ float aa_post(const StepParams& p, int q, int x, int y, int z) {
  using T = typename Store<S>::T;
  const T* f = static_cast<const T*>(p.src);
  const long long k = p.aa_parity == 0 ? aa_index(p, opp(q), x, y, z)
                                       : aa_index(p, q, x + cx(q), y + cy(q), z + cz(q));
  if (kCheckBounds && !in_range(k, 1, p.aa_elems, p.state)) return 0.f;
  return Store<S>::to_float(f[k]);
}

// The population i streaming into interior cell (x, y, z) for the next step
// (shifted by the weight), by the pull scheme's boundary rules.
template <int S>
__device__ __forceinline__ float aa_pull(const StepParams& p, int i, int x, int y, int z) {
  int q, ys, zs;
  const int kind = row_source(p, i, cy(i), cz(i), y, z, q, ys, zs);
  if (kind == SRC_CONST) return p.feq_top[i];
  if (kind == SRC_OWN_X) return aa_post<S>(p, q, x, ys, zs);
  const int xs = source_x(p, x, cx(i));
  // the inflow equilibrium as the pull scheme's inflow ghost slot holds it:
  // rounded to the storage type
  if (xs < 0) return Store<S>::to_float(Store<S>::from_double((double)p.feq_in[ys * NQ + q]));
  return aa_post<S>(p, q, xs, ys, zs);
}

// The five directions entering through a face: face 0/1: x = 0 / nx - 1
// (c_x = +1 / -1), 2/3: y = 0 / ny - 1, 4/5: z = 0 / nz - 1; d = 0..4.
__device__ __forceinline__ int aa_inward(int face, int d) {
  const int axis = face >> 1, sign = (face & 1) ? -1 : 1;
  int n = 0;
#pragma unroll
  for (int i = 1; i < NQ; i++) {
    const int c = axis == 0 ? cx(i) : axis == 1 ? cy(i) : cz(i);
    if (c == sign) {
      if (n == d) return i;
      n++;
    }
  }
  return 0;
}

// Boundary fill before a step: for every cell X of the domain's faces and
// every direction i entering through that face (its upstream cell X - c_i
// lies outside), aa_pull's value goes to the slot the step reads it from:
// ghost slot opp(i) at X - c_i before B, slot i at X before A.  Stored, the
// inflow value is rounded to the storage type as in the pull scheme's ghost
// slot.  One thread per (face cell, direction), so the loads of the fill are
// all in flight at once; a cell on an edge or corner is reached through
// several faces and writes the same value each time.  The fill reads only
// slots whose upstream cell is inside, which no fill writes.
// Grid: blockIdx.z = 5 face + d (30 slices, face and direction uniform per
// block); the face's two coordinates (a fast, b slow) come from the block
// and thread indices, a over x (y on the x faces), b over z (y on the z
// faces), so no index is decoded by division; grid-stride loops cover faces
// larger than the grid (aa_fill_grid).
template <int S>
__global__ void aa_fill_kernel(StepParams p) {
  using T = typename Store<S>::T;
  T* f = static_cast<T*>(p.dst);
  const int face = (int)blockIdx.z / 5, d = (int)blockIdx.z - 5 * face;
  const int na = face < 2 ? p.ny : p.nx, nb = face < 4 ? p.nz : p.ny;
  const int i = aa_inward(face, d);
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous step has completed
  for (int b = blockIdx.y; b < nb; b += gridDim.y) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x) {
      int x, y, z;
      if (face < 2) {
        x = face ? p.nx - 1 : 0;
        y = a;
        z = b;
      } else if (face < 4) {
        x = a;
        y = face == 3 ? p.ny - 1 : 0;
        z = b;
      } else {
        x = a;
        y = b;
        z = face == 5 ? p.nz - 1 : 0;
      }
      const float v = aa_pull<S>(p, i, x, y, z);
      const long long at = p.aa_parity == 0 ? aa_index(p, opp(i), x - cx(i), y - cy(i), z - cz(i))
                                            : aa_index(p, i, x, y, z);
      if (!kCheckBounds || in_range(at, 1, p.aa_elems, p.state)) Store<S>::st(f + at, v);
    }
  }
}

// Launch shape of aa_fill_kernel: 256 threads along the fast coordinate
// (x, or y on the x faces), one block row per slow coordinate up to the
// grid's y limit, 30 face-direction slices.
inline dim3 aa_fill_grid(int nx, int ny, int nz) {
  const int na = nx > ny ? nx : ny, nb = nz > ny ? nz : ny;
  return dim3((unsigned)((na + 255) / 256), (unsigned)(nb < 65535 ? nb : 65535), 30u);
}

// Per-launch element offsets of the 19 reads and the 19 writes relative to
// the cell's slot of direction 0 (computed on the host for the step kind).
struct AAStep {
  StepParams p;
  long long rd[NQ], wr[NQ];
  // units: 128 x-cells x 2 z-rows at one y, numbered (y, z-group, x-chunk),
  // or with x-binned statistics over several chunks (y, x-chunk, z-group), so
  // consecutive units of a block share their x-bins and flush less often
  int nunit, nxc, nzg, xc_outer;
};

constexpr int AA_XT = 128, AA_ZR = 2;

// One AA step (B or A, by the offsets) of the model-variant form (the default
// model steps the AA layout on the pull scheme's tile pipeline, step_kernel
// with AK >= 0): block b takes the units [b U / G, (b + 1) U / G); one
// thread per cell; plane statistics kept in registers while the unit's row
// and x-bin stay the same.
template <int S, bool STATS, bool VAR>
__global__ void __launch_bounds__(AA_XT * AA_ZR, 3) aa_step_kernel(AAStep a) {
  using T = typename Store<S>::T;
  const StepParams& p = a.p;
  T* const f = static_cast<T*>(p.dst);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int lane = (ty * AA_XT + tx) & 31;
  __shared__ float s_gx;
  // launched as a programmatic dependent of the fill (and the fill of the
  // previous step): wait for it before touching memory
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (tx < 32 && ty == 0) {
    // bulk velocity of the previous step (exact fixed-point sum) for the controller;
    // block 0 clears the slot the next step accumulates into
    float g = p.g[0];
    if (p.ctrl && p.have_prev)
      g = (float)(p.g0x + p.gain * (p.u_target - (double)p.ub_part[p.slot_read] *
                                                     (1.0 / 4294967296.0) * p.inv_cells));
    if (tx == 0) {
      s_gx = g;
      if (blockIdx.x == 0) p.ub_part[(p.slot_write + 1) % 3] = 0;
    }
  }
  __syncthreads();
  const float gx = s_gx, gy = p.g[1], gz = p.g[2];
  const long long u0 = (long long)blockIdx.x * a.nunit / gridDim.x;
  const long long u1 = (long long)(blockIdx.x + 1) * a.nunit / gridDim.x;
  float q[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  int qy = -1, qbin = -1;  // row and x-bin the sums belong to
  long long ub_fix = 0;
  bool bad = false;
  auto flush = [&]() {
    const unsigned act = __ballot_sync(0xffffffffu, qbin >= 0);
    if (act) {
      const int b0 = __shfl_sync(0xffffffffu, qbin, __ffs(act) - 1);
      const long long m = (long long)p.nbins * p.ny;
      if (__all_sync(0xffffffffu, qbin < 0 || qbin == b0)) {
        const int yy = __shfl_sync(0xffffffffu, qy, __ffs(act) - 1);
#pragma unroll
        for (int k = 0; k < 9; k++) {
          const float v = warp_sum(q[k]);
          if (lane == 0) atomicAdd(p.stats + k * m + (long long)b0 * p.ny + yy, (double)v);
        }
      } else if (qbin >= 0) {
#pragma unroll
        for (int k = 0; k < 9; k++) atomicAdd(p.stats + k * m + (long long)qbin * p.ny + qy, (double)q[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 9; k++) q[k] = 0.f;
    qbin = -1;
  };
  for (long long u = u0; u < u1; u++) {
    int xc, zg, y;
    if (a.xc_outer) {
      zg = (int)(u % a.nzg);
      const long long r = u / a.nzg;
      xc = (int)(r % a.nxc);
      y = (int)(r / a.nxc);
    } else {
      xc = (int)(u % a.nxc);
      const long long r = u / a.nxc;
      zg = (int)(r % a.nzg);
      y = (int)(r / a.nzg);
    }
    const int x = xc * AA_XT + tx, z = zg * AA_ZR + ty;
    const bool active = x < p.nx && z < p.nz;
    const int bin = active ? (int)(((long long)x * p.nbins) / p.nx) : -1;
    if (STATS && (y != qy || __any_sync(0xffffffffu, qbin >= 0 && bin != qbin))) {
      flush();
      qy = y;
    }
    if (active) {
      const long long c0 = aa_index(p, 0, x, y, z);
      T* const cell = f + c0;
      float fi[NQ];
#pragma unroll
      for (int i = 0; i < NQ; i++) {  // plain loads: in place
        if (kCheckBounds && !in_range(c0 + a.rd[i], 1, p.aa_elems, p.state)) { fi[i] = 0.f; continue; }
        fi[i] = Store<S>::to_float(cell[a.rd[i]]);
      }
      const float kd = drag_factor(p, x, y);
      auto put = [&](int i, float v) {
        if (!kCheckBounds || in_range(c0 + a.wr[i], 1, p.aa_elems, p.state)) Store<S>::st(cell + a.wr[i], v);
      };
      Macro m;
      if (VAR) {
        m = moments<VAR>(fi, gx, gy, gz, kd, p.drag_x_only);
        collide<VAR>(fi, m, p.tau0, p.c18, p.edm, p.tau_rho2, put);
      } else {  // the default model: the same arithmetic as the pull kernel
        const MacroV<float> mv = moments_v<float>(fi, gx, gy, gz, kd, kd > 0.f, p.tau0, p.c18);
        collide_v<float>(fi, mv, put);
        m = Macro{mv.drho, mv.rho, mv.ux, mv.uy, mv.uz, mv.Fx, mv.Fy, mv.Fz};
      }
      ub_fix += __float2ll_rn(m.ux * 4294967296.0f);
      bad |= !(fabsf(m.drho) < 1e30f);
      if (STATS) {
        q[0] += m.ux; q[1] += m.uy; q[2] += m.uz;
        q[3] += m.ux * m.ux; q[4] += m.uy * m.uy; q[5] += m.uz * m.uz;
        q[6] += m.ux * m.uy; q[7] += m.ux * m.uz; q[8] += m.uy * m.uz;
        qbin = bin;
      }
    }
  }
  if (STATS) flush();
  if (bad) atomicOr(&p.state->nan_flag, 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ub_fix += __shfl_xor_sync(0xffffffffu, ub_fix, o);
  if (lane == 0 && ub_fix != 0)
    atomicAdd(reinterpret_cast<unsigned long long*>(p.ub_part + p.slot_write),
              (unsigned long long)ub_fix);
}

// f = f_eq(1, u0) with the seeded perturbations (as init_kernel), written in
// the swapped layout (no step done).
template <int S>
__global__ void aa_init_kernel(StepParams p, InitParams ip) {
  using T = typename Store<S>::T;
  T* f = static_cast<T*>(p.dst);
  const long long n = (long long)p.nx * p.ny * p.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % p.nx);
    const long long r = c / p.nx;
    const int y = (int)(r % p.ny);
    const int z = (int)(r / p.ny);
    double u[3] = {ip.u_prof ? ip.u_prof[y] : 0.0, 0.0, 0.0};
    for (int a = 0; a < 3; a++) u[a] += ip.amp * uniform_pm1(ip.seed, 3ull * (uint64_t)c + a);
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int i = 0; i < NQ; i++) {
      const double cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
      const long long k = aa_index(p, opp(i), x, y, z);
      if (!kCheckBounds || in_range(k, 1, p.aa_elems, p.state))
        f[k] = Store<S>::from_double(wgt_d(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
    }
  }
}

// Global mass, first pass: sums of the post-collision offsets per block.
template <int S>
__global__ void aa_mass_partial_kernel(StepParams p, double* partial) {
  const long long n = (long long)p.nx * p.ny * p.nz * NQ;
  double acc = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(k % NQ);
    const long long c = k / NQ;
    const int x = (int)(c % p.nx);
    const long long r = c / p.nx;
    acc += (double)aa_post<S>(p, q, x, (int)(r % p.ny), (int)(r / p.ny));
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

// Density and velocity the next step computes (the read-out of macro_kernel).
template <int S, class OutT>
__global__ void aa_macro_kernel(StepParams p, OutT* out) {
  const long long n = (long long)p.nx * p.ny * p.nz;
  // the driving acceleration the next step uses: from the one exact sum of
  // the one-cell AA kernel, or from the tile pipeline's per-block partials
  float gx = p.aa_ub_sum ? p.g[0] : controlled_gx(p, threadIdx.x & 31);
  if (p.aa_ub_sum && p.ctrl && p.have_prev)
    gx = (float)(p.g0x + p.gain * (p.u_target - (double)p.ub_part[p.slot_read] *
                                                    (1.0 / 4294967296.0) * p.inv_cells));
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % p.nx);
    const long long r = c / p.nx;
    const int y = (int)(r % p.ny);
    const int z = (int)(r / p.ny);
    float f[NQ];
#pragma unroll
    for (int i = 0; i < NQ; i++) f[i] = aa_pull<S>(p, i, x, y, z);
    const Macro m = moments<true>(f, gx, p.g[1], p.g[2], drag_factor(p, x, y), p.drag_x_only);
    out[c] = m.rho;
    out[n + c] = m.ux;
    out[2 * n + c] = m.uy;
    out[3 * n + c] = m.uz;
  }
}

}  // namespace lbm
