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
#include <climits>
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
// ld2 / st2: two adjacent values at a 4-byte aligned address (16-bit types:
// one 32-bit access), rounded to nearest like st.
template <> struct Store<0> {
  using T = float;
  static __device__ __forceinline__ float ld(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ float to_float(T v) { return v; }
  static __device__ __forceinline__ void st(T* p, float v) { *p = v; }
  static __host__ __device__ __forceinline__ T from_double(double v) { return (float)v; }
  static __device__ __forceinline__ float2 ld2(const T* p) { return make_float2(p[0], p[1]); }
  static __device__ __forceinline__ void st2(T* p, float2 v) { p[0] = v.x; p[1] = v.y; }
};
template <> struct Store<1> {
  using T = __half;
  static __device__ __forceinline__ float ld(const T* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ float to_float(T v) { return __half2float(v); }
  static __device__ __forceinline__ void st(T* p, float v) { *p = __float2half_rn(v); }
  static __host__ __device__ __forceinline__ T from_double(double v) { return __double2half(v); }
  static __device__ __forceinline__ float2 ld2(const T* p) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
  }
  static __device__ __forceinline__ void st2(T* p, float2 v) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.x, v.y);
  }
  // the two values of a packed word (low half first); unpack2_again is the
  // same conversion, written so the compiler does not merge it with an earlier
  // unpack2 of the same word (the collision converts again rather than keep
  // 19 more registers alive)
  static __device__ __forceinline__ float2 unpack2(uint32_t r) {
    float2 v;
    asm("{.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;}"
        : "=f"(v.x), "=f"(v.y) : "r"(r));
    return v;
  }
  static __device__ __forceinline__ float2 unpack2_again(uint32_t r) {
    float2 v;
    asm volatile("{.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;}"
                 : "=f"(v.x), "=f"(v.y) : "r"(r));
    return v;
  }
};
template <> struct Store<2> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float ld(const T* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ float to_float(T v) { return __bfloat162float(v); }
  static __device__ __forceinline__ void st(T* p, float v) { *p = __float2bfloat16_rn(v); }
  static __host__ __device__ __forceinline__ T from_double(double v) { return __double2bfloat16(v); }
  static __device__ __forceinline__ float2 ld2(const T* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  }
  static __device__ __forceinline__ void st2(T* p, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.x, v.y);
  }
  // a BF16 value is the high half of the FP32 value with the same bits
  static __device__ __forceinline__ float2 unpack2(uint32_t r) {
    return make_float2(__uint_as_float(r << 16), __uint_as_float(r & 0xffff0000u));
  }
  static __device__ __forceinline__ float2 unpack2_again(uint32_t r) {
    uint32_t lo, hi;
    asm volatile("{\n\tshl.b32 %0, %2, 16;\n\tand.b32 %1, %2, 0xffff0000;\n\t}" : "=r"(lo), "=r"(hi) : "r"(r));
    return make_float2(__uint_as_float(lo), __uint_as_float(hi));
  }
};

// ---- device-resident controller / health state --------------------------------
struct DevState {
  unsigned int nan_flag;      // set when a cell produced a non-finite value
  unsigned int timeout_flag;  // set when a bounded device wait gave up
  unsigned int tile_ctr[2];   // dynamic tile counters, one per step parity
  unsigned int bounds_flag;   // checked builds (LBM_CHECK_BOUNDS): an index left its buffer
  unsigned int pad[3];
};

// Checked builds verify every bulk copy and every global store of the step
// against the buffer it addresses; a violation sets bounds_flag and skips the
// access (a skipped copy leaves its stage's wait to run out).  Off by default.
#ifdef LBM_CHECK_BOUNDS
constexpr bool kCheckBounds = true;
#else
constexpr bool kCheckBounds = false;
#endif
__device__ __forceinline__ bool in_range(long long lo, long long len, long long size,
                                         DevState* st) {
  if (lo >= 0 && len >= 0 && lo + len <= size) return true;
  atomicOr(&st->bounds_flag, 1u);
  return false;
}

constexpr int MAX_BLOCKS = 4096;  // per-block bulk-velocity partials per slot
// threads per block of the step kernels for cpt cells per thread (a tile is
// that many threads' cells; three blocks of 256 threads fit an SM).  Six
// blocks of 128 threads (one tile row) for two cells per thread measured the
// same within 1 % (B300: channel FP16 0.0926 -> 0.0941 ms, canopy FP16 0.3355
// -> 0.3332 ms).
__host__ __device__ constexpr int block_threads(int cpt) { return cpt > 0 ? 256 : 256; }
constexpr int MAX_XBINS = 64;

// ---- population layout in HBM ------------------------------------------------------
// One population set is f[y][z][xc][q][XTP]: rows are cut into chunks of XT
// cells (XT = 64, 128 or 256) and a chunk-row (y, z, xc) holds the 19
// direction rows of the chunk back to back, each XTP = XT + 2G elements with
// G one 128-byte line: cell x = xc*XT + tx sits in slot G + tx, on whole lines.
// Slot G-1 holds, for the directions with c_x = +1, the value of the column
// left of the chunk (previous chunk, periodic wrap, or the inflow
// equilibrium); slot G + n (n = cells of the chunk) holds, for c_x = -1, the
// column right of it (next chunk, periodic wrap, or a zero-gradient copy at
// an outflow).  Cells on chunk edges refresh these ghost slots when they
// store, so a tile's sources are exactly its staged rows: a direction row is
// copied with the one ghost its c_x reads.
template <int XT, int S>
struct Geo {
  using T = typename Store<S>::T;
  static constexpr int G = 128 / (int)sizeof(T);
  static constexpr int XTP = XT + 2 * G;
  static constexpr int ROW = NQ * XTP;  // elements per chunk-row
};

struct StepParams {
  const void* src;
  void* dst;
  int nx, ny, nz, nxc;      // nxc chunks of XT cells per row
  int x_io;                 // x boundary mode: X_PERIODIC, X_INOUT or X_HALO
  int io_one;               // X_INOUT with a last chunk of one cell
  int y_walls;              // 1: bounce-back bottom + `top` kind; 0: periodic
  int top;                  // 1 bounce-back, 2 free-slip, 3 equilibrium
  float tau0, c18;          // c18 = 18 sqrt(2) C_s^2
  float g[3];               // driving acceleration (g[0] replaced by the controller)
  int ctrl;                 // bulk-velocity controller on
  int have_prev;            // a previous step measured U_b
  double g0x, gain, u_target, inv_cells;
  long long* ub_part;       // [2][MAX_BLOCKS] per-block sums of u_x in 2^-32 fixed point, slot = step parity
  int slot_read, slot_write, nprev;  // nprev: blocks of the previous launch
  int canopy_x0, canopy_x1;
  const float* kdrag;       // ny values C_D a(y), or nullptr
  const float* lad;         // ny values a(y), or nullptr (inputs of the learned correction)
  const float* feq_in;      // [ny][19] shifted f_eq(1, u_in(y)) for the inflow column
  float feq_top[NQ];        // shifted f_eq(1, u_top) (equilibrium top)
  // tiling: tile = (y, z-group, x-chunk), block = (XT, ry) threads; tiles
  // are numbered y-major, then z-group, then chunk, or with x-binned
  // statistics over several chunks then chunk, then z-group (consecutive
  // tiles of a block then share their x-bins, so its statistics sums are
  // flushed when the chunk changes, not at every tile)
  int nzg;
  int xc_outer;
  int t_in, t_mid, t_fast;  // tile-number radices (chunks / z-groups); t_fast: ntiles < 2^23
  float t_in_inv, t_mid_inv;
  long long ntiles;
  int nstage;               // tiles in flight per block
  int withhold;             // >= 0: block 0 never issues this fill (test of the timeout path)
  // work split of one domain: block b first walks the static run of tiles
  // [b * static_tiles, (b + 1) * static_tiles), then takes tiles one by one
  // from [gridDim.x * static_tiles, ntiles) through tile_ctr[ctr_slot]
  int static_tiles;
  int ctr_slot;
  // statistics
  double* stats;            // [9][nbins][ny] FP64 sums
  int nbins;
  int bins_even;            // x-bins of one even width: cells x, x + 1 (x even) share their bin
  DevState* state;
  // learned first-layer correction: extra (x, z) acceleration of the cells at
  // y = 0, per column [z][x], or nullptr
  const float2* accel0;
  // model variants (read only by the variant form of the step kernel and by
  // the read-outs): canopy drag on the streamwise component only (Eq.
  // forestForce as worded), exact-difference forcing instead of Guo's (Eq.
  // bodyforce), Q^1/2 / rho^2 under the root of tau_total (the tau_total
  // equation as printed) instead of / rho (Eq. strain solved for tau)
  int drag_x_only, edm, tau_rho2;
  // AA-pattern storage (one population set, lbm_aa.cuh): row pitch and lead
  // of the set in elements, and the layout of the current state (0 swapped,
  // after an even number of steps; 1 streamed)
  long long aa_pitch, aa_lead, aa_elems;  // aa_elems: elements of the set (checked builds)
  int aa_parity;
  long long aa_wr[NQ];  // the step's write offsets of direction i from the cell's slot of direction 0
  int aa_ub_sum;        // the bulk-velocity sum is one exact sum per step in three slots (one-cell AA kernel)
};

// x boundary modes of StepParams::x_io
enum : int { X_PERIODIC = 0, X_INOUT = 1, X_HALO = 2 };

// element index of population q at cell (x, y, z)
template <int XT, int S>
__device__ __forceinline__ long long pop_index(const StepParams& p, int q, int x, int y, int z) {
  return ((long long)((y * p.nz + z) * p.nxc + x / XT) * NQ + q) * Geo<XT, S>::XTP + Geo<XT, S>::G +
         x % XT;
}

// Source of direction i for a cell at row (y, z): plane q, row (ys, zs), and
// how it enters: shifted in x by -c_x (streaming), taken from the own column
// (halfway bounce-back), or a constant (equilibrium top).  Streaming with the
// y boundaries of Algorithm 1's "stream" step.
enum : int { SRC_SHIFT = 0, SRC_OWN_X = 1, SRC_CONST = 2 };

__device__ __forceinline__ int row_source(const StepParams& p, int i, int dy, int dz, int y, int z,
                                          int& q, int& ys, int& zs) {
  q = i;
  ys = y - dy;
  zs = z - dz;
  if (zs < 0) zs += p.nz;
  if (zs >= p.nz) zs -= p.nz;
  if (ys < 0 || ys >= p.ny) {
    if (!p.y_walls) {
      ys = ys < 0 ? ys + p.ny : ys - p.ny;
    } else if (ys < 0 || p.top == 1) {
      q = (i == 0) ? 0 : ((i & 1) ? i + 1 : i - 1);  // bounce-back: own cell, reversed
      ys = y;
      zs = z;
      return SRC_OWN_X;
    } else if (p.top == 2) {
      q = miry(i);  // free slip: mirrored, upstream in x and z
      ys = y;
    } else {
      return SRC_CONST;  // equilibrium top
    }
  }
  return SRC_SHIFT;
}

// Source column of a shifted direction: x - c_x with periodic wrap, the
// inflow column (x = -1: returns -1), or the outflow copy (clamped).
// At an x-halo face the column outside (-1 or nx) is returned: its values sit
// in the ghost slots the halo exchange filled.
__device__ __forceinline__ int source_x(const StepParams& p, int x, int dx) {
  int xs = x - dx;
  if (p.x_io == X_HALO) return xs;
  if (xs < 0) xs = p.x_io == X_INOUT ? -1 : p.nx - 1;
  if (xs >= p.nx) xs = p.x_io == X_INOUT ? p.nx - 1 : 0;
  return xs;
}

struct Macro {
  float drho, rho, ux, uy, uz, Fx, Fy, Fz;
};

// Directions come in pairs (i, i+1) with c_{i+1} = -c_i (i odd).  Pair sums
// and differences give the moments with half the additions.  VAR: the model
// variants may be on (drag_x_only: the drag acts on u_x alone).
template <bool VAR = false>
__device__ __forceinline__ Macro moments(const float* f, float gx, float gy, float gz, float k,
                                         int drag_x_only = 0) {
  Macro m;
  float sm[NQ], df[NQ];
#pragma unroll
  for (int i = 1; i < NQ; i += 2) {
    sm[i] = f[i] + f[i + 1];
    df[i] = f[i] - f[i + 1];
  }
  float drho = f[0];
#pragma unroll
  for (int i = 1; i < NQ; i += 2) drho += sm[i];
  float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
  for (int i = 1; i < NQ; i += 2) {
    if (cx(i) == 1) mx += df[i];
    if (cx(i) == -1) mx -= df[i];
    if (cy(i) == 1) my += df[i];
    if (cy(i) == -1) my -= df[i];
    if (cz(i) == 1) mz += df[i];
    if (cz(i) == -1) mz -= df[i];
  }
  const float rho = 1.0f + drho;
  const float inv_rho = 1.0f / rho;
  // Eq. momentum: rho u = m + F/2 with the driving part of F ...
  float vx = (mx + 0.5f * rho * gx) * inv_rho;
  float vy = (my + 0.5f * rho * gy) * inv_rho;
  float vz = (mz + 0.5f * rho * gz) * inv_rho;
  float Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
  if (VAR && drag_x_only && k > 0.f) {
    // ... and a streamwise canopy drag g_c = (-k |u| u_x, 0, 0): u_y = v_y,
    // u_z = v_z, and u_x solves u_x (1 + (k/2) |u|) = v_x with
    // |u|^2 = u_x^2 + v_y^2 + v_z^2 (monotone in u_x).  Newton from the
    // vector-drag root, which is within O((k|v|)^2) of it: two steps reach
    // FP32 rounding for k|v| << 1.
    const float s2 = vy * vy + vz * vz;
    float ux = vx * (2.0f / (1.0f + sqrtf(1.0f + 2.0f * k * sqrtf(vx * vx + s2))));
#pragma unroll
    for (int it = 0; it < 2; it++) {
      const float r = sqrtf(ux * ux + s2);
      const float phi = ux + 0.5f * k * ux * r - vx;
      const float dphi = 1.0f + 0.5f * k * (r + (r > 0.f ? ux * ux / r : 0.f));
      ux -= phi / dphi;
    }
    vx = ux;
    Fx -= rho * k * sqrtf(ux * ux + s2) * ux;
  } else if (k > 0.f) {
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

// BGK-Smagorinsky collision with Guo forcing on shifted populations, written
// per pair (i, i+1): with e = c_i . u and h = c_i . F,
//   f_eq - w = W (drho + rho (4.5 e^2 - 1.5 u.u)) +- 3 W rho e      (Eq. local_eq)
//   F_i      = (1 - om/2) W (9 e h - 3 u.F)      +- 3 (1 - om/2) W h (Eq. bodyforce)
// so the even and odd parts are evaluated once per pair.  Pi_neq (Eq. tensor)
// needs only the pair sums of f - f_eq.  The post-collision values
// f* = f - om (f - f_eq) + F_i are handed to `emit(i, value)`.  VAR: the
// variants may be on (tau_rho2: Q^1/2 / rho^2 under the root of tau_total;
// edm: the exact-difference forcing of collide_edm).
template <class Emit>
__device__ __forceinline__ void collide_edm(const float* f, const Macro& m, float tau0, float c18,
                                            int tau_rho2, Emit&& emit);

template <bool VAR = false, class Emit>
__device__ __forceinline__ void collide(const float* f, const Macro& m, float tau0, float c18,
                                        int edm, int tau_rho2, Emit&& emit) {
  if (VAR && edm) {
    collide_edm(f, m, tau0, c18, tau_rho2, emit);
    return;
  }
  const float ux = m.ux, uy = m.uy, uz = m.uz;
  const float uu = ux * ux + uy * uy + uz * uz;
  const float base = m.drho - 1.5f * m.rho * uu;  // even part without the e^2 term
  const float r45 = 4.5f * m.rho;
  const float r3 = 3.0f * m.rho;
  float sym[NQ];
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int i = 1; i < NQ; i += 2) {
    const float w = wgt(i);
    float ei;
    if (i == 1) ei = ux; else if (i == 3) ei = uy; else if (i == 5) ei = uz;
    else if (i == 7) ei = ux + uy; else if (i == 9) ei = ux - uy;
    else if (i == 11) ei = ux + uz; else if (i == 13) ei = ux - uz;
    else if (i == 15) ei = uy + uz; else ei = uy - uz;
    sym[i] = w * (base + r45 * ei * ei);
    const float npair = (f[i] + f[i + 1]) - 2.0f * sym[i];  // sum over the pair of f - f_eq
    if (cx(i) != 0) pxx += npair;
    if (cy(i) != 0) pyy += npair;
    if (cz(i) != 0) pzz += npair;
    if (cx(i) * cy(i) == 1) pxy += npair;
    if (cx(i) * cy(i) == -1) pxy -= npair;
    if (cx(i) * cz(i) == 1) pxz += npair;
    if (cx(i) * cz(i) == -1) pxz -= npair;
    if (cy(i) * cz(i) == 1) pyz += npair;
    if (cy(i) * cz(i) == -1) pyz -= npair;
  }
  const float q2 = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
  const float rr = (VAR && tau_rho2) ? m.rho * m.rho : m.rho;
  const float tau = 0.5f * (tau0 + sqrtf(tau0 * tau0 + c18 * sqrtf(q2) / rr));
  const float om = 1.0f / tau;
  const float keep = 1.0f - om;
  const float pre = 1.0f - 0.5f * om;
  const float uF3 = 3.0f * (ux * m.Fx + uy * m.Fy + uz * m.Fz);
  // rest population: e = h = 0
  {
    const float w = wgt(0);
    const float feq0 = w * base;
    emit(0, keep * f[0] + om * feq0 - pre * w * uF3);
  }
#pragma unroll
  for (int i = 1; i < NQ; i += 2) {
    const float w = wgt(i);
    float ei, hi;
    if (i == 1) { ei = ux; hi = m.Fx; } else if (i == 3) { ei = uy; hi = m.Fy; }
    else if (i == 5) { ei = uz; hi = m.Fz; }
    else if (i == 7) { ei = ux + uy; hi = m.Fx + m.Fy; }
    else if (i == 9) { ei = ux - uy; hi = m.Fx - m.Fy; }
    else if (i == 11) { ei = ux + uz; hi = m.Fx + m.Fz; }
    else if (i == 13) { ei = ux - uz; hi = m.Fx - m.Fz; }
    else if (i == 15) { ei = uy + uz; hi = m.Fy + m.Fz; }
    else { ei = uy - uz; hi = m.Fy - m.Fz; }
    const float pw = pre * w;
    const float even = om * sym[i] + pw * (9.0f * ei * hi - uF3);
    const float odd = om * (w * r3 * ei) + 3.0f * pw * hi;
    emit(i, keep * f[i] + (even + odd));
    emit(i + 1, keep * f[i + 1] + (even - odd));
  }
}

// Exact-difference forcing (Kupershtokh): relaxation towards f_eq(rho, u_b)
// at the bare velocity u_b = m/rho = u - g/2 (u the force-corrected velocity
// of `m`, g = F/rho the total acceleration), and the force term
// F_i = f_eq(rho, u_b + g) - f_eq(rho, u_b).  With e = c_i . u_b, h = c_i . g:
//   F_i = W rho (4.5 h (2e + h) - 3 u_b.g - 1.5 g.g) +- 3 W rho h,
// even and odd parts per pair as in collide().  Pi_neq and tau_total use the
// same f_eq(rho, u_b).
template <class Emit>
__device__ __forceinline__ void collide_edm(const float* f, const Macro& m, float tau0, float c18,
                                            int tau_rho2, Emit&& emit) {
  const float inv_rho = 1.0f / m.rho;
  const float gx = m.Fx * inv_rho, gy = m.Fy * inv_rho, gz = m.Fz * inv_rho;
  const float ux = m.ux - 0.5f * gx, uy = m.uy - 0.5f * gy, uz = m.uz - 0.5f * gz;
  const float uu = ux * ux + uy * uy + uz * uz;
  const float base = m.drho - 1.5f * m.rho * uu;
  const float r45 = 4.5f * m.rho;
  const float r3 = 3.0f * m.rho;
  float sym[NQ];
  float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
  for (int i = 1; i < NQ; i += 2) {
    const float ei = cx(i) * ux + cy(i) * uy + cz(i) * uz;
    sym[i] = wgt(i) * (base + r45 * ei * ei);
    const float npair = (f[i] + f[i + 1]) - 2.0f * sym[i];
    if (cx(i) != 0) pxx += npair;
    if (cy(i) != 0) pyy += npair;
    if (cz(i) != 0) pzz += npair;
    pxy += (float)(cx(i) * cy(i)) * npair;
    pxz += (float)(cx(i) * cz(i)) * npair;
    pyz += (float)(cy(i) * cz(i)) * npair;
  }
  const float q2 = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
  const float rr = tau_rho2 ? m.rho * m.rho : m.rho;
  const float tau = 0.5f * (tau0 + sqrtf(tau0 * tau0 + c18 * sqrtf(q2) / rr));
  const float om = 1.0f / tau;
  const float keep = 1.0f - om;
  const float ug = 3.0f * (ux * gx + uy * gy + uz * gz) + 1.5f * (gx * gx + gy * gy + gz * gz);
  emit(0, keep * f[0] + om * (wgt(0) * base) - wgt(0) * m.rho * ug);
#pragma unroll
  for (int i = 1; i < NQ; i += 2) {
    const float w = wgt(i);
    const float ei = cx(i) * ux + cy(i) * uy + cz(i) * uz;
    const float hi = cx(i) * gx + cy(i) * gy + cz(i) * gz;
    const float even = om * sym[i] + w * m.rho * (4.5f * hi * (2.0f * ei + hi) - ug);
    const float odd = om * (w * r3 * ei) + w * r3 * hi;
    emit(i, keep * f[i] + (even + odd));
    emit(i + 1, keep * f[i + 1] + (even - odd));
  }
}

// ---- the default model's collision on one cell (float) or two (float2) ---------------
// Written once with explicit round-to-nearest operations (no contraction left
// to the compiler), so one cell per thread (scalar instructions) and two cells
// per thread (packed FP32x2 instructions: FFMA2, FADD2, FMUL2) give
// bit-identical results.  Division and square root are the same per-component
// approximations (-prec-div=false, -prec-sqrt=false) in both.
template <class V>
struct VOps;
template <>
struct VOps<float> {
  static __device__ __forceinline__ float c(float a) { return a; }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float d) { return __fmaf_rn(a, b, d); }
  static __device__ __forceinline__ float neg(float a) { return -a; }
  static __device__ __forceinline__ float div(float a, float b) { return a / b; }
  static __device__ __forceinline__ float sqrt(float a) { return sqrtf(a); }
  // a where k > 0, else b
  static __device__ __forceinline__ float where_pos(float k, float a, float b) { return k > 0.f ? a : b; }
};
template <>
struct VOps<float2> {
  static __device__ __forceinline__ float2 c(float a) { return make_float2(a, a); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  // one packed subtraction (rounded like add(a, -b))
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a)),
          "l"(*reinterpret_cast<const unsigned long long*>(&b)));
    return *reinterpret_cast<const float2*>(&d);
  }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 d) { return __ffma2_rn(a, b, d); }
  static __device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
  static __device__ __forceinline__ float2 div(float2 a, float2 b) { return make_float2(a.x / b.x, a.y / b.y); }
  static __device__ __forceinline__ float2 sqrt(float2 a) { return make_float2(sqrtf(a.x), sqrtf(a.y)); }
  static __device__ __forceinline__ float2 where_pos(float2 k, float2 a, float2 b) {
    return make_float2(k.x > 0.f ? a.x : b.x, k.y > 0.f ? a.y : b.y);
  }
};

template <class V>
struct MacroV {
  V drho, rho, ux, uy, uz, Fx, Fy, Fz;
  V om;  // 1 / tau_total
};

// Eqs. density and momentum with the driving acceleration and the canopy
// drag solved jointly (as moments()).  k: C_D a(y) per cell; a cell with
// k = 0 keeps u and F as without drag (selected, so two cells side by side
// give what each gives alone).  fg(i) gives f_i - w_i.  Also the relaxation
// rate 1/tau_total (Eqs. nu_t, strain, tau_total) from Pi_neq (Eq. tensor),
// which follows from the second moments S of f - w (the same pair sums): the
// second moment of the D3Q19 equilibrium is rho c_s^2 I + rho u u exactly
// (the lattice is isotropic to fourth order) and sum_i c_i c_i w_i = c_s^2 I,
// so Pi_neq = sum_i c_i c_i (f_i - f_eq_i) = S - c_s^2 drho I - rho u u.
template <class V, class Get>
__device__ __forceinline__ MacroV<V> moments_g(Get&& fg, V gx, V gy, V gz, V k, bool any_drag,
                                               float tau0, float c18) {
  using O = VOps<V>;
  V sm[NQ], df[NQ];
#pragma unroll
  for (int i = 1; i < NQ; i += 2) {
    const V a = fg(i), b = fg(i + 1);
    sm[i] = O::add(a, b);
    df[i] = O::sub(a, b);
  }
  V drho = fg(0);
#pragma unroll
  for (int i = 1; i < NQ; i += 2) drho = O::add(drho, sm[i]);
  // odd directions 1 (+x), 3 (+y), 5 (+z), 7 (+x+y), 9 (+x-y), 11 (+x+z),
  // 13 (+x-z), 15 (+y+z), 17 (+y-z)
  const V mx = O::add(O::add(O::add(O::add(df[1], df[7]), df[9]), df[11]), df[13]);
  const V my = O::add(O::add(O::sub(O::add(df[3], df[7]), df[9]), df[15]), df[17]);
  const V mz = O::sub(O::add(O::sub(O::add(df[5], df[11]), df[13]), df[15]), df[17]);
  const V sxx = O::add(O::add(O::add(O::add(sm[1], sm[7]), sm[9]), sm[11]), sm[13]);
  const V syy = O::add(O::add(O::add(O::add(sm[3], sm[7]), sm[9]), sm[15]), sm[17]);
  const V szz = O::add(O::add(O::add(O::add(sm[5], sm[11]), sm[13]), sm[15]), sm[17]);
  const V sxy = O::sub(sm[7], sm[9]);
  const V sxz = O::sub(sm[11], sm[13]);
  const V syz = O::sub(sm[15], sm[17]);
  MacroV<V> m;
  m.drho = drho;
  m.rho = O::add(O::c(1.0f), drho);
  const V inv_rho = O::div(O::c(1.0f), m.rho);
  const V hr = O::mul(O::c(0.5f), m.rho);
  V vx = O::mul(O::fma(hr, gx, mx), inv_rho);
  V vy = O::mul(O::fma(hr, gy, my), inv_rho);
  V vz = O::mul(O::fma(hr, gz, mz), inv_rho);
  m.Fx = O::mul(m.rho, gx);
  m.Fy = O::mul(m.rho, gy);
  m.Fz = O::mul(m.rho, gz);
  if (any_drag) {
    // g_c = -k |u| u with u = v + g_c/2: u parallel to v, |u| = s |v|,
    // s = 2 / (1 + sqrt(1 + 2 k |v|)) (s = 1 where k = 0)
    const V vn = O::sqrt(O::fma(vx, vx, O::fma(vy, vy, O::mul(vz, vz))));
    const V s = O::div(O::c(2.0f), O::add(O::c(1.0f), O::sqrt(O::fma(O::mul(O::c(2.0f), k), vn, O::c(1.0f)))));
    const V ux = O::mul(vx, s), uy = O::mul(vy, s), uz = O::mul(vz, s);
    const V rk = O::mul(O::mul(O::c(-1.0f), m.rho), O::mul(O::mul(k, s), vn));  // -rho k |u|
    m.Fx = O::where_pos(k, O::fma(rk, ux, m.Fx), m.Fx);
    m.Fy = O::where_pos(k, O::fma(rk, uy, m.Fy), m.Fy);
    m.Fz = O::where_pos(k, O::fma(rk, uz, m.Fz), m.Fz);
    vx = O::where_pos(k, ux, vx);
    vy = O::where_pos(k, uy, vy);
    vz = O::where_pos(k, uz, vz);
  }
  m.ux = vx;
  m.uy = vy;
  m.uz = vz;
  const V nr = O::mul(O::c(-1.0f), m.rho);
  const V nrux = O::mul(nr, vx), nruy = O::mul(nr, vy);
  const V d3 = O::mul(O::c(1.0f / 3.0f), drho);
  const V pxx = O::fma(nrux, vx, O::sub(sxx, d3));
  const V pyy = O::fma(nruy, vy, O::sub(syy, d3));
  const V pzz = O::fma(O::mul(nr, vz), vz, O::sub(szz, d3));
  const V pxy = O::fma(nrux, vy, sxy);
  const V pxz = O::fma(nrux, vz, sxz);
  const V pyz = O::fma(nruy, vz, syz);
  const V off = O::fma(pxy, pxy, O::fma(pxz, pxz, O::mul(pyz, pyz)));
  const V q2 = O::fma(pxx, pxx, O::fma(pyy, pyy, O::fma(pzz, pzz, O::mul(O::c(2.0f), off))));
  // tau_total = (tau0 + sqrt(arg)) / 2, so 1/tau_total = 2 / (tau0 + sqrt(arg))
  const V arg = O::fma(O::mul(O::c(c18), O::sqrt(q2)), inv_rho, O::c(tau0 * tau0));
  m.om = O::div(O::c(2.0f), O::add(O::c(tau0), O::sqrt(arg)));
  return m;
}

template <class V>
__device__ __forceinline__ MacroV<V> moments_v(const V* f, V gx, V gy, V gz, V k, bool any_drag,
                                               float tau0, float c18) {
  return moments_g<V>([&](int i) { return f[i]; }, gx, gy, gz, k, any_drag, tau0, c18);
}

// BGK-Smagorinsky collision with Guo forcing (as collide()), per pair
// (i, i+1) from the even and odd parts of f_eq and of the forcing term.
// c_i . a for the odd direction i of a pair, from the components of a
template <class V>
__device__ __forceinline__ V pair_dot(int i, V ax, V ay, V az) {
  using O = VOps<V>;
  return i == 1 ? ax : i == 3 ? ay : i == 5 ? az : i == 7 ? O::add(ax, ay) : i == 9 ? O::sub(ax, ay)
       : i == 11 ? O::add(ax, az) : i == 13 ? O::sub(ax, az) : i == 15 ? O::add(ay, az)
       : O::sub(ay, az);
}

// Relaxation (Eqs. lbe, bgk) at the rate m.om of moments_g, plus Guo's
// forcing term; fg(i) gives f_i - w_i again.
template <class V, class Get, class Emit>
__device__ __forceinline__ void collide_g(Get&& fg, const MacroV<V>& m, Emit&& emit) {
  using O = VOps<V>;
  const V ux = m.ux, uy = m.uy, uz = m.uz;
  const V uu = O::fma(ux, ux, O::fma(uy, uy, O::mul(uz, uz)));
  const V base = O::fma(O::mul(O::c(-1.5f), m.rho), uu, m.drho);  // drho - 1.5 rho u.u
  const V r45 = O::mul(O::c(4.5f), m.rho);
  const V r3 = O::mul(O::c(3.0f), m.rho);
  const V om = m.om;
  const V keep = O::sub(O::c(1.0f), om);
  const V pre = O::fma(O::c(-0.5f), om, O::c(1.0f));
  const V nuF3 = O::mul(O::c(-3.0f), O::fma(ux, m.Fx, O::fma(uy, m.Fy, O::mul(uz, m.Fz))));  // -3 u.F
  {
    const V pw = O::mul(pre, O::c(wgt(0)));
    emit(0, O::fma(keep, fg(0), O::fma(om, O::mul(O::c(wgt(0)), base), O::mul(pw, nuF3))));
  }
#pragma unroll
  for (int i = 1; i < NQ; i += 2) {
    const V e = pair_dot<V>(i, ux, uy, uz);
    const V h = pair_dot<V>(i, m.Fx, m.Fy, m.Fz);
    const V sym = O::mul(O::c(wgt(i)), O::fma(O::mul(r45, e), e, base));  // even part of f_eq - w
    const V pw = O::mul(pre, O::c(wgt(i)));
    const V even = O::fma(om, sym, O::mul(pw, O::fma(O::mul(O::c(9.0f), e), h, nuF3)));
    const V odd = O::fma(om, O::mul(O::mul(O::c(wgt(i)), r3), e), O::mul(O::mul(O::c(3.0f), pw), h));
    emit(i, O::fma(keep, fg(i), O::add(even, odd)));
    emit(i + 1, O::fma(keep, fg(i + 1), O::sub(even, odd)));
  }
}

template <class V, class Emit>
__device__ __forceinline__ void collide_v(const V* f, const MacroV<V>& m, Emit&& emit) {
  collide_g<V>([&](int i) { return f[i]; }, m, emit);
}

__device__ __forceinline__ float drag_factor(const StepParams& p, int x, int y) {
  if (p.kdrag == nullptr || x < p.canopy_x0 || x >= p.canopy_x1) return 0.f;
  return __ldg(p.kdrag + y);
}

// Controller input: the bulk velocity of the previous step, summed by one
// warp from that step's per-block partials.  Every cell adds its u_x in
// 2^-32 fixed point, so the integer sums are exact whichever block handled
// which tile: every block gets the same value and reruns are bitwise
// reproducible.  Call with a full warp.
__device__ __forceinline__ double prev_bulk_velocity(const StepParams& p, int lane) {
  const long long* part = p.ub_part + (long long)p.slot_read * MAX_BLOCKS;
  long long s = 0;
  for (int k = lane; k < p.nprev; k += 32) s += part[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return (double)s * (1.0 / 4294967296.0) * p.inv_cells;
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

// Plane statistics of one warp: its lanes' sums for row y (taken from the
// shared-memory slots `qs`, stride NT (threads per block), and cleared) are added to the FP64
// accumulators, one warp-reduced add per quantity when the lanes share an
// x-bin, else one add per lane.  Called by every lane; no block barrier.
template <int NT>
__device__ __forceinline__ void flush_warp_stats(const StepParams& p, float* qs, int& last_x, int y,
                                                 int lane) {
  float q[9];
#pragma unroll
  for (int k = 0; k < 9; k++) {
    q[k] = qs[k * NT];
    qs[k * NT] = 0.f;
  }
  const int bin = last_x >= 0 ? (int)(((long long)last_x * p.nbins) / p.nx) : -1;
  const unsigned act = __ballot_sync(0xffffffffu, bin >= 0);
  if (act) {
    const int b0 = __shfl_sync(0xffffffffu, bin, __ffs(act) - 1);
    const long long m = (long long)p.nbins * p.ny;
    double* acc = p.stats + (long long)y;
    if (__all_sync(0xffffffffu, bin < 0 || bin == b0)) {
#pragma unroll
      for (int k = 0; k < 9; k++) {
        const float v = warp_sum(q[k]);
        if (lane == 0) atomicAdd(acc + k * m + (long long)b0 * p.ny, (double)v);
      }
    } else if (bin >= 0) {
#pragma unroll
      for (int k = 0; k < 9; k++) atomicAdd(acc + k * m + (long long)bin * p.ny, (double)q[k]);
    }
  }
  last_x = -1;
}

// Step epilogue: health flags and this block's share of the bulk velocity
// (exact integer sum of the fixed-point cell values).
__device__ __forceinline__ void finish_step(const StepParams& p, long long ub_fix, bool bad,
                                            bool late, long long* s_ub, int lane, int warp,
                                            int tid, int nthreads, int part) {
  if (bad) atomicOr(&p.state->nan_flag, 1u);
  if (late) atomicOr(&p.state->timeout_flag, 1u);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ub_fix += __shfl_xor_sync(0xffffffffu, ub_fix, o);
  if (lane == 0) s_ub[warp] = ub_fix;
  __syncthreads();
  if (tid == 0 && part >= 0) {
    long long sum = 0;
    for (int kk = 0; kk < (nthreads + 31) / 32; kk++) sum += s_ub[kk];
    p.ub_part[(long long)p.slot_write * MAX_BLOCKS + part] = sum;
  }
}

struct TileGeom {
  int xc, zg, y;
};

// tiles number fewer than cells (< 2^31): 32-bit arithmetic
// t / n for t < 2^23 from a float reciprocal: the rounded quotient is off by
// at most one, which the remainder corrects.
__device__ __forceinline__ unsigned div_small(unsigned t, unsigned n, float inv) {
  unsigned q = __float2uint_rz(__uint2float_rn(t) * inv);
  const int r = (int)(t - q * n);
  return r < 0 ? q - 1 : (r >= (int)n ? q + 1 : q);
}

__device__ __forceinline__ TileGeom tile_geom(const StepParams& p, long long t) {
  TileGeom g;
  // t = (y * n_mid + mid) * n_in + in, (in, mid) = (chunk, z-group) or swapped
  const unsigned tt = (unsigned)t, n_in = p.t_in, n_mid = p.t_mid;
  unsigned r, y;
  if (p.t_fast) {
    r = div_small(tt, n_in, p.t_in_inv);
    y = div_small(r, n_mid, p.t_mid_inv);
  } else {
    r = tt / n_in;
    y = r / n_mid;
  }
  const int in = (int)(tt - r * n_in), mid = (int)(r - y * n_mid);
  g.xc = p.xc_outer ? mid : in;
  g.zg = p.xc_outer ? in : mid;
  g.y = (int)y;
  return g;
}

// ---- TMA bulk copies and mbarriers --------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// bulk copy global -> shared: 16-byte aligned addresses, size a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// one test of the phase with the given parity (may suspend the thread briefly)
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait for the phase with the given parity; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t k = 0; k < limit; k++)
    if (mbar_try(bar, parity)) return true;
  return false;
}
// polls before a wait gives up and sets the timeout flag: a poll may suspend
// for a few microseconds (B300: about 4.5 us), so about a second, against
// waits of microseconds on the normal path
constexpr uint32_t WAIT_LIMIT = 1u << 18;

// Direction components packed two bits each (1: +1, 2: -1) and the y-mirror
// five bits each, so lanes holding different directions run the same code.
__host__ __device__ constexpr uint64_t pack_comp(int axis) {
  uint64_t w = 0;
  for (int i = 0; i < NQ; i++) {
    const int c = axis == 0 ? cx(i) : axis == 1 ? cy(i) : cz(i);
    w |= (uint64_t)(c == 1 ? 1 : c == -1 ? 2 : 0) << (2 * i);
  }
  return w;
}
__host__ __device__ constexpr uint64_t pack_miry(int half) {
  uint64_t w = 0;
  for (int i = 0; i < NQ; i++) {
    const int bit = 5 * i - 64 * half;
    if (bit >= 0 && bit < 64) w |= (uint64_t)miry(i) << bit;
    if (half == 1 && bit < 0 && bit > -5) w |= (uint64_t)miry(i) >> (-bit);
  }
  return w;
}
__device__ __forceinline__ int unpack_comp(uint64_t w, int i) {
  const int b = (int)((w >> (2 * i)) & 3u);
  return b == 1 ? 1 : (b == 2 ? -1 : 0);
}
__device__ __forceinline__ int unpack_miry(int i) {
  constexpr uint64_t lo = pack_miry(0), hi = pack_miry(1);
  const int bit = 5 * i;
  const uint64_t v = bit < 64 ? ((lo >> bit) | (bit > 59 ? hi << (64 - bit) : 0)) : (hi >> (bit - 64));
  return (int)(v & 31u);
}

// Shared-memory row of one direction: [halo | XT cells | halo], the halos
// 16 bytes wide; cell tx sits at H + tx.
template <int XT, int S>
struct Stage {
  using T = typename Store<S>::T;
  static constexpr int H = 16 / (int)sizeof(T);
  static constexpr int SROW = XT + 2 * H;
};

// Producer: the lanes of one warp issue the bulk copies of tile t into a
// stage: per tile row and direction, the chunk's cells of the source row plus
// the ghost slot on the side its c_x streams from (16 bytes on that side).
// AK >= 0: the AA-pattern layout (one set, rows of aa_pitch elements in
// planes [q][z + 1][y + 1], 128-byte aligned; a spare line before the first
// and after the last row).  Step B (AK = 0) stages, per direction i, the
// row of slot opp(i) at (y - c_y, z - c_z) shifted by -c_x with the 16-byte
// block on the side c_x streams from, as the pull scheme; step A (AK = 1)
// the row of slot i at (y, z) itself.  The boundary fill before the step has
// written every slot these rows hold outside the domain.
template <int XT, int S, int AK = -1>
__device__ __forceinline__ void issue_tile(const StepParams& p, const TileGeom& g,
                                           unsigned char* stage, uint64_t* bar, int lane) {
  using T = typename Store<S>::T;
  using Gm = Geo<XT, S>;
  using St = Stage<XT, S>;
  constexpr int H = St::H;
  constexpr uint64_t kCX = pack_comp(0), kCY = pack_comp(1), kCZ = pack_comp(2);
  const int ry = blockDim.y;
  const int nrows = min(ry, p.nz - g.zg * ry);
  const int n = min(XT, p.nx - g.xc * XT);
  const int nal = (n + H - 1) / H * H;  // cells rounded up to 16 bytes (stays in the row)
  if constexpr (AK >= 0) {
    uint32_t per_row = 0;
    for (int i = 0; i < NQ; i++) per_row += (uint32_t)(nal + (AK == 0 && cx(i) != 0 ? H : 0)) * sizeof(T);
    if (lane == 0) mbar_expect_tx(bar, per_row * (uint32_t)nrows);
    __syncwarp();
    const T* set = static_cast<const T*>(p.src);
    const int x0 = g.xc * XT;
    for (int k = lane; k < nrows * NQ; k += 32) {
      const int r = k / NQ, i = k - r * NQ;
      const int z = g.zg * ry + r;
      const int q = AK == 0 ? opp(i) : i;
      const int ys = AK == 0 ? g.y - unpack_comp(kCY, i) : g.y;
      const int zs = AK == 0 ? z - unpack_comp(kCZ, i) : z;
      const int dxi = AK == 0 ? unpack_comp(kCX, i) : 0;
      const long long row = p.aa_lead + (((long long)q * (p.nz + 2) + (zs + 1)) * (p.ny + 2) + (ys + 1)) * p.aa_pitch;
      const T* src = set + row + x0;
      T* dst = reinterpret_cast<T*>(stage) + (r * NQ + i) * St::SROW + H;
      const int lo = dxi == 1 ? -H : 0, len = nal + (dxi != 0 ? H : 0);
      if (kCheckBounds) {
        const long long dofs = (dst + lo) - reinterpret_cast<T*>(stage);
        if (!in_range(row + x0 + lo, len, p.aa_elems, p.state) ||
            !in_range(dofs, len, (long long)ry * NQ * St::SROW, p.state))
          continue;
      }
      bulk_g2s(dst + lo, src + lo, (uint32_t)len * sizeof(T), bar);
    }
    return;
  }
  const bool eq_top_row = p.y_walls && p.top == 3 && g.y == p.ny - 1;
  // bytes per tile row: 19 rows of nal cells, the 10 with c_x != 0 with their
  // 16-byte ghost block (also for bounce-back rows, where it is not read);
  // constant rows (equilibrium top) are not copied
  uint32_t per_row = 0;
  for (int i = 0; i < NQ; i++) {
    if (eq_top_row && cy(i) == -1) continue;
    per_row += (uint32_t)(nal + (cx(i) != 0 ? H : 0)) * sizeof(T);
  }
  if (lane == 0) mbar_expect_tx(bar, per_row * (uint32_t)nrows);
  __syncwarp();
  const T* base = static_cast<const T*>(p.src) + Gm::G;
  for (int k = lane; k < nrows * NQ; k += 32) {
    const int r = k / NQ, i = k - r * NQ;
    const int z = g.zg * ry + r;
    int q, ys, zs;
    const int kind = row_source(p, i, unpack_comp(kCY, i), unpack_comp(kCZ, i), g.y, z, q, ys, zs);
    if (kind == SRC_CONST) continue;
    const int dxi = unpack_comp(kCX, i);
    const T* src = base + (long long)((ys * p.nz + zs) * p.nxc + g.xc) * Gm::ROW + (long long)q * Gm::XTP;
    T* dst = reinterpret_cast<T*>(stage) + (r * NQ + i) * St::SROW + H;
    const int lo = dxi == 1 ? -H : 0, len = nal + (dxi != 0 ? H : 0);
    if (kCheckBounds) {
      const long long set = (long long)p.ny * p.nz * p.nxc * Gm::ROW;  // elements of a set
      const long long so = (src + lo) - static_cast<const T*>(p.src);
      const long long dofs = (dst + lo) - reinterpret_cast<T*>(stage);
      if (!in_range(so, len, set, p.state) ||
          !in_range(dofs, len, (long long)ry * NQ * St::SROW, p.state))
        continue;
    }
    bulk_g2s(dst + lo, src + lo, (uint32_t)len * sizeof(T), bar);
  }
}

// ---- the fused step -----------------------------------------------------------------
// Persistent blocks walk a contiguous range of tiles (tile = ry rows of XT
// cells at one y).  The block keeps `nstage` tiles of source rows in flight
// (TMA bulk copies into shared memory, one mbarrier per stage); every thread
// reads its cell's 19 populations from the staged rows (shared loads at
// immediate offsets), collides in registers (moments, canopy velocity,
// Smagorinsky tau, BGK + Guo) and stores whole lines to HBM.  A stage is
// released when every warp has consumed it (monotonic per-stage count); the
// refill is then claimed (compare-and-swap on the next fill index) by the
// first warp that looks, at the top of its iteration or while it waits for
// data, so the copies are issued by a warp with time to spare and no
// block-wide barrier sits in the loop.
// Invariant: fills choose their tiles strictly in fill order (warp 0 issues
// the first round in order before any claim can succeed; later fills are
// claimed one at a time), so once a fill comes back empty no later stage holds
// a tile and the consumers may leave at the first empty stage with no copy in
// flight.  (Issuing prologue fills from several warps at once broke this and
// let a block end with copies still landing in its shared memory.)
// CPT: cells per thread along x, 1 or 2 (16-bit storage, default model:
// packed FP32x2 arithmetic on two adjacent cells, one 32-bit access per pair
// where the pair is aligned); the block is (XT / CPT) x (256 CPT / XT).
// BATCH: a work item of an ensemble (a short static run of one box, the
// pipeline started anew for each): two choices differ from the single domain's
// persistent blocks, see kItemBarrier and kItemInlineGhosts.
template <int XT, int S, bool STATS, bool VAR, int CPT, bool BATCH = false, int AK = -1>
__device__ __forceinline__ void step_tiles(const StepParams& p, long long t0l, int ntile, int part,
                                           bool dynamic) {
  static_assert(CPT == 1 || (CPT == 2 && !VAR), "two cells per thread: default model only");
  static_assert(AK < 0 || (!VAR && !BATCH), "AA-pattern tiles: default model, one domain");
  using T = typename Store<S>::T;
  using Gm = Geo<XT, S>;
  using St = Stage<XT, S>;
  constexpr int TPR = XT / CPT;  // threads per tile row
  constexpr int NT = block_threads(CPT);
  extern __shared__ __align__(128) unsigned char smem[];
  // per-thread statistics sums, kept in shared memory rather than registers
  // (the collision needs every register the three-blocks-per-SM budget allows)
  __shared__ float s_q[STATS ? 9 * NT : 1];
  __shared__ long long s_ub[8];
  __shared__ __align__(8) uint64_t s_bar[8];
  __shared__ unsigned int s_done[8];  // warps that released each stage (monotonic)
  __shared__ int s_fill;              // next fill to issue: 8 * round + stage
  __shared__ int s_nfill;             // fills issued so far (their copies may be in flight)
  __shared__ int4 s_geo[8];           // (xc, zg, y, 1) of the tile each stage holds; y < 0: none

  const int tx = threadIdx.x;
  const int tid = threadIdx.y * TPR + tx;
  const int nthreads = TPR * blockDim.y;
  const int lane = tid & 31, warp = tid >> 5;
  const unsigned int nwarps = (unsigned int)nthreads / 32;
  const int stage_bytes = (int)blockDim.y * NQ * St::SROW * (int)sizeof(T);
  // s_fill: the next fill as 8 * round + stage (fill j = round * nstage +
  // stage, so no division in the loop); kBusy is or-ed in while a warp is
  // choosing that fill's tile (one choice at a time, so dynamic tiles are
  // taken in fill order); kNoMoreFills once a fill came back empty
  constexpr int kBusy = 1 << 29, kNoMoreFills = 1 << 30;

  if (tid == 0) {
    for (int k = 0; k < p.nstage; k++) {
      mbar_init(&s_bar[k], 1);
      s_done[k] = 0;
    }
    s_fill = 8;  // round 1, stage 0: warp 0 issues round 0
    s_nfill = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (STATS) {
#pragma unroll
    for (int k = 0; k < 9; k++) s_q[k * NT + tid] = 0.f;
  }
  // Launched as a programmatic dependent of the previous step: let the next
  // step's blocks be scheduled as this grid's blocks retire, then wait here
  // until the previous step has completed and its writes are visible (both
  // are no-ops for an ordinary launch).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // Tile of the j-th fill (lane 0): the static run first, then (dynamic) one
  // tile at a time from the step's counter; -1 once none is left.
  auto tile_of_fill = [&](int j) -> long long {
    if (j < ntile) return t0l + j;
    if (!dynamic) return -1;
    const long long t = (long long)gridDim.x * p.static_tiles +
                        atomicAdd(&p.state->tile_ctr[p.ctr_slot], 1u);
    return t < p.ntiles ? t : -1;
  };
  // Fill stage rs with the j-th tile (whole warp): lane 0 picks the tile,
  // publishes its geometry (released by the mbarrier arrive) and, for a
  // claimed fill, hands the next fill on; the lanes issue the copies.  With no
  // tile left the stage completes empty and no further fill is claimed.
  auto fill = [&](int j, int rs, int next) {  // next: s_fill after a claimed fill, else -1
    TileGeom g{0, 0, -1};
    if (lane == 0) {
      s_nfill = j + 1;  // fills are issued in order
      const long long t = tile_of_fill(j);
      if (t >= 0) {
        g = tile_geom(p, t);
        s_geo[rs] = make_int4(g.xc, g.zg, g.y, 1);
        if (next >= 0) *reinterpret_cast<volatile int*>(&s_fill) = next;
      } else {
        s_geo[rs] = make_int4(0, 0, -1, 0);
        *reinterpret_cast<volatile int*>(&s_fill) = kNoMoreFills;
        mbar_arrive(&s_bar[rs]);
      }
    }
    g.xc = __shfl_sync(0xffffffffu, g.xc, 0);
    g.zg = __shfl_sync(0xffffffffu, g.zg, 0);
    g.y = __shfl_sync(0xffffffffu, g.y, 0);
    // (a withheld fill neither arrives nor copies: its stage's wait can only run out)
    if (g.y >= 0 && !(j == p.withhold && blockIdx.x == 0))
      issue_tile<XT, S, AK>(p, g, smem + rs * stage_bytes, &s_bar[rs], lane);
  };

  if (tid == 0 && dynamic && blockIdx.x == 0) p.state->tile_ctr[1 - p.ctr_slot] = 0u;  // next step's
  __syncthreads();
  // Warp 0 issues the first fills; the other warps go straight to waiting on
  // them (the mbarriers publish the tiles), each warp computing the driving
  // acceleration itself.  (A block barrier after warp 0 had computed it for
  // all, tried with 16-bit storage, was slower once three blocks share an
  // SM: B300, channel 256x128x128, 0.0990 -> 0.0969 ms without it.)
  if (warp == 0) {
    for (int k = 0; k < p.nstage; k++) fill(k, k, -1);
  }
  // An ensemble's work items start the pipeline about eight times as often as
  // the persistent single-domain blocks: there the other warps wait at a
  // barrier while warp 0 issues the first fills rather than poll beside it
  // (B300, 64-box FP16 ensemble: 1.31 ms per step with polling and the ghost
  // copies below, 1.02 ms with the barrier and ghosts stored with the cells).
  constexpr bool kItemBarrier = BATCH && sizeof(T) == 2;
  // Ensemble rows are short (a chunk edge in nearly every active warp): there
  // the two-cell form stores the ghost slots with the cells instead of copying
  // them from the stored line afterwards.
  constexpr bool kItemInlineGhosts = BATCH;
  if (kItemBarrier) __syncthreads();
  const float gx = controlled_gx(p, lane), gy = p.g[1], gz = p.g[2];
  T* dst = static_cast<T*>(p.dst) + Gm::G + CPT * tx;
  T* const dst0 = static_cast<T*>(p.dst) + Gm::G;  // slot G of direction 0, chunk-row 0

  // Issue the next fill if its stage has been released by every warp and no
  // other warp has claimed it (whole warp; lane 0 decides).
  auto try_refill = [&]() {
    int j = -1;
    if (lane == 0) {
      const int jn = *reinterpret_cast<volatile int*>(&s_fill);
      if (jn < kBusy) {
        const unsigned need = (unsigned)(jn >> 3) * nwarps;
        const unsigned done = *reinterpret_cast<volatile unsigned*>(&s_done[jn & 7]);
        if (done >= need && atomicCAS(&s_fill, jn, jn | kBusy) == jn) j = jn;
      }
    }
    j = __shfl_sync(0xffffffffu, j, 0);
    if (j >= 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int k = j & 7, r = j >> 3;
      fill(r * p.nstage + k, k, k + 1 == p.nstage ? (r + 1) * 8 : j + 1);
    }
  };

  long long ub_fix = 0;  // sum of u_x over this thread's cells, 2^-32 fixed point
  bool bad = false, late = false;
  float* const qs = s_q + tid;  // this thread's 9 sums, stride NT
  int last_x = -1;  // column of the last cell this thread accumulated (-1: none)
  int stat_y = -1;  // row the sums in qs belong to
  int stat_xc = -1;
  const bool flush_on_chunk = p.nbins > 1 && p.nxc > 1;

  int sp = 0;  // 8 * mbarrier phase parity + stage of this iteration's tile
  for (;; sp = ((sp & 7) + 1 == p.nstage) ? ((sp & 8) ^ 8) : sp + 1) {
    const int st = sp & 7;
    const uint32_t parity = (uint32_t)sp >> 3;
    const unsigned char* stage = smem + st * stage_bytes;

    try_refill();
    bool ready = false;
    for (uint32_t k = 0; k < WAIT_LIMIT; k++) {
      if (__all_sync(0xffffffffu, mbar_try(&s_bar[st], parity))) {
        ready = true;
        break;
      }
      try_refill();
    }
    if (!ready) {
      late = true;
      break;
    }
    const int4 gq = s_geo[st];  // published by the fill (mbarrier release/acquire)
    if (gq.z < 0) break;        // no tile left for this block
    if constexpr (CPT == 1) {
      const int xc = gq.x, y = gq.z;
      const int x = xc * XT + tx;
      const int z = gq.y * blockDim.y + threadIdx.y;
      const bool active = (x < p.nx) && (z < p.nz);
      if (STATS && (y != stat_y || (flush_on_chunk && xc != stat_xc))) {
        if (stat_y >= 0) flush_warp_stats<NT>(p, qs, last_x, stat_y, lane);
        stat_y = y;
        stat_xc = xc;
      }

      float f[NQ];
      Macro m;
      MacroV<float> mv;
      if (active) {
        const T* sm = reinterpret_cast<const T*>(stage) + threadIdx.y * NQ * St::SROW + St::H + tx;
        // streaming from the staged rows; at a free-slip top the staged row is
        // already the mirrored one, so only bounce-back (own column) and the
        // equilibrium top (constant) differ, on the five directions entering
        // through the wall
  #pragma unroll
        for (int i = 0; i < NQ; i++) f[i] = Store<S>::to_float(sm[i * St::SROW - (AK == 1 ? 0 : cx(i))]);
        if (AK < 0 && p.y_walls) {
          if (y == 0) {
  #pragma unroll
            for (int i = 0; i < NQ; i++)
              if (cy(i) == 1) f[i] = Store<S>::to_float(sm[i * St::SROW]);
          }
          if (y == p.ny - 1 && p.top != 2) {
  #pragma unroll
            for (int i = 0; i < NQ; i++)
              if (cy(i) == -1) f[i] = p.top == 1 ? Store<S>::to_float(sm[i * St::SROW]) : p.feq_top[i];
          }
        }
        float gxc = gx, gzc = gz;
        if (p.accel0 != nullptr && y == 0) {
          const float2 a = p.accel0[(long long)z * p.nx + x];
          gxc = gx + a.x;
          gzc = gz + a.y;
        }
        const float kd = drag_factor(p, x, y);
        if (VAR) {
          m = moments<VAR>(f, gxc, gy, gzc, kd, p.drag_x_only);
        } else {
          mv = moments_v<float>(f, gxc, gy, gzc, kd, kd > 0.f, p.tau0, p.c18);
          m = Macro{mv.drho, mv.rho, mv.ux, mv.uy, mv.uz, mv.Fx, mv.Fy, mv.Fz};
        }
      }
      // release the stage: the moments consumed every staged value of this warp
      __syncwarp();
      if (lane == 0) atomicAdd(&s_done[st], 1u);
      if (AK >= 0 && active) {
        // AA-pattern layout: direction i goes to the slot of the step's kind at
        // offset aa_wr[i] from the cell's slot of direction 0; no ghost slots
        const long long c0 = p.aa_lead + (((long long)(z + 1)) * (p.ny + 2) + (y + 1)) * p.aa_pitch + x;
        T* const cell = static_cast<T*>(p.dst) + c0;
        collide_v<float>(f, mv, [&](int i, float v) {
          if (!kCheckBounds || in_range(c0 + p.aa_wr[i], 1, p.aa_elems, p.state)) Store<S>::st(cell + p.aa_wr[i], v);
        });
        ub_fix += __float2ll_rn(m.ux * 4294967296.0f);
        bad |= !(fabsf(m.drho) < 1e30f);
        if (STATS) {
          qs[0 * NT] += m.ux; qs[1 * NT] += m.uy; qs[2 * NT] += m.uz;
          qs[3 * NT] += m.ux * m.ux; qs[4 * NT] += m.uy * m.uy; qs[5 * NT] += m.uz * m.uz;
          qs[6 * NT] += m.ux * m.uy; qs[7 * NT] += m.ux * m.uz; qs[8 * NT] += m.uy * m.uz;
          last_x = x;
        }
      } else if (active) {
        const int crow0 = (y * p.nz + z) * p.nxc;  // chunk-row of chunk 0 of this row
        T* out = dst + (long long)(unsigned)(crow0 + xc) * Gm::ROW;
        // ghost slots this cell feeds (edge lanes only): its c_x = +1 values to
        // the left ghost of the chunk on its right, its c_x = -1 values to the
        // right ghost of the chunk on its left (periodic wrap), or beside itself
        // at an outflow (zero gradient); at an x-halo face none (the halo
        // exchange sends them to the neighbouring slab and fills these ghosts)
        T* gr = nullptr;
        T* gl = nullptr;
        if (tx == 0 || tx == XT - 1 || x == p.nx - 1) {
          if (x == p.nx - 1) {
            if (p.x_io == X_PERIODIC) gr = dst0 + (long long)(unsigned)crow0 * Gm::ROW - 1;
            else if (p.x_io == X_INOUT) gl = out + 1;  // outflow: its own slot G + n (a one-cell last chunk: below)
          } else if (tx == XT - 1) {
            gr = dst0 + (long long)(unsigned)(crow0 + xc + 1) * Gm::ROW - 1;
          }
          if (x == 0) {
            if (p.x_io == X_PERIODIC) {
              const int xl = p.nxc - 1;
              gl = dst0 + (long long)(unsigned)(crow0 + xl) * Gm::ROW + (p.nx - xl * XT);
            }
          } else if (tx == 0) {
            gl = dst0 + (long long)(unsigned)(crow0 + xc - 1) * Gm::ROW + XT;
          }
        }
        auto put = [&](int i, float v) {
          if (kCheckBounds) {
            const long long set = (long long)p.ny * p.nz * p.nxc * Gm::ROW;
            T* const d0 = static_cast<T*>(p.dst);
            if (in_range(out + i * Gm::XTP - d0, 1, set, p.state)) Store<S>::st(out + i * Gm::XTP, v);
            if (cx(i) == 1 && gr && in_range(gr + i * Gm::XTP - d0, 1, set, p.state))
              Store<S>::st(gr + i * Gm::XTP, v);
            if (cx(i) == -1 && gl && in_range(gl + i * Gm::XTP - d0, 1, set, p.state))
              Store<S>::st(gl + i * Gm::XTP, v);
            return;
          }
          Store<S>::st(out + i * Gm::XTP, v);
          if (cx(i) == 1 && gr) Store<S>::st(gr + i * Gm::XTP, v);
          if (cx(i) == -1 && gl) Store<S>::st(gl + i * Gm::XTP, v);
        };
        if (VAR) collide<VAR>(f, m, p.tau0, p.c18, p.edm, p.tau_rho2, put);
        else collide_v<float>(f, mv, put);
        if (p.io_one && x == p.nx - 1) {
          // a one-cell last chunk at an outflow: gl went to the previous
          // chunk's right ghost, so the zero-gradient copy beside the cell is
          // taken from the line it just stored
  #pragma unroll
          for (int i = 0; i < NQ; i++)
            if (cx(i) == -1 &&
                (!kCheckBounds || in_range(out + 1 + i * Gm::XTP - static_cast<T*>(p.dst), 1,
                                           (long long)p.ny * p.nz * p.nxc * Gm::ROW, p.state)))
              out[1 + i * Gm::XTP] = __ldcg(out + i * Gm::XTP);
        }
        ub_fix += __float2ll_rn(m.ux * 4294967296.0f);
        // health: a non-finite density (a non-finite velocity or population
        // makes the density non-finite by the next step at the latest)
        bad |= !(fabsf(m.drho) < 1e30f);
        if (STATS) {
          qs[0 * NT] += m.ux; qs[1 * NT] += m.uy; qs[2 * NT] += m.uz;
          qs[3 * NT] += m.ux * m.ux; qs[4 * NT] += m.uy * m.uy; qs[5 * NT] += m.uz * m.uz;
          qs[6 * NT] += m.ux * m.uy; qs[7 * NT] += m.ux * m.uz; qs[8 * NT] += m.uy * m.uz;
          last_x = x;
        }
      }
    } else {
      const int xc = gq.x, y = gq.z;
      const int x = xc * XT + 2 * tx;  // cells x and x + 1
      const int z = gq.y * blockDim.y + threadIdx.y;
      const bool active = (x < p.nx) && (z < p.nz);
      const bool act1 = active && x + 1 < p.nx;
      if (STATS && (y != stat_y || (flush_on_chunk && xc != stat_xc))) {
        if (stat_y >= 0) flush_warp_stats<NT>(p, qs, last_x, stat_y, lane);
        stat_y = y;
        stat_xc = xc;
      }

      // the 19 populations of cells x and x + 1 as packed words of the
      // storage type (low half: cell x), converted to FP32 by the moments and
      // again by the collision: 19 registers instead of 38
      uint32_t raw[NQ] = {};
      MacroV<float2> m;
      const bool eqtop = AK < 0 && p.y_walls && p.top == 3 && y == p.ny - 1;
      auto f_at = [&](int i, bool again) -> float2 {
        if (cy(i) == -1 && eqtop) return make_float2(p.feq_top[i], p.feq_top[i]);
        return again ? Store<S>::unpack2_again(raw[i]) : Store<S>::unpack2(raw[i]);
      };
      if (active) {
        const T* sm = reinterpret_cast<const T*>(stage) + threadIdx.y * NQ * St::SROW + St::H + 2 * tx;
        const unsigned short* sh = reinterpret_cast<const unsigned short*>(sm);
        // streaming from the staged rows: rows with c_x = 0 hold the pair at an
        // aligned offset (one 32-bit load), the others one cell to the side
        // (two 16-bit loads); at a wall the own column (bounce-back) or, at a
        // free-slip top, the staged row that is already the mirrored one
  #pragma unroll
        for (int i = 0; i < NQ; i++) {
          if (cx(i) == 0 || AK == 1) raw[i] = *reinterpret_cast<const uint32_t*>(sm + i * St::SROW);
          else raw[i] = __byte_perm(sh[i * St::SROW - cx(i)], sh[i * St::SROW + 1 - cx(i)], 0x5410);
        }
        if (AK < 0 && p.y_walls) {
          if (y == 0) {
  #pragma unroll
            for (int i = 0; i < NQ; i++)
              if (cy(i) == 1) raw[i] = *reinterpret_cast<const uint32_t*>(sm + i * St::SROW);
          }
          if (y == p.ny - 1 && p.top == 1) {
  #pragma unroll
            for (int i = 0; i < NQ; i++)
              if (cy(i) == -1) raw[i] = *reinterpret_cast<const uint32_t*>(sm + i * St::SROW);
          }
        }
        float2 gxc = make_float2(gx, gx), gzc = make_float2(gz, gz);
        if (p.accel0 != nullptr && y == 0) {
          const float2* a = p.accel0 + (long long)z * p.nx + x;
          const float2 a0 = a[0], a1 = act1 ? a[1] : make_float2(0.f, 0.f);
          gxc = make_float2(gx + a0.x, gx + a1.x);
          gzc = make_float2(gz + a0.y, gz + a1.y);
        }
        const float2 kd = make_float2(drag_factor(p, x, y), drag_factor(p, x + 1, y));
        m = moments_g<float2>([&](int i) { return f_at(i, false); }, gxc, make_float2(gy, gy), gzc, kd,
                              kd.x > 0.f || kd.y > 0.f, p.tau0, p.c18);
      }
      // release the stage: the moments consumed every staged value of this warp
      __syncwarp();
      if (lane == 0) atomicAdd(&s_done[st], 1u);
      if (active) {
        const int crow0 = (y * p.nz + z) * p.nxc;  // chunk-row of chunk 0 of this row
        T* out = dst + (long long)(unsigned)(crow0 + xc) * Gm::ROW;
        const long long set = (long long)p.ny * p.nz * p.nxc * Gm::ROW;
        T* const d0 = static_cast<T*>(p.dst);
        auto put1 = [&](T* q, float v) {
          if (!kCheckBounds || in_range(q - d0, 1, set, p.state)) Store<S>::st(q, v);
        };
        ub_fix += __float2ll_rn(m.ux.x * 4294967296.0f);
        bad |= !(fabsf(m.drho.x) < 1e30f);
        if (act1) {
          ub_fix += __float2ll_rn(m.ux.y * 4294967296.0f);
          bad |= !(fabsf(m.drho.y) < 1e30f);
        }
        if (STATS) {
          const float2 u = m.ux, v = m.uy, w = m.uz;
          const bool split = act1 && p.nbins > 1 && !p.bins_even &&
                             ((long long)x * p.nbins) / p.nx != ((long long)(x + 1) * p.nbins) / p.nx;
          if (act1 && !split) {  // both cells in the thread's sums
            qs[0 * NT] += u.x + u.y; qs[1 * NT] += v.x + v.y; qs[2 * NT] += w.x + w.y;
            qs[3 * NT] += u.x * u.x + u.y * u.y; qs[4 * NT] += v.x * v.x + v.y * v.y;
            qs[5 * NT] += w.x * w.x + w.y * w.y; qs[6 * NT] += u.x * v.x + u.y * v.y;
            qs[7 * NT] += u.x * w.x + u.y * w.y; qs[8 * NT] += v.x * w.x + v.y * w.y;
          } else {
            qs[0 * NT] += u.x; qs[1 * NT] += v.x; qs[2 * NT] += w.x;
            qs[3 * NT] += u.x * u.x; qs[4 * NT] += v.x * v.x; qs[5 * NT] += w.x * w.x;
            qs[6 * NT] += u.x * v.x; qs[7 * NT] += u.x * w.x; qs[8 * NT] += v.x * w.x;
            if (split) {
              // the pair straddles an x-bin edge: the second cell's sums go straight out
              const long long mm = (long long)p.nbins * p.ny;
              double* acc = p.stats + ((long long)(x + 1) * p.nbins) / p.nx * p.ny + y;
              atomicAdd(acc + 0 * mm, (double)u.y); atomicAdd(acc + 1 * mm, (double)v.y);
              atomicAdd(acc + 2 * mm, (double)w.y); atomicAdd(acc + 3 * mm, (double)(u.y * u.y));
              atomicAdd(acc + 4 * mm, (double)(v.y * v.y)); atomicAdd(acc + 5 * mm, (double)(w.y * w.y));
              atomicAdd(acc + 6 * mm, (double)(u.y * v.y)); atomicAdd(acc + 7 * mm, (double)(u.y * w.y));
              atomicAdd(acc + 8 * mm, (double)(v.y * w.y));
            }
          }
          last_x = x;
        }
        if constexpr (AK >= 0) {
          // AA-pattern layout: cells x, x + 1 to the slots of the step's kind
          // (offsets aa_wr from the cell's slot of direction 0): step A and the
          // c_x = 0 directions of step B as aligned pairs, the other directions
          // of step B one cell to the side as two 16-bit stores; the second
          // cell's element only where that cell exists; no ghost slots
          const long long c0 = p.aa_lead + (((long long)(z + 1)) * (p.ny + 2) + (y + 1)) * p.aa_pitch + x;
          T* const cell = static_cast<T*>(p.dst) + c0;
          auto put_aa = [&](long long o, float v) {
            if (!kCheckBounds || in_range(c0 + o, 1, p.aa_elems, p.state)) Store<S>::st(cell + o, v);
          };
          collide_g<float2>([&](int i) { return f_at(i, true); }, m, [&](int i, float2 v) {
            const long long o = p.aa_wr[i];
            if (AK == 0 && cx(i) != 0) {
              put_aa(o, v.x);
              if (act1) put_aa(o + 1, v.y);
            } else if (act1) {
              if (!kCheckBounds || in_range(c0 + o, 2, p.aa_elems, p.state)) Store<S>::st2(cell + o, v);
            } else {
              put_aa(o, v.x);
            }
          });
        } else if constexpr (kItemInlineGhosts) {
          // Ghost slots the pair feeds, stored with the cells: at most one for
          // its c_x = +1 values (offset gro from `out`, cell grc) and one for
          // its c_x = -1 values (glo, cell glc); a two-cell last chunk of an
          // outflow row takes its outflow copy from the stored line (copy1).
          constexpr int kNone = INT_MIN;
          int gro = kNone, glo = kNone;
          bool grc = false, glc = false, copy1 = false;
          if (tx == 0 || tx == TPR - 1 || x + 1 >= p.nx - 1) {
            const long long own = (long long)(unsigned)(crow0 + xc) * Gm::ROW + 2 * tx;  // out - dst0
            if (x == p.nx - 1) {
              if (p.x_io == X_PERIODIC) gro = (int)((long long)(unsigned)crow0 * Gm::ROW - 1 - own);
              else if (p.x_io == X_INOUT) glo = 1;
            } else if (act1 && x + 1 == p.nx - 1) {
              grc = glc = true;
              if (p.x_io == X_PERIODIC) gro = (int)((long long)(unsigned)crow0 * Gm::ROW - 1 - own);
              else if (p.x_io == X_INOUT) glo = 2;
            } else if (act1 && tx == TPR - 1) {
              grc = true;
              gro = (int)((long long)(unsigned)(crow0 + xc + 1) * Gm::ROW - 1 - own);
            }
            int left = kNone;
            if (x == 0) {
              if (p.x_io == X_PERIODIC) {
                const int xl = p.nxc - 1;
                left = (int)((long long)(unsigned)(crow0 + xl) * Gm::ROW + (p.nx - xl * XT) - own);
              }
            } else if (tx == 0) {
              left = (int)((long long)(unsigned)(crow0 + xc - 1) * Gm::ROW + XT - own);
            }
            if (left != kNone) {
              copy1 = glc && glo == 2;
              glo = left;
              glc = false;
            }
          }
          collide_g<float2>([&](int i) { return f_at(i, true); }, m, [&](int i, float2 v) {
            T* o = out + i * Gm::XTP;
            if (act1) {
              if (!kCheckBounds || in_range(o - d0, 2, set, p.state)) Store<S>::st2(o, v);
            } else {
              put1(o, v.x);
            }
            if (cx(i) == 1 && gro != kNone) put1(o + gro, grc ? v.y : v.x);
            if (cx(i) == -1 && glo != kNone) put1(o + glo, glc ? v.y : v.x);
          });
          if (copy1) {
  #pragma unroll
            for (int i = 0; i < NQ; i++)
              if (cx(i) == -1) put1(out + 2 + i * Gm::XTP, Store<S>::to_float(__ldcg(out + 1 + i * Gm::XTP)));
          }
        } else {
          collide_g<float2>([&](int i) { return f_at(i, true); }, m, [&](int i, float2 v) {
            T* o = out + i * Gm::XTP;
            if (act1) {
              if (!kCheckBounds || in_range(o - d0, 2, set, p.state)) Store<S>::st2(o, v);
            } else {
              put1(o, v.x);
            }
          });
          // Ghost slots the pair feeds (as for one cell per thread): at most one
          // for its c_x = +1 values (offset gro from `out`, cell grc) and one
          // for its c_x = -1 values (glo, cell glc).  Cell x can be the first of
          // its chunk or the last of the domain, cell x + 1 the last of its
          // chunk or of the domain.  Only a two-cell last chunk of an outflow
          // row needs both a chunk ghost and the outflow copy on the c_x = -1
          // side (copy1).  The edge lanes copy the values from the line they just
          // stored, so the other lanes' stores carry no ghost code.
          if (tx == 0 || tx == TPR - 1 || x + 1 >= p.nx - 1) {
            constexpr int kNone = INT_MIN;
            int gro = kNone, glo = kNone;
            bool grc = false, glc = false, copy1 = false;
            const long long own = (long long)(unsigned)(crow0 + xc) * Gm::ROW + 2 * tx;  // out - dst0
            if (x == p.nx - 1) {
              if (p.x_io == X_PERIODIC) gro = (int)((long long)(unsigned)crow0 * Gm::ROW - 1 - own);
              else if (p.x_io == X_INOUT) glo = 1;
            } else if (act1 && x + 1 == p.nx - 1) {
              grc = glc = true;
              if (p.x_io == X_PERIODIC) gro = (int)((long long)(unsigned)crow0 * Gm::ROW - 1 - own);
              else if (p.x_io == X_INOUT) glo = 2;
            } else if (act1 && tx == TPR - 1) {
              grc = true;
              gro = (int)((long long)(unsigned)(crow0 + xc + 1) * Gm::ROW - 1 - own);
            }
            int left = kNone;
            if (x == 0) {
              if (p.x_io == X_PERIODIC) {
                const int xl = p.nxc - 1;
                left = (int)((long long)(unsigned)(crow0 + xl) * Gm::ROW + (p.nx - xl * XT) - own);
              }
            } else if (tx == 0) {
              left = (int)((long long)(unsigned)(crow0 + xc - 1) * Gm::ROW + XT - own);
            }
            if (left != kNone) {
              copy1 = glc && glo == 2;  // and the outflow copy of cell x + 1
              glo = left;
              glc = false;
            }
            // a stored value to another slot (the same bits, so the same as
            // storing the FP32 value there)
            auto copy = [&](long long to, int from) {
              if (!kCheckBounds || in_range(out + to - d0, 1, set, p.state)) out[to] = __ldcg(out + from);
            };
            if (gro != kNone) {
    #pragma unroll
              for (int i = 0; i < NQ; i++)
                if (cx(i) == 1) copy((long long)gro + i * Gm::XTP, (grc ? 1 : 0) + i * Gm::XTP);
            }
            if (glo != kNone) {
    #pragma unroll
              for (int i = 0; i < NQ; i++)
                if (cx(i) == -1) copy((long long)glo + i * Gm::XTP, (glc ? 1 : 0) + i * Gm::XTP);
            }
            if (copy1) {
    #pragma unroll
              for (int i = 0; i < NQ; i++)
                if (cx(i) == -1) copy(2 + i * Gm::XTP, 1 + i * Gm::XTP);
            }
          }
        }
        if (AK < 0 && p.io_one && x == p.nx - 1) {
          // a one-cell last chunk at an outflow (its cell is the pair's first):
          // the zero-gradient copy beside the cell from the line it just stored
  #pragma unroll
          for (int i = 0; i < NQ; i++)
            if (cx(i) == -1 &&
                (!kCheckBounds || in_range(out + 1 + i * Gm::XTP - d0, 1, set, p.state)))
              out[1 + i * Gm::XTP] = __ldcg(out + i * Gm::XTP);
        }
      }
    }
  }
  if (STATS && stat_y >= 0) flush_warp_stats<NT>(p, qs, last_x, stat_y, lane);
  finish_step(p, ub_fix, bad, late, s_ub, lane, warp, tid, nthreads, part);
  // Leave no copy in flight when the block ends: after a timed-out wait some
  // issued fills were never consumed.  (On the normal path every issued fill
  // has completed; the waits return at once.)  finish_step ended with a
  // block barrier, so s_nfill is final.  A drain wait that runs out too (a
  // copy still landing after about a second) is reported as a timeout: the
  // block then ends with that copy in flight and the context is unusable.
  if (tid == 0) {
    const int nf = s_nfill;
    bool drained = true;
    for (int k = 0; k < p.nstage && k < nf; k++) {
      const int uses = (nf - 1 - k) / p.nstage + 1;  // fills that went into stage k
      drained &= mbar_wait(&s_bar[k], (uint32_t)((uses - 1) & 1), WAIT_LIMIT);
    }
    if (!drained) atomicOr(&p.state->timeout_flag, 1u);
  }
}

// One domain: block b walks its static run of tiles, then shares the rest.
// VAR: the model-variant form (flags in p); the default form has none of
// their code.
// AK >= 0: one step of the AA-pattern layout (0: step B, 1: step A) with the
// same tile pipeline, in place (every location is read and written by the
// same cell: step B reads slot opp(i) at x - c_i and writes slot i at x + c_i,
// step A reads slot i and writes slot opp(i) of cell x, so no tile's stores
// touch another tile's sources).
template <int XT, int S, bool STATS, bool VAR, int CPT, int AK = -1>
__global__ void __launch_bounds__(block_threads(CPT), 768 / block_threads(CPT)) step_kernel(StepParams p) {
  step_tiles<XT, S, STATS, VAR, CPT, false, AK>(p, (long long)blockIdx.x * p.static_tiles, p.static_tiles,
                                                blockIdx.x, true);
}

// Many independent domains (an ensemble of boxes) in one launch: work item
// w = (box, first tile, tiles) per block; the block runs the same tile loop
// with its box's parameters copied to shared memory.
struct BatchWork {
  int box, ntile;
  long long t0;
};

template <int XT, int S, bool STATS, int CPT>
__global__ void __launch_bounds__(block_threads(CPT), 768 / block_threads(CPT)) batch_step_kernel(
    const StepParams* __restrict__ boxes, const BatchWork* __restrict__ work) {
  __shared__ __align__(16) StepParams s_p;
  const BatchWork w = work[blockIdx.x];
  {
    static_assert(sizeof(StepParams) % 4 == 0, "copied as words");
    const unsigned* src = reinterpret_cast<const unsigned*>(boxes + w.box);
    unsigned* dst = reinterpret_cast<unsigned*>(&s_p);
    for (int k = threadIdx.y * blockDim.x + threadIdx.x; k < (int)(sizeof(StepParams) / 4);
         k += blockDim.x * blockDim.y)
      dst[k] = src[k];
  }
  __syncthreads();
  step_tiles<XT, S, STATS, false, CPT, true>(s_p, w.t0, w.ntile, -1, false);
}

// ---- ghost slots from the cells (after init, set_f) ----------------------------------
// One thread per (chunk-row, side, direction with c_x != 0).  The inflow
// ghosts hold the inflow equilibrium and are never rewritten by a step; the
// ghosts at an x-halo face are left to the halo exchange.
template <int XT, int S>
__global__ void ghost_kernel(StepParams p, void* fv) {
  using T = typename Store<S>::T;
  using Gm = Geo<XT, S>;
  T* f = static_cast<T*>(fv) + Gm::G;
  const long long rows = (long long)p.ny * p.nz * p.nxc;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < rows * 10;
       k += (long long)gridDim.x * blockDim.x) {
    const long long cr = k / 10;
    const int j = (int)(k - cr * 10);
    const int xc = (int)(cr % p.nxc);
    const long long yz = cr / p.nxc;
    const int y = (int)(yz / p.nz);
    const int x0 = xc * XT, n = min(XT, p.nx - x0);
    // j < 5: left ghost of c_x = +1 directions 1 7 9 11 13; j >= 5: right, 2 8 10 12 14
    const int i = j < 5 ? (j == 0 ? 1 : 5 + 2 * j) : (j == 5 ? 2 : 2 * (j - 5) + 6);
    T* row = f + cr * Gm::ROW + (long long)i * Gm::XTP;
    auto cell = [&](int xc2, int t) { return f[((yz * p.nxc) + xc2) * Gm::ROW + (long long)i * Gm::XTP + t]; };
    if (j < 5) {
      if (xc > 0) row[-1] = cell(xc - 1, XT - 1);
      else if (p.x_io == X_INOUT) row[-1] = Store<S>::from_double((double)p.feq_in[y * NQ + i]);
      else if (p.x_io == X_PERIODIC) row[-1] = cell(p.nxc - 1, p.nx - 1 - (p.nxc - 1) * XT);
    } else {
      if (xc < p.nxc - 1) row[n] = cell(xc + 1, 0);
      else if (p.x_io == X_INOUT) row[n] = row[n - 1];
      else if (p.x_io == X_PERIODIC) row[n] = cell(0, 0);
    }
  }
}

// ---- x-halo exchange of a slab (one domain cut into x-slabs) --------------------------
// Per step a slab face passes on only what streams across it (Eq. lbe: the
// pull reaches one column, and only for the five directions with c_x = +-1).
// Face buffers are [d][y][z] in the storage type, d indexing the directions
// 1, 7, 9, 11, 13 (c_x = +1) or 2, 8, 10, 12, 14 (c_x = -1).
__host__ __device__ constexpr int halo_dir(int side, int d) {  // side 1: c_x = +1
  return side ? (d == 0 ? 1 : 5 + 2 * d) : (d == 0 ? 2 : 6 + 2 * d);
}

// Pack the post-collision state f: lo <- the c_x = -1 values of column 0 (for
// the left neighbour's right halo), hi <- the c_x = +1 values of column nx - 1
// (for the right neighbour's left halo).
template <int XT, int S>
__global__ void halo_pack_kernel(StepParams p, const void* fv, void* lo, void* hi) {
  using T = typename Store<S>::T;
  const T* f = static_cast<const T*>(fv);
  const long long per = (long long)p.ny * p.nz;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 10 * per;
       k += (long long)gridDim.x * blockDim.x) {
    const int side = k >= 5 * per ? 1 : 0;
    const long long r = k - side * 5 * per;
    const int d = (int)(r / per);
    const long long yz = r - d * per;
    const int y = (int)(yz / p.nz), z = (int)(yz - (long long)y * p.nz);
    const T v = f[pop_index<XT, S>(p, halo_dir(side, d), side ? p.nx - 1 : 0, y, z)];
    static_cast<T*>(side ? hi : lo)[r] = v;
  }
}

// Unpack received faces into the ghost slots of f (the state the next step
// reads): lo (the left neighbour's c_x = +1 values) into slot G - 1 of chunk 0,
// hi (the right neighbour's c_x = -1 values) into slot G + n of the last chunk.
template <int XT, int S>
__global__ void halo_unpack_kernel(StepParams p, void* fv, const void* lo, const void* hi) {
  using T = typename Store<S>::T;
  T* f = static_cast<T*>(fv);
  const long long per = (long long)p.ny * p.nz;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 10 * per;
       k += (long long)gridDim.x * blockDim.x) {
    const int side = k >= 5 * per ? 1 : 0;  // 0: from the left, 1: from the right
    const long long r = k - side * 5 * per;
    const int d = (int)(r / per);
    const long long yz = r - d * per;
    const int y = (int)(yz / p.nz), z = (int)(yz - (long long)y * p.nz);
    const long long at = side ? pop_index<XT, S>(p, halo_dir(0, d), p.nx - 1, y, z) + 1
                              : pop_index<XT, S>(p, halo_dir(1, d), 0, y, z) - 1;
    f[at] = static_cast<const T*>(side ? hi : lo)[r];
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
  int nx, ny, nz, nxc;
  const double* u_prof;  // ny values or nullptr
  uint64_t seed;
  double amp;
};

template <int XT, int S>
__global__ void init_kernel(InitParams p) {
  using T = typename Store<S>::T;
  using Gm = Geo<XT, S>;
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
    T* cell = f + (((long long)y * p.nz + z) * p.nxc + x / XT) * Gm::ROW + Gm::G + x % XT;
#pragma unroll
    for (int i = 0; i < NQ; i++) {
      const double cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
      const double fs = wgt_d(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);  // f_eq(1,u) - w_i
      cell[i * Gm::XTP] = Store<S>::from_double(fs);
    }
  }
}

// ---- global mass: deterministic two-pass FP64 reduction ------------------------------
template <int XT, int S>
__global__ void mass_partial_kernel(const void* fv, int nx, long long rows, int nxc, double* partial) {
  using T = typename Store<S>::T;
  using Gm = Geo<XT, S>;
  const T* f = static_cast<const T*>(fv);
  double acc = 0.0;
  const long long total = rows * nx * NQ;  // (row, q, x) over the real cells
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long row = k / ((long long)nx * NQ);
    const long long rem = k - row * nx * NQ;
    const int q = (int)(rem / nx), x = (int)(rem - (long long)q * nx);
    acc += (double)Store<S>::ld(f + (row * nxc + x / XT) * Gm::ROW + (long long)q * Gm::XTP + Gm::G +
                                x % XT);
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


// ---- macroscopic fields of the next step (pull + moments only) ------------------------
// Direct loads with the same boundary rules as the step (not performance critical).
// The 19 (shifted) populations cell (x, y, z) streams in for the next step,
// gathered one by one with the step's boundary rules (readouts, not the step).
template <int XT, int S>
__device__ __forceinline__ void gather_cell(const StepParams& p, int x, int y, int z, float* f) {
  using T = typename Store<S>::T;
  const T* src = static_cast<const T*>(p.src);
#pragma unroll
  for (int i = 0; i < NQ; i++) {
    int q, ys, zs;
    const int kind = row_source(p, i, cy(i), cz(i), y, z, q, ys, zs);
    if (kind == SRC_CONST) {
      f[i] = p.feq_top[i];
    } else if (kind == SRC_OWN_X) {
      f[i] = Store<S>::ld(src + pop_index<XT, S>(p, q, x, ys, zs));
    } else {
      const int xs = source_x(p, x, cx(i));
      if (p.x_io == X_HALO && xs < 0)  // the left halo: ghost slot G - 1 of chunk 0
        f[i] = Store<S>::ld(src + pop_index<XT, S>(p, q, 0, ys, zs) - 1);
      else if (p.x_io == X_HALO && xs >= p.nx)  // the right halo: slot G + n of the last chunk
        f[i] = Store<S>::ld(src + pop_index<XT, S>(p, q, p.nx - 1, ys, zs) + 1);
      else
        f[i] = xs < 0 ? p.feq_in[ys * NQ + q] : Store<S>::ld(src + pop_index<XT, S>(p, q, xs, ys, zs));
    }
  }
}

// Strain-rate magnitude |S| = sqrt(2 S:S) of a cell from its non-equilibrium
// momentum flux (Eq. tensor) through Pi_neq = -2 rho c_s^2 tau_total S, with
// f_eq and tau_total as in the collision (the model variants included).
__device__ __forceinline__ float strain_rate(const float* f, const Macro& m, float tau0, float c18,
                                             int edm = 0, int tau_rho2 = 0) {
  const float hx = edm ? 0.5f * m.Fx / m.rho : 0.f, hy = edm ? 0.5f * m.Fy / m.rho : 0.f,
              hz = edm ? 0.5f * m.Fz / m.rho : 0.f;  // exact difference: f_eq at u - g/2
  const float ux = m.ux - hx, uy = m.uy - hy, uz = m.uz - hz;
  // Pi_neq = S - c_s^2 (rho - 1) I - rho u u, S the second moments of the
  // shifted populations (the second moment of f_eq is rho c_s^2 I + rho u u)
  float sxx = 0.f, syy = 0.f, szz = 0.f, sxy = 0.f, sxz = 0.f, syz = 0.f;
#pragma unroll
  for (int i = 1; i < NQ; i += 2) {
    const float sp = f[i] + f[i + 1];
    if (cx(i) != 0) sxx += sp;
    if (cy(i) != 0) syy += sp;
    if (cz(i) != 0) szz += sp;
    if (cx(i) * cy(i) != 0) sxy += (float)(cx(i) * cy(i)) * sp;
    if (cx(i) * cz(i) != 0) sxz += (float)(cx(i) * cz(i)) * sp;
    if (cy(i) * cz(i) != 0) syz += (float)(cy(i) * cz(i)) * sp;
  }
  const float d3 = m.drho * (1.0f / 3.0f), r = m.rho;
  const float pxx = sxx - d3 - r * ux * ux, pyy = syy - d3 - r * uy * uy, pzz = szz - d3 - r * uz * uz;
  const float pxy = sxy - r * ux * uy, pxz = sxz - r * ux * uz, pyz = syz - r * uy * uz;
  const float q2 = pxx * pxx + pyy * pyy + pzz * pzz + 2.0f * (pxy * pxy + pxz * pxz + pyz * pyz);
  const float q = sqrtf(q2);
  const float tau = 0.5f * (tau0 + sqrtf(tau0 * tau0 + c18 * q / (tau_rho2 ? m.rho * m.rho : m.rho)));
  return 2.1213203435596424f * q / (m.rho * tau);  // sqrt(2) / (2 c_s^2) = 3 / sqrt(2)
}

template <int XT, int S, class OutT = float>
__global__ void macro_kernel(StepParams p, OutT* out) {
  const long long n = (long long)p.nx * p.ny * p.nz;
  const float gx = controlled_gx(p, threadIdx.x & 31);  // blockDim.x is a multiple of 32
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % p.nx);
    const long long r = c / p.nx;
    const int y = (int)(r % p.ny);
    const int z = (int)(r / p.ny);
    float f[NQ];
    gather_cell<XT, S>(p, x, y, z, f);
    const Macro m = moments<true>(f, gx, p.g[1], p.g[2], drag_factor(p, x, y), p.drag_x_only);
    out[c] = m.rho;
    out[n + c] = m.ux;
    out[2 * n + c] = m.uy;
    out[3 * n + c] = m.uz;
  }
}

}  // namespace lbm
