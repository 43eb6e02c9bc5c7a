// lbm_api.cu -- host side of the C ABI declared in include/lbm.h.
//
// Owns the context (grid, parameters, device buffers carved from one
// workspace), enqueues the kernels of lbm_device.cuh on the context's stream,
// and converts populations between the device storage (row-interleaved
// [y][z][x-chunk][q][x], shifted by the lattice weights, FP32/FP16/BF16) and
// the public FP64 layout ([q][z][y][x], unshifted).  No lattice Boltzmann
// arithmetic runs on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_diag.cuh"
#include "lbm_kernels.h"

using namespace lbm;

namespace {

constexpr size_t kAlign = 256;
// LBM_STATIC_PERCENT (for experiments) fixes the static share of every step's
// tiles; by default it follows the run length (static_percent below)
constexpr int kMassBlocks = 1024;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t elem_bytes(int storage) { return (storage & 0xff) == LBM_F32 ? 4 : 2; }

// storage argument: an element type, or-ed with LBM_STORAGE_AA for the
// AA-pattern layout (one population set)
bool storage_ok(int32_t storage) {
  const int t = storage & 0xff, flags = storage & ~0xff;
  return t >= 0 && t <= 2 && (flags == 0 || flags == LBM_STORAGE_AA);
}
bool is_aa(int32_t storage) { return (storage & LBM_STORAGE_AA) != 0; }

// AA-pattern set: rows of nx + 2 cells rounded up to whole 128-byte lines (the
// left ghost of a row is the previous row's last slot), planes [q][z][y] with
// a ghost layer in y and z, one line before the first row.
struct AAShape {
  long long pitch, lead, elems;
};
AAShape aa_shape_of(const lbm_grid& g, int storage) {
  const long long line = 128 / (long long)elem_bytes(storage);
  AAShape a;
  a.pitch = (g.nx + 2 + line - 1) / line * line;
  a.lead = line;
  a.elems = a.lead + (long long)NQ * (g.nz + 2) * (g.ny + 2) * a.pitch + line;
  return a;
}

// chunk width: the smallest of 64, 128, 256 cells that covers a row, else 256
int chunk_width(int nx) { return nx <= 64 ? 64 : (nx <= 128 ? 128 : 256); }

struct Shape {
  int xt, nxc, g, xtp;  // chunk width, chunks per row, ghost line, direction-row length
  long long row;        // elements per chunk-row (19 direction rows)
  long long elems;      // elements per population set
};

// xt: chunk width, 0 = chunk_width(nx)
Shape shape_of(const lbm_grid& gr, int storage, int xt = 0) {
  Shape s;
  s.xt = xt ? xt : chunk_width(gr.nx);
  s.nxc = (gr.nx + s.xt - 1) / s.xt;
  s.g = 128 / (int)elem_bytes(storage);
  s.xtp = s.xt + 2 * s.g;
  s.row = (long long)NQ * s.xtp;
  s.elems = (long long)gr.ny * gr.nz * s.nxc * s.row;
  return s;
}

struct Layout {
  size_t f_bytes, stats_off, state_off, ubpart_off, kdrag_off, lad_off, feqin_off, uprof_off,
      mass_off, accel_off, total;
};

Layout layout_of(const lbm_grid& g, int storage, int nbins, int xt = 0) {
  Layout L;
  const Shape s = shape_of(g, storage, xt);
  const long long elems = is_aa(storage) ? aa_shape_of(g, storage).elems : s.elems;
  L.f_bytes = align_up((size_t)elems * elem_bytes(storage), kAlign);
  size_t off = is_aa(storage) ? L.f_bytes : 2 * L.f_bytes;  // AA: one set
  L.stats_off = off;  off += align_up(sizeof(double) * 9 * nbins * g.ny, kAlign);
  L.state_off = off;  off += align_up(sizeof(DevState), kAlign);
  L.ubpart_off = off; off += align_up(sizeof(long long) * 2 * MAX_BLOCKS, kAlign);
  L.kdrag_off = off;  off += align_up(sizeof(float) * g.ny, kAlign);
  L.lad_off = off;    off += align_up(sizeof(float) * g.ny, kAlign);
  L.feqin_off = off;  off += align_up(sizeof(float) * NQ * g.ny, kAlign);
  L.uprof_off = off;  off += align_up(sizeof(double) * g.ny, kAlign);
  L.mass_off = off;   off += align_up(sizeof(double) * (kMassBlocks + 1), kAlign);
  L.accel_off = off;  off += align_up(sizeof(float2) * g.nx * g.nz, kAlign);
  L.total = off;
  return L;
}

bool grid_ok(const lbm_grid* g) {
  if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1) return false;
  const long long cells = (long long)g->nx * g->ny * g->nz;
  if (cells >= (1ll << 31)) return false;
  const bool xper = g->x_lo == LBM_BC_PERIODIC && g->x_hi == LBM_BC_PERIODIC;
  const bool xio = (g->x_lo == LBM_BC_INFLOW && g->x_hi == LBM_BC_OUTFLOW) ||
                   (g->x_lo == LBM_BC_HALO && g->x_hi == LBM_BC_HALO);
  const bool yper = g->y_lo == LBM_BC_PERIODIC && g->y_hi == LBM_BC_PERIODIC;
  const bool ywall = g->y_lo == LBM_BC_BOUNCEBACK &&
                     (g->y_hi == LBM_BC_BOUNCEBACK || g->y_hi == LBM_BC_FREESLIP ||
                      g->y_hi == LBM_BC_EQUILIBRIUM);
  const bool zper = g->z_lo == LBM_BC_PERIODIC && g->z_hi == LBM_BC_PERIODIC;
  return (xper || xio) && (yper || ywall) && zper;
}

}  // namespace

struct lbm_ctx {
  lbm_grid grid;
  int storage = 0, nbins = 1;   // element type (lbm_storage without flags)
  bool aa = false;              // AA-pattern layout: one population set
  bool aa_tma = false;          // ... stepped by the pull scheme's tile pipeline (default model)
  AAShape ash{};
  double tau0 = 0, cs = 0;
  lbm_forcing forcing;
  std::vector<double> lad, uprof;
  uint64_t seed = 0;
  double init_perturb = 0;
  Shape sh;
  long long cells = 0;
  Layout L;
  char* ws = nullptr;
  bool owns_ws = false;
  cudaStream_t stream = nullptr;
  int cur = 0;                // population set holding the current state
  int64_t steps = 0;
  bool stats_on = false;
  int64_t stats_samples = 0;
  float* macro_buf = nullptr;
  int sm_count = 0, blocks_per_sm = 0;
  int device = 0;             // the device the context was created on
  int last_grid = 0;          // blocks of the previous step launch (partials to sum)
  int nstage = 0;             // tiles in flight per block
  int test_withhold = -1;     // lbm_test_withhold_fill: fill block 0 skips in the next step
  size_t stage_smem = 0;      // dynamic shared memory per block
  dim3 block;
  int nzg = 0;
  lbm_status status = LBM_OK;
  std::string err;
  lbm_batch* batch = nullptr;  // owning ensemble, if this domain is one of its boxes
  const lbm_mlp* mlp = nullptr;  // learned first-layer correction in use, if any
  float lam = 0.f;               // its velocity relaxation rate
  float* feat_buf = nullptr;     // staging buffer of lbm_features
  unsigned char* readout = nullptr;  // pinned host copies of the statistics and health flags:
                                     // slot 0 for lbm_stats, slots 1 and 2 for the pipelined read-out
  unsigned char* readout_dev = nullptr;  // the same buffer's device address (mapped pinned memory)
  cudaEvent_t rd_ev[2] = {nullptr, nullptr};  // completion of the pipelined copies
  int64_t rd_samples[2] = {0, 0};             // steps accumulated when each copy was enqueued
  int rd_first = 0, rd_pending = 0;           // oldest pending slot (0/1), pending count

  void* fbuf(int k) const { return ws + (size_t)k * L.f_bytes; }
  double* stats() const { return reinterpret_cast<double*>(ws + L.stats_off); }
  DevState* state() const { return reinterpret_cast<DevState*>(ws + L.state_off); }
  long long* ub_part() const { return reinterpret_cast<long long*>(ws + L.ubpart_off); }
  float* kdrag() const { return reinterpret_cast<float*>(ws + L.kdrag_off); }
  float* lad_dev() const { return reinterpret_cast<float*>(ws + L.lad_off); }
  float2* accel() const { return reinterpret_cast<float2*>(ws + L.accel_off); }
  float* feq_in() const { return reinterpret_cast<float*>(ws + L.feqin_off); }
  double* uprof_dev() const { return reinterpret_cast<double*>(ws + L.uprof_off); }
  double* mass_buf() const { return reinterpret_cast<double*>(ws + L.mass_off); }
  // device element index of the post-collision population q at cell (x, y, z)
  // of the current state (AA: in the layout of the current step parity)
  long long dev_index(int q, int x, int y, int z) const {
    if (aa) {
      auto at = [&](int qq, int xx, int yy, int zz) {
        return ash.lead + (((long long)qq * (grid.nz + 2) + (zz + 1)) * (grid.ny + 2) + (yy + 1)) * ash.pitch + xx;
      };
      return (steps & 1) == 0 ? at(opp(q), x, y, z) : at(q, x + cx(q), y + cy(q), z + cz(q));
    }
    return (((long long)y * grid.nz + z) * sh.nxc + x / sh.xt) * sh.row + (long long)q * sh.xtp +
           sh.g + x % sh.xt;
  }
  // elements of one population set
  long long set_elems() const { return aa ? ash.elems : sh.elems; }
};

// A correction network: parameters and training state on the device.
struct lbm_mlp {
  float* theta = nullptr;       // [MLP_NP] weights, biases and normalisation (FP32 master copy)
  float* adam_m = nullptr;      // [MLP_NW] Adam first moments
  float* adam_v = nullptr;      // [MLP_NW] Adam second moments
  float* grad = nullptr;        // [MLP_NW] gradient of the last batch
  float* sse = nullptr;         // sum of squared errors of the last pass
  float* scratch = nullptr;     // training activations and deltas
  long long scratch_rows = 0;
  float* data = nullptr;        // training set on the device (X then Y)
  long long data_rows = 0;
  int* perm = nullptr;          // sample order of an epoch
  long long adam_t = 0;         // Adam steps taken
  cudaStream_t stream = nullptr;
  std::string err;
};

namespace {

lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg) {
  if (c && c->status == LBM_OK) {
    c->status = s;
    c->err = msg;
  }
  return s;
}

lbm_status arg_error(lbm_ctx* c, const std::string& msg) {
  if (c) c->err = msg;  // argument errors are not sticky
  return LBM_ERR_ARG;
}

#define CK(ctx, call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail((ctx), LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Shifted equilibrium f_eq(1, u) - w_i in FP64 (for the boundary tables).
void feq_shift(const double u[3], double out[NQ]) {
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < NQ; i++) {
    const double cu = cx(i) * u[0] + cy(i) * u[1] + cz(i) * u[2];
    out[i] = wgt_d(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
  }
}

// Share of a step's tiles handed out as fixed contiguous runs, the rest taken one
// by one by whichever block is free.  The three blocks of an SM do not run at
// the same speed (the first scheduled is ~15 % faster), so long runs need a
// dynamic share of about that size; short runs pay more for dynamic tiles
// than the imbalance costs them; 16-bit storage (shorter tiles in time)
// reaches that point sooner.  B300, ms per step at 92 / 90 / 88 / 85 %:
// 256x128x128 channel (37 tiles per block) FP32 0.1186 / 0.1185 / 0.1200 /
// 0.1228, FP16 0.1129 / 0.1128 / 0.1146 / 0.1162; 512x128x256 canopy (148)
// FP32 0.4607 / 0.4530 / 0.4495 / 0.4562, FP16 0.4373 / 0.4295 / 0.4230 /
// 0.4180; 1024x256x512 canopy (1180) FP32 at 90 / 85 %: 3.54 / 3.36.
long long static_percent(long long tiles_per_block, size_t elem) {
#ifdef LBM_STATIC_PERCENT
  (void)tiles_per_block;
  (void)elem;
  return LBM_STATIC_PERCENT;
#else
  if (tiles_per_block <= 64) return 90;
  return (elem == 2 || tiles_per_block > 256) ? 85 : 88;
#endif
}

int step_grid(const lbm_ctx* c) {
  const long long ntiles = (long long)c->sh.nxc * c->nzg * c->grid.ny;
  const long long want = (long long)c->sm_count * c->blocks_per_sm;
  return (int)std::max<long long>(1, std::min<long long>({want, ntiles, (long long)MAX_BLOCKS}));
}

StepParams make_params(const lbm_ctx* c) {
  StepParams p;
  std::memset(&p, 0, sizeof(p));
  const lbm_grid& g = c->grid;
  p.nx = g.nx; p.ny = g.ny; p.nz = g.nz; p.nxc = c->sh.nxc;
  p.x_io = g.x_lo == LBM_BC_INFLOW ? X_INOUT : g.x_lo == LBM_BC_HALO ? X_HALO : X_PERIODIC;
  p.y_walls = g.y_lo == LBM_BC_BOUNCEBACK;
  p.top = g.y_hi == LBM_BC_BOUNCEBACK ? 1 : g.y_hi == LBM_BC_FREESLIP ? 2 : 3;
  p.tau0 = (float)c->tau0;
  p.c18 = (float)(18.0 * std::sqrt(2.0) * c->cs * c->cs);
  for (int a = 0; a < 3; a++) p.g[a] = (float)c->forcing.g[a];
  p.ctrl = c->forcing.u_bulk_target > 0.0;
  p.g0x = c->forcing.g[0];
  p.gain = c->forcing.ctrl_gain;
  p.u_target = c->forcing.u_bulk_target;
  p.inv_cells = 1.0 / (double)c->cells;
  const int64_t t = c->steps;
  p.have_prev = t > 0;
  p.ub_part = c->ub_part();
  p.slot_read = (int)((t + 1) % 2);
  p.slot_write = (int)(t % 2);
  p.nprev = c->last_grid;
  p.canopy_x0 = c->forcing.x_canopy_begin;
  p.canopy_x1 = c->forcing.x_canopy_end;
  p.kdrag = c->lad.empty() ? nullptr : c->kdrag();
  p.lad = c->lad.empty() ? nullptr : c->lad_dev();
  p.accel0 = c->mlp ? c->accel() : nullptr;
  p.feq_in = c->feq_in();
  double ft[NQ];
  feq_shift(c->forcing.u_top, ft);
  for (int i = 0; i < NQ; i++) p.feq_top[i] = (float)ft[i];
  p.nzg = c->nzg;
  p.ntiles = (long long)c->sh.nxc * c->nzg * g.ny;
  p.nstage = c->nstage;
  p.withhold = c->test_withhold;
  // a share of the tiles in fixed contiguous runs per block, the rest handed
  // out one by one to whichever block is free (blocks of an SM do not run at
  // the same speed)
  {
    const long long grid = step_grid(c);
    p.static_tiles =
        (int)(p.ntiles * static_percent(p.ntiles / grid, elem_bytes(c->storage)) / 100 / grid);
  }
  p.ctr_slot = (int)(c->steps & 1);
  p.stats = c->stats();
  p.nbins = c->nbins;
  p.bins_even = c->nbins > 0 && g.nx % c->nbins == 0 && (g.nx / c->nbins) % 2 == 0;
  p.xc_outer = c->stats_on && c->nbins > 1 && c->sh.nxc > 1;
  p.t_in = p.xc_outer ? p.nzg : p.nxc;
  p.t_mid = p.xc_outer ? p.nxc : p.nzg;
  p.t_in_inv = 1.0f / (float)p.t_in;
  p.t_mid_inv = 1.0f / (float)p.t_mid;
  p.t_fast = p.ntiles < (1ll << 23);
  p.io_one = p.x_io == X_INOUT && g.nx - (c->sh.nxc - 1) * c->sh.xt == 1;
  p.drag_x_only = c->forcing.drag_streamwise_only;
  p.edm = c->forcing.scheme == LBM_FORCE_EXACT_DIFFERENCE;
  p.tau_rho2 = c->forcing.sgs_rho_power == 2;
  p.aa_pitch = c->ash.pitch;
  p.aa_lead = c->ash.lead;
  p.aa_elems = c->aa ? c->ash.elems : 0;
  p.aa_parity = (int)(c->steps & 1);
  p.aa_ub_sum = c->aa && !c->aa_tma;
  if (p.aa_ub_sum) {
    // the one-cell AA kernel's bulk-velocity sums rotate through three slots
    // (written, read, cleared for the next step)
    p.slot_write = (int)(c->steps % 3);
    p.slot_read = (int)((c->steps + 2) % 3);
  }
  if (c->aa) {
    // write offsets of the step's kind from the cell's slot of direction 0:
    // step B (from the swapped layout) slot i at x + c_i, step A slot opp(i)
    const long long ys = c->ash.pitch, zs = (g.ny + 2) * ys, qs = (g.nz + 2) * zs;
    for (int i = 0; i < NQ; i++) {
      const long long shift = (long long)cz(i) * zs + (long long)cy(i) * ys + cx(i);
      p.aa_wr[i] = p.aa_parity == 0 ? (long long)i * qs + shift : (long long)opp(i) * qs;
    }
  }
  p.state = c->state();
  if (c->aa) {
    p.src = p.dst = c->fbuf(0);  // one set, read and written in place
  } else {
    p.src = c->fbuf(c->cur);
    p.dst = c->fbuf(1 - c->cur);
  }
  return p;
}

// Instantiate a functor over the storage type (AA-pattern kernels).
template <typename Fn>
void dispatch_s(const lbm_ctx* c, Fn&& fn) {
  if (c->storage == LBM_F32) fn(std::integral_constant<int, 0>());
  else if (c->storage == LBM_F16_SHIFTED) fn(std::integral_constant<int, 1>());
  else fn(std::integral_constant<int, 2>());
}

// Instantiate a functor over (chunk width, storage type).
template <typename Fn>
void dispatch(const lbm_ctx* c, Fn&& fn) {
  auto by_storage = [&](auto xt) {
    if (c->storage == LBM_F32) fn(xt, std::integral_constant<int, 0>());
    else if (c->storage == LBM_F16_SHIFTED) fn(xt, std::integral_constant<int, 1>());
    else fn(xt, std::integral_constant<int, 2>());
  };
  if (c->sh.xt == 64) by_storage(std::integral_constant<int, 64>());
  else if (c->sh.xt == 128) by_storage(std::integral_constant<int, 128>());
  else by_storage(std::integral_constant<int, 256>());
}

bool uses_variant(const lbm_forcing& f) {
  return f.drag_streamwise_only != 0 || f.scheme == LBM_FORCE_EXACT_DIFFERENCE ||
         f.sgs_rho_power == 2;
}

template <int XT, int S>
void launch_step(const lbm_ctx* c, const StepParams& p, bool stats) {
  // programmatic dependent launch: the blocks of this step may start while the
  // previous step's last blocks finish; the kernel waits (griddepcontrol.wait)
  // before it touches memory the previous step wrote or reads
  Kern<XT, S>::step(dim3(step_grid(c)), c->block, c->stage_smem, c->stream, p, stats,
                    uses_variant(c->forcing), true);
}

// Launch shape and shared-memory stages of a step kernel form: a chunk of XT
// cells per tile row with cpt cells per thread, block_threads(cpt) cpt / XT
// rows (consecutive z) per tile; as many tiles in flight as fit beside three
// blocks per SM and their static shared memory (about 9 KB with statistics):
// at most 8, at least 2 (three with the chunk widths used here).
struct StagePlan {
  dim3 block;
  int nstage;
  size_t smem;
};
template <int XT, int S>
StagePlan stage_plan(int cpt) {
  using St = Stage<XT, S>;
  StagePlan sp;
  const int nt = block_threads(cpt);
  sp.block = dim3(XT / cpt, nt * cpt / XT, 1);
  const size_t stage = (size_t)sp.block.y * NQ * St::SROW * sizeof(typename Store<S>::T);
  const size_t budget = 62 * 1024 * nt / 256;
  sp.nstage = (int)std::max<size_t>(2, std::min<size_t>(8, budget / stage));
  sp.smem = sp.nstage * stage;
  return sp;
}

template <int XT, int S>
void plan_stages(lbm_ctx* c) {
  const bool var = uses_variant(c->forcing);
  const StagePlan def = stage_plan<XT, S>(Kern<XT, S>::cells_per_thread(false));
  const StagePlan vf = stage_plan<XT, S>(Kern<XT, S>::cells_per_thread(true));
  Kern<XT, S>::configure(def.smem, vf.smem);  // per form: the same for every context
  Kern<XT, S>::aa_configure(def.smem);
  const StagePlan& own = var ? vf : def;
  c->block = own.block;
  c->nstage = own.nstage;
  c->stage_smem = own.smem;
  c->nzg = (c->grid.nz + (int)c->block.y - 1) / (int)c->block.y;
}

template <int XT, int S>
int occupancy(const lbm_ctx* c) {
  return Kern<XT, S>::occupancy(c->block, c->stage_smem, uses_variant(c->forcing));
}

// Ghost slots of both population sets from their cells: the current set
// needs all of them; the other keeps the inflow ghosts, which no step
// rewrites (its other ghosts are written by the next step before any read).
template <int XT, int S>
void launch_ghosts(const lbm_ctx* c) {
  StepParams p = make_params(c);
  Kern<XT, S>::ghosts(c->sm_count * 4, c->stream, p, c->fbuf(c->cur));
  Kern<XT, S>::ghosts(c->sm_count * 4, c->stream, p, c->fbuf(1 - c->cur));
}

template <int XT, int S>
void launch_init(const lbm_ctx* c) {
  InitParams ip;
  ip.f = c->fbuf(c->cur);
  ip.nx = c->grid.nx; ip.ny = c->grid.ny; ip.nz = c->grid.nz; ip.nxc = c->sh.nxc;
  ip.u_prof = c->uprof_dev();
  ip.seed = c->seed;
  ip.amp = c->init_perturb;
  Kern<XT, S>::init(c->sm_count * 8, c->stream, ip);
  launch_ghosts<XT, S>(c);
}

template <int XT, int S>
void launch_mass(const lbm_ctx* c) {
  Kern<XT, S>::mass(kMassBlocks, c->stream, c->fbuf(c->cur), c->grid.nx,
                    (long long)c->grid.ny * c->grid.nz, c->sh.nxc, c->mass_buf());
  mass_final_kernel<<<1, 32, 0, c->stream>>>(c->mass_buf(), kMassBlocks, (double)c->cells,
                                              c->mass_buf() + kMassBlocks);
}

template <int XT, int S>
void launch_macro(const lbm_ctx* c, const StepParams& p, float* out) {
  Kern<XT, S>::macro(c->sm_count * 8, c->stream, p, out);
}

// The density and velocity the next step computes, in either layout.
void launch_macro_any(const lbm_ctx* c, const StepParams& p, float* out) {
  if (c->aa)
    dispatch_s(c, [&](auto s) { KernAA<decltype(s)::value>::macro(c->sm_count * 8, c->stream, p, out); });
  else
    dispatch(c, [&](auto xt, auto s) { launch_macro<decltype(xt)::value, decltype(s)::value>(c, p, out); });
}

// The correction's inputs over all first-cell columns into X, and with th
// the network's layer-0 acceleration for the next step from them.
void launch_correction(const lbm_ctx* c, const float* th, float* X) {
  const StepParams p = make_params(c);
  const long long cols = (long long)c->grid.nx * c->grid.nz;
  if (th) {
    // features and network in one pass: resident blocks of four warps, each
    // staging the weights once and taking tiles of 16 columns in turn
    const long long tiles = (cols + 15) / 16;
    dispatch(c, [&](auto xt, auto s) {
      using K = Kern<decltype(xt)::value, decltype(s)::value>;
      const long long resident = (long long)c->sm_count * K::correction_occupancy();
      const int blocks = (int)std::max<long long>(1, std::min<long long>((tiles + 3) / 4, resident));
      K::correction(blocks, c->stream, p, th, c->lam, c->accel());
    });
    return;
  }
  const int fblocks = (int)std::max<long long>(1, std::min<long long>((cols + 255) / 256,
                                                                      (long long)c->sm_count * 16));
  dispatch(c, [&](auto xt, auto s) {
    Kern<decltype(xt)::value, decltype(s)::value>::features(fblocks, c->stream, p, X);
  });
}

// The feature staging buffer (nx*nz rows of 9 floats), allocated on first use.
lbm_status ensure_feat_buf(lbm_ctx* c) {
  if (c->feat_buf) return LBM_OK;
  const size_t cols = (size_t)c->grid.nx * c->grid.nz;
  if (cudaMalloc(&c->feat_buf, sizeof(float) * cols * MLP_IN) != cudaSuccess) {
    cudaGetLastError();
    c->feat_buf = nullptr;
    return fail(c, LBM_ERR_OOM, "cudaMalloc of the correction's feature buffer failed");
  }
  return LBM_OK;
}

lbm_status check_device(lbm_ctx* c) {
  CK(c, cudaStreamSynchronize(c->stream));
  CK(c, cudaGetLastError());
  DevState st;
  CK(c, cudaMemcpy(&st, c->state(), sizeof(st), cudaMemcpyDeviceToHost));
  if (st.bounds_flag) return fail(c, LBM_ERR_BOUNDS, "an index left its buffer (checked build)");
  if (st.timeout_flag)
    return fail(c, LBM_ERR_TIMEOUT, "a device wait gave up after its iteration limit");
  if (st.nan_flag) return fail(c, LBM_ERR_NAN, "a cell produced a non-finite density");
  return LBM_OK;
}

#define READY(c)                                     \
  do {                                               \
    if (!(c)) return LBM_ERR_ARG;                    \
    if ((c)->status != LBM_OK) return LBM_ERR_STATE; \
  } while (0)

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t k = 0; k < n; k++) {
    h ^= p[k];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

extern "C" {

size_t lbm_workspace_bytes(const lbm_grid* grid, int32_t storage, int32_t stats_xbins) {
  if (!grid_ok(grid) || !storage_ok(storage) || stats_xbins < 1 ||
      stats_xbins > MAX_XBINS || stats_xbins > grid->nx)
    return 0;
  if (is_aa(storage) && grid->x_lo == LBM_BC_HALO) return 0;  // slabs use the pull layout
  return layout_of(*grid, storage, stats_xbins).total;
}

}  // extern "C"

namespace {
// lbm_create with an optional chunk width (0: chunk_width(nx)); an ensemble
// lays all its boxes out with one width so one kernel serves them all.
lbm_status create_ctx(const lbm_grid* grid, double tau0, double cs, const double* lad,
                      const lbm_forcing* forcing, int32_t storage, int32_t stats_xbins,
                      uint64_t seed, double init_perturb, void* workspace,
                      size_t workspace_bytes, int xt, cudaStream_t stream, lbm_ctx** out) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (xt != 0 && xt != 64 && xt != 128 && xt != 256) return LBM_ERR_ARG;
  const size_t need = lbm_workspace_bytes(grid, storage, stats_xbins) == 0
                          ? 0
                          : layout_of(*grid, storage, stats_xbins, xt).total;
  if (need == 0 || !forcing || !(tau0 > 0.5) || !(cs >= 0.0) || !std::isfinite(tau0) ||
      !std::isfinite(cs) || !std::isfinite(init_perturb))
    return LBM_ERR_ARG;
  if (forcing->u_bulk_target > 0.0 && !(forcing->ctrl_gain >= 0.0)) return LBM_ERR_ARG;
  if (grid->x_lo == LBM_BC_INFLOW && !forcing->u_in_profile) return LBM_ERR_ARG;
  // a slab of a larger domain: the controller would need the global bulk velocity
  if (grid->x_lo == LBM_BC_HALO && forcing->u_bulk_target > 0.0) return LBM_ERR_ARG;
  if ((forcing->drag_streamwise_only != 0 && forcing->drag_streamwise_only != 1) ||
      (forcing->scheme != LBM_FORCE_GUO && forcing->scheme != LBM_FORCE_EXACT_DIFFERENCE) ||
      forcing->sgs_rho_power < 0 || forcing->sgs_rho_power > 2 || forcing->reserved != 0)
    return LBM_ERR_ARG;
  if (workspace && workspace_bytes < need) return LBM_ERR_OOM;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return LBM_ERR_ARG;

  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_OOM;
  c->grid = *grid;
  c->storage = storage & 0xff;
  c->aa = is_aa(storage);
  c->ash = aa_shape_of(*grid, storage);
  c->nbins = stats_xbins;
  c->tau0 = tau0;
  c->cs = cs;
  c->forcing = *forcing;
  c->forcing.u_in_profile = nullptr;
  if (lad) c->lad.assign(lad, lad + grid->ny);
  c->uprof.assign(grid->ny, 0.0);
  if (forcing->u_in_profile) c->uprof.assign(forcing->u_in_profile, forcing->u_in_profile + grid->ny);
  c->seed = seed;
  c->init_perturb = init_perturb;
  c->sh = shape_of(*grid, storage & 0xff, xt);
  c->cells = (long long)grid->nx * grid->ny * grid->nz;
  c->L = layout_of(*grid, storage, stats_xbins, xt);
  c->stream = stream;

  auto bail = [&](lbm_status s) {
    if (c->owns_ws && c->ws) cudaFree(c->ws);
    delete c;
    return s;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return bail(LBM_ERR_CUDA);
  c->device = dev;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return bail(LBM_ERR_CUDA);
  if (workspace) {
    c->ws = static_cast<char*>(workspace);
  } else {
    if (cudaMalloc(&c->ws, c->L.total) != cudaSuccess) {
      cudaGetLastError();
      c->ws = nullptr;
      return bail(LBM_ERR_OOM);
    }
    c->owns_ws = true;
  }

  // launch shape and stages (plan_stages): per chunk width, storage and model form
  c->aa_tma = c->aa && !uses_variant(c->forcing);
  if (c->aa_tma) {
    dispatch(c, [&](auto xt, auto s) {
      plan_stages<decltype(xt)::value, decltype(s)::value>(c);
      c->blocks_per_sm = Kern<decltype(xt)::value, decltype(s)::value>::aa_occupancy(c->block, c->stage_smem);
    });
  } else if (c->aa) {
    dispatch_s(c, [&](auto s) { c->blocks_per_sm = KernAA<decltype(s)::value>::occupancy(); });
  } else {
    dispatch(c, [&](auto xt, auto s) {
      plan_stages<decltype(xt)::value, decltype(s)::value>(c);
      c->blocks_per_sm = occupancy<decltype(xt)::value, decltype(s)::value>(c);
    });
  }
  if (cudaGetLastError() != cudaSuccess) return bail(LBM_ERR_CUDA);

  // boundary tables and inputs
  std::vector<float> kd(grid->ny, 0.f), la(grid->ny, 0.f), fin((size_t)NQ * grid->ny, 0.f);
  for (int y = 0; y < grid->ny; y++) {
    if (!c->lad.empty()) kd[y] = (float)(forcing->cd * c->lad[y]);
    if (!c->lad.empty()) la[y] = (float)c->lad[y];
    const double u[3] = {c->uprof[y], 0.0, 0.0};
    double fs[NQ];
    feq_shift(u, fs);
    for (int i = 0; i < NQ; i++) fin[(size_t)y * NQ + i] = (float)fs[i];
  }
  if (cudaMemsetAsync(c->ws, 0, c->L.total, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->kdrag(), kd.data(), sizeof(float) * grid->ny, cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->lad_dev(), la.data(), sizeof(float) * grid->ny, cudaMemcpyHostToDevice,
                      c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->feq_in(), fin.data(), sizeof(float) * fin.size(),
                      cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->uprof_dev(), c->uprof.data(), sizeof(double) * grid->ny,
                      cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
    return bail(LBM_ERR_CUDA);
  if (c->aa) {
    InitParams ip{};
    ip.nx = grid->nx; ip.ny = grid->ny; ip.nz = grid->nz;
    ip.u_prof = c->uprof_dev();
    ip.seed = c->seed;
    ip.amp = c->init_perturb;
    const StepParams p = make_params(c);
    dispatch_s(c, [&](auto s) { KernAA<decltype(s)::value>::init(c->sm_count * 8, c->stream, p, ip); });
  } else {
    dispatch(c, [&](auto xt, auto s) { launch_init<decltype(xt)::value, decltype(s)::value>(c); });
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(LBM_ERR_CUDA);
  *out = c;
  return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_grid* grid, double tau0, double cs, const double* lad,
                      const lbm_forcing* forcing, int32_t storage, int32_t stats_xbins,
                      uint64_t seed, double init_perturb, void* workspace,
                      size_t workspace_bytes, lbm_ctx** out) {
  return create_ctx(grid, tau0, cs, lad, forcing, storage, stats_xbins, seed, init_perturb,
                    workspace, workspace_bytes, 0, nullptr, out);
}

lbm_status lbm_set_stream(lbm_ctx* c, void* stream) {
  READY(c);
  CK(c, cudaStreamSynchronize(c->stream));
  c->stream = static_cast<cudaStream_t>(stream);
  return LBM_OK;
}

namespace {
// The launch of one AA step: the boundary fill, then step B (from the
// swapped layout) or A (from the streamed one) with its read and write
// offsets relative to the cell's slot of direction 0.
lbm_status aa_step(lbm_ctx* c) {
  const StepParams p = make_params(c);
  const lbm_grid& g = c->grid;
  AAStep a;
  a.p = p;
  const long long ys = c->ash.pitch, zs = (g.ny + 2) * ys, qs = (g.nz + 2) * zs;
  for (int i = 0; i < NQ; i++) {
    const long long own = (long long)i * qs, rev = (long long)opp(i) * qs;
    const long long shift = (long long)cz(i) * zs + (long long)cy(i) * ys + cx(i);
    if (p.aa_parity == 0) {  // B
      a.rd[i] = rev - shift;
      a.wr[i] = own + shift;
    } else {  // A
      a.rd[i] = own;
      a.wr[i] = rev;
    }
  }
  a.nxc = (g.nx + AA_XT - 1) / AA_XT;
  a.nzg = (g.nz + AA_ZR - 1) / AA_ZR;
  a.nunit = a.nxc * a.nzg * g.ny;
  a.xc_outer = c->stats_on && c->nbins > 1 && a.nxc > 1;
  const int grid = (int)std::max<long long>(1, std::min<long long>(a.nunit, (long long)c->sm_count * c->blocks_per_sm));
  if (c->aa_tma) {
    // the boundary fill, then the step on the tile pipeline (both
    // programmatic dependents of the kernel before them)
    dispatch(c, [&](auto xt, auto s) {
      KernAA<decltype(s)::value>::fill(c->stream, p);
      Kern<decltype(xt)::value, decltype(s)::value>::aa_step(dim3(step_grid(c)), c->block, c->stage_smem,
                                                             c->stream, p, c->stats_on);
    });
    CK(c, cudaGetLastError());
    c->last_grid = step_grid(c);
    c->steps++;
    if (c->stats_on) c->stats_samples++;
    return LBM_OK;
  }
  dispatch_s(c, [&](auto s) {
    KernAA<decltype(s)::value>::fill(c->stream, p);
    KernAA<decltype(s)::value>::step(grid, c->stream, a, c->stats_on, uses_variant(c->forcing));
  });
  CK(c, cudaGetLastError());
  c->steps++;
  if (c->stats_on) c->stats_samples++;
  return LBM_OK;
}
}  // namespace

lbm_status lbm_step(lbm_ctx* c, int32_t n) {
  READY(c);
  if (n < 0) return arg_error(c, "lbm_step: n < 0");
  if (c->aa) {
    for (int32_t k = 0; k < n; k++) {
      const lbm_status s = aa_step(c);
      if (s != LBM_OK) return s;
    }
    return LBM_OK;
  }
  for (int32_t k = 0; k < n; k++) {
    const StepParams p = make_params(c);
    dispatch(c, [&](auto xt, auto s) {
      launch_step<decltype(xt)::value, decltype(s)::value>(c, p, c->stats_on);
    });
    CK(c, cudaGetLastError());
    c->test_withhold = -1;  // a test hook acts on one step
    c->last_grid = step_grid(c);
    c->cur = 1 - c->cur;
    c->steps++;
    if (c->stats_on) c->stats_samples++;
    if (c->mlp) {
      // the next step's layer-0 acceleration from the new state
      launch_correction(c, c->mlp->theta, c->feat_buf);
      CK(c, cudaGetLastError());
    }
  }
  return LBM_OK;
}

lbm_status lbm_test_withhold_fill(lbm_ctx* c, int32_t fill) {
  READY(c);
  if (fill < 0) return arg_error(c, "lbm_test_withhold_fill: fill < 0");
  if (c->aa) return arg_error(c, "lbm_test_withhold_fill: the AA layout has no tile fills");
  c->test_withhold = fill;
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
  READY(c);
  return check_device(c);
}

lbm_status lbm_stats_reset(lbm_ctx* c, int32_t enable) {
  READY(c);
  CK(c, cudaMemsetAsync(c->stats(), 0, sizeof(double) * 9 * c->nbins * c->grid.ny, c->stream));
  c->stats_on = enable != 0;
  c->stats_samples = 0;
  return LBM_OK;
}

namespace {

size_t readout_bytes(const lbm_ctx* c) { return c->L.state_off + sizeof(DevState) - c->L.stats_off; }

// pinned read-out slots (three, allocated on first use)
lbm_status ensure_readout(lbm_ctx* c, const char* who) {
  if (c->readout) return LBM_OK;
  const size_t slot = align_up(readout_bytes(c), kAlign);
  if (cudaMallocHost(&c->readout, 3 * slot) != cudaSuccess) {
    cudaGetLastError();
    c->readout = nullptr;
    return fail(c, LBM_ERR_OOM, std::string(who) + ": cudaMallocHost of the readout buffer failed");
  }
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->readout_dev), c->readout, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(c->readout);
    c->readout = nullptr;
    c->readout_dev = nullptr;
    return fail(c, LBM_ERR_CUDA, std::string(who) + ": the readout buffer has no device address");
  }
  return LBM_OK;
}

unsigned char* readout_slot(const lbm_ctx* c, int k) {
  return c->readout + (size_t)k * align_up(readout_bytes(c), kAlign);
}

// Health flags and the averages of one read-out slot.
lbm_status finish_readout(lbm_ctx* c, const unsigned char* buf, int64_t nsamples, double* out,
                          int64_t* samples) {
  const int ny = c->grid.ny, nb = c->nbins, nx = c->grid.nx;
  const size_t m = (size_t)nb * ny;
  const DevState* st = reinterpret_cast<const DevState*>(buf + (c->L.state_off - c->L.stats_off));
  if (st->bounds_flag) return fail(c, LBM_ERR_BOUNDS, "an index left its buffer (checked build)");
  if (st->timeout_flag)
    return fail(c, LBM_ERR_TIMEOUT, "a device wait gave up after its iteration limit");
  if (st->nan_flag) return fail(c, LBM_ERR_NAN, "a cell produced a non-finite density");
  const double* acc = reinterpret_cast<const double*>(buf);
  std::vector<long long> width(nb, 0);
  for (int x = 0; x < nx; x++) width[(long long)x * nb / nx]++;
  for (int b = 0; b < nb; b++)
    for (int y = 0; y < ny; y++) {
      const size_t k = (size_t)b * ny + y;
      const double cnt = (double)nsamples * (double)c->grid.nz * (double)width[b];
      const double inv = cnt > 0 ? 1.0 / cnt : 0.0;
      const double mu = acc[0 * m + k] * inv, mv = acc[1 * m + k] * inv, mw = acc[2 * m + k] * inv;
      out[0 * m + k] = mu;
      out[1 * m + k] = mv;
      out[2 * m + k] = mw;
      out[3 * m + k] = acc[3 * m + k] * inv - mu * mu;
      out[4 * m + k] = acc[4 * m + k] * inv - mv * mv;
      out[5 * m + k] = acc[5 * m + k] * inv - mw * mw;
      out[6 * m + k] = acc[6 * m + k] * inv - mu * mv;
      out[7 * m + k] = acc[7 * m + k] * inv - mu * mw;
      out[8 * m + k] = acc[8 * m + k] * inv - mv * mw;
    }
  if (samples) *samples = nsamples;
  return LBM_OK;
}

}  // namespace

lbm_status lbm_stats(lbm_ctx* c, double* out, size_t n, int64_t* samples) {
  READY(c);
  if (!out || n < 9 * (size_t)c->nbins * c->grid.ny) return arg_error(c, "lbm_stats: output too small");
  lbm_status s = ensure_readout(c, "lbm_stats");
  if (s != LBM_OK) return s;
  // one asynchronous copy of the statistics and the health flags (adjacent in
  // the workspace) into pinned memory, then one wait on the context's stream
  CK(c, cudaMemcpyAsync(readout_slot(c, 0), c->ws + c->L.stats_off, readout_bytes(c),
                        cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  CK(c, cudaGetLastError());
  return finish_readout(c, readout_slot(c, 0), c->stats_samples, out, samples);
}

lbm_status lbm_stats_begin(lbm_ctx* c) {
  READY(c);
  if (c->rd_pending == 2) return arg_error(c, "lbm_stats_begin: two read-outs already pending");
  lbm_status s = ensure_readout(c, "lbm_stats_begin");
  if (s != LBM_OK) return s;
  const int k = (c->rd_first + c->rd_pending) & 1;
  if (!c->rd_ev[k]) CK(c, cudaEventCreateWithFlags(&c->rd_ev[k], cudaEventDisableTiming));
  {
    // the read-out kernel (a programmatic dependent of the step before it)
    // writes the slot through the pinned buffer's device address
    static_assert(sizeof(DevState) % 16 == 0 && kAlign % 16 == 0, "the read-out moves 16-byte words");
    const long long n16 = (long long)(readout_bytes(c) / 16);
    const size_t slot = (size_t)(readout_slot(c, 1 + k) - c->readout);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)std::max<long long>(1, std::min<long long>((n16 + 255) / 256, 148)));
    cfg.blockDim = dim3(256);
    cfg.stream = c->stream;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(c, cudaLaunchKernelEx(&cfg, readout_kernel, reinterpret_cast<const uint4*>(c->ws + c->L.stats_off),
                             reinterpret_cast<uint4*>(c->readout_dev + slot), n16));
  }
  CK(c, cudaEventRecord(c->rd_ev[k], c->stream));
  c->rd_samples[k] = c->stats_samples;
  c->rd_pending++;
  return LBM_OK;
}

lbm_status lbm_stats_end(lbm_ctx* c, double* out, size_t n, int64_t* samples) {
  READY(c);
  if (c->rd_pending == 0) return arg_error(c, "lbm_stats_end: no read-out pending");
  if (!out || n < 9 * (size_t)c->nbins * c->grid.ny)
    return arg_error(c, "lbm_stats_end: output too small");
  const int k = c->rd_first;
  CK(c, cudaEventSynchronize(c->rd_ev[k]));
  CK(c, cudaGetLastError());
  c->rd_first ^= 1;
  c->rd_pending--;
  return finish_readout(c, readout_slot(c, 1 + k), c->rd_samples[k], out, samples);
}

lbm_status lbm_mass(lbm_ctx* c, double* out) {
  READY(c);
  if (!out) return arg_error(c, "lbm_mass: out is NULL");
  if (c->aa) {
    const StepParams p = make_params(c);
    dispatch_s(c, [&](auto s) { KernAA<decltype(s)::value>::mass(kMassBlocks, c->stream, p, c->mass_buf()); });
    mass_final_kernel<<<1, 32, 0, c->stream>>>(c->mass_buf(), kMassBlocks, (double)c->cells,
                                                c->mass_buf() + kMassBlocks);
  } else {
    dispatch(c, [&](auto xt, auto s) { launch_mass<decltype(xt)::value, decltype(s)::value>(c); });
  }
  CK(c, cudaGetLastError());
  lbm_status s = check_device(c);
  if (s != LBM_OK) return s;
  CK(c, cudaMemcpy(out, c->mass_buf() + kMassBlocks, sizeof(double), cudaMemcpyDeviceToHost));
  return LBM_OK;
}

lbm_status lbm_get_f(lbm_ctx* c, double* host, size_t n) {
  READY(c);
  if (!host || n != (size_t)NQ * c->cells) return arg_error(c, "lbm_get_f: wrong size");
  lbm_status s = check_device(c);
  if (s != LBM_OK) return s;
  const size_t eb = elem_bytes(c->storage);
  std::vector<unsigned char> raw((size_t)c->set_elems() * eb);
  CK(c, cudaMemcpy(raw.data(), c->fbuf(c->cur), raw.size(), cudaMemcpyDeviceToHost));
  const lbm_grid& g = c->grid;
  for (int i = 0; i < NQ; i++)
    for (int z = 0; z < g.nz; z++)
      for (int y = 0; y < g.ny; y++)
        for (int x = 0; x < g.nx; x++) {
          const size_t dk = (size_t)c->dev_index(i, x, y, z);
          double v;
          if (c->storage == LBM_F32) v = reinterpret_cast<const float*>(raw.data())[dk];
          else if (c->storage == LBM_F16_SHIFTED)
            v = __half2float(reinterpret_cast<const __half*>(raw.data())[dk]);
          else v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(raw.data())[dk]);
          host[(((size_t)i * g.nz + z) * g.ny + y) * g.nx + x] = wgt_d(i) + v;
        }
  return LBM_OK;
}

lbm_status lbm_set_f(lbm_ctx* c, const double* host, size_t n) {
  READY(c);
  if (!host || n != (size_t)NQ * c->cells) return arg_error(c, "lbm_set_f: wrong size");
  CK(c, cudaStreamSynchronize(c->stream));
  const size_t eb = elem_bytes(c->storage);
  std::vector<unsigned char> raw((size_t)c->set_elems() * eb, 0);
  const lbm_grid& g = c->grid;
  for (int i = 0; i < NQ; i++)
    for (int z = 0; z < g.nz; z++)
      for (int y = 0; y < g.ny; y++)
        for (int x = 0; x < g.nx; x++) {
          const size_t dk = (size_t)c->dev_index(i, x, y, z);
          const double v = host[(((size_t)i * g.nz + z) * g.ny + y) * g.nx + x] - wgt_d(i);
          if (c->storage == LBM_F32) reinterpret_cast<float*>(raw.data())[dk] = (float)v;
          else if (c->storage == LBM_F16_SHIFTED)
            reinterpret_cast<__half*>(raw.data())[dk] = Store<1>::from_double(v);
          else reinterpret_cast<__nv_bfloat16*>(raw.data())[dk] = Store<2>::from_double(v);
        }
  CK(c, cudaMemcpy(c->fbuf(c->cur), raw.data(), raw.size(), cudaMemcpyHostToDevice));
  // (AA: the slots a step reads from outside the domain are filled before each step)
  if (!c->aa)
    dispatch(c, [&](auto xt, auto s) { launch_ghosts<decltype(xt)::value, decltype(s)::value>(c); });
  CK(c, cudaGetLastError());
  CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_get_macro(lbm_ctx* c, double* rho, double* u, size_t n) {
  READY(c);
  if (!rho || !u || n != (size_t)c->cells) return arg_error(c, "lbm_get_macro: wrong size");
  if (!c->macro_buf) {
    if (cudaMalloc(&c->macro_buf, sizeof(float) * 4 * c->cells) != cudaSuccess) {
      cudaGetLastError();
      c->macro_buf = nullptr;
      return fail(c, LBM_ERR_OOM, "lbm_get_macro: cudaMalloc of the field buffer failed");
    }
  }
  const StepParams p = make_params(c);
  launch_macro_any(c, p, c->macro_buf);
  CK(c, cudaGetLastError());
  lbm_status s = check_device(c);
  if (s != LBM_OK) return s;
  std::vector<float> h((size_t)4 * c->cells);
  CK(c, cudaMemcpy(h.data(), c->macro_buf, sizeof(float) * h.size(), cudaMemcpyDeviceToHost));
  for (long long k = 0; k < c->cells; k++) rho[k] = h[k];
  for (long long k = 0; k < 3 * c->cells; k++) u[k] = h[c->cells + k];
  return LBM_OK;
}

lbm_status lbm_get_q(lbm_ctx* c, double* q, size_t n) {
  READY(c);
  if (!q || n != (size_t)c->cells) return arg_error(c, "lbm_get_q: wrong size");
  if (!c->macro_buf) {
    if (cudaMalloc(&c->macro_buf, sizeof(float) * 4 * c->cells) != cudaSuccess) {
      cudaGetLastError();
      c->macro_buf = nullptr;
      return fail(c, LBM_ERR_OOM, "lbm_get_q: cudaMalloc of the field buffer failed");
    }
  }
  const StepParams p = make_params(c);
  launch_macro_any(c, p, c->macro_buf);
  // Q into the density plane of the field buffer (the kernel reads the velocity planes only)
  const lbm_grid& g = c->grid;
  q_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(c->macro_buf + c->cells, c->macro_buf, g.nx,
                                                   g.ny, g.nz, g.x_lo == LBM_BC_PERIODIC,
                                                   g.y_lo == LBM_BC_PERIODIC);
  CK(c, cudaGetLastError());
  lbm_status s = check_device(c);
  if (s != LBM_OK) return s;
  std::vector<float> h((size_t)c->cells);
  CK(c, cudaMemcpy(h.data(), c->macro_buf, sizeof(float) * h.size(), cudaMemcpyDeviceToHost));
  for (long long k = 0; k < c->cells; k++) q[k] = h[k];
  return LBM_OK;
}

lbm_status lbm_drive(lbm_ctx* c, double g[3], double* u_bulk) {
  READY(c);
  if (!g || !u_bulk) return arg_error(c, "lbm_drive: NULL output");
  lbm_status s = check_device(c);
  if (s != LBM_OK) return s;
  double ub = 0.0;
  if (c->steps > 0 && c->aa && !c->aa_tma) {  // one exact sum per step, three slots in rotation
    long long sum = 0;
    CK(c, cudaMemcpy(&sum, c->ub_part() + (size_t)((c->steps + 2) % 3), sizeof(long long),
                     cudaMemcpyDeviceToHost));
    ub = (double)sum / 4294967296.0 / (double)c->cells;
  } else if (c->steps > 0) {
    std::vector<long long> part(c->last_grid);
    CK(c, cudaMemcpy(part.data(), c->ub_part() + (size_t)((c->steps + 1) % 2) * MAX_BLOCKS,
                     sizeof(long long) * part.size(), cudaMemcpyDeviceToHost));
    long long sum = 0;
    for (long long v : part) sum += v;
    ub = (double)sum / 4294967296.0 / (double)c->cells;
  }
  for (int a = 0; a < 3; a++) g[a] = c->forcing.g[a];
  if (c->forcing.u_bulk_target > 0.0 && c->steps > 0)
    g[0] = c->forcing.g[0] + c->forcing.ctrl_gain * (c->forcing.u_bulk_target - ub);
  *u_bulk = ub;
  return LBM_OK;
}

// ---- x-slab halo exchange -------------------------------------------------------------
size_t lbm_halo_bytes(const lbm_ctx* c) {
  if (!c || c->grid.x_lo != LBM_BC_HALO) return 0;
  return (size_t)5 * c->grid.ny * c->grid.nz * elem_bytes(c->storage);
}

namespace {
lbm_status halo_call(lbm_ctx* c, const void* lo, const void* hi, bool pack, const char* who) {
  if (c->grid.x_lo != LBM_BC_HALO) return arg_error(c, std::string(who) + ": the context has no halo faces");
  if (!lo || !hi) return arg_error(c, std::string(who) + ": NULL face buffer");
  if ((reinterpret_cast<uintptr_t>(lo) | reinterpret_cast<uintptr_t>(hi)) % 16 != 0)
    return arg_error(c, std::string(who) + ": face buffers must be 16-byte aligned");
  const StepParams p = make_params(c);
  const long long n = 10ll * c->grid.ny * c->grid.nz;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, c->sm_count * 4ll));
  dispatch(c, [&](auto xt, auto s) {
    using K = Kern<decltype(xt)::value, decltype(s)::value>;
    if (pack) K::halo_pack(blocks, c->stream, p, c->fbuf(c->cur), const_cast<void*>(lo), const_cast<void*>(hi));
    else K::halo_unpack(blocks, c->stream, p, c->fbuf(c->cur), lo, hi);
  });
  CK(c, cudaGetLastError());
  return LBM_OK;
}
}  // namespace

lbm_status lbm_halo_pack(lbm_ctx* c, void* to_lo, void* to_hi) {
  READY(c);
  return halo_call(c, to_lo, to_hi, true, "lbm_halo_pack");
}

lbm_status lbm_halo_unpack(lbm_ctx* c, const void* from_lo, const void* from_hi) {
  READY(c);
  return halo_call(c, from_lo, from_hi, false, "lbm_halo_unpack");
}

// ---- checkpoint ----------------------------------------------------------------------
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version, storage, nbins, pad;
  lbm_grid grid;
  int64_t steps, stats_samples;
  int32_t stats_on, last_grid;
  uint64_t payload_bytes, checksum;
};
}  // namespace

lbm_status lbm_save(lbm_ctx* c, const char* path) {
  READY(c);
  if (!path) return arg_error(c, "lbm_save: path is NULL");
  lbm_status s = check_device(c);
  if (s != LBM_OK) return s;
  const size_t fb = (size_t)c->set_elems() * elem_bytes(c->storage);
  const size_t sb = sizeof(double) * 9 * c->nbins * c->grid.ny;
  const size_t ub = sizeof(long long) * 2 * MAX_BLOCKS;
  std::vector<unsigned char> payload(fb + sb + ub);
  CK(c, cudaMemcpy(payload.data(), c->fbuf(c->cur), fb, cudaMemcpyDeviceToHost));
  CK(c, cudaMemcpy(payload.data() + fb, c->stats(), sb, cudaMemcpyDeviceToHost));
  CK(c, cudaMemcpy(payload.data() + fb + sb, c->ub_part(), ub, cudaMemcpyDeviceToHost));
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "LBMB300\0", 8);
  h.version = 3;
  h.storage = c->storage | (c->aa ? LBM_STORAGE_AA : 0);
  h.nbins = c->nbins;
  h.grid = c->grid;
  h.steps = c->steps;
  h.stats_samples = c->stats_samples;
  h.stats_on = c->stats_on;
  h.last_grid = c->last_grid;
  h.payload_bytes = payload.size();
  h.checksum = fnv1a(payload.data(), payload.size());
  FILE* fp = std::fopen(path, "wb");
  if (!fp) {
    c->err = std::string("lbm_save: cannot open ") + path;
    return LBM_ERR_IO;
  }
  const bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 &&
                  std::fwrite(payload.data(), 1, payload.size(), fp) == payload.size();
  const bool closed = std::fclose(fp) == 0;
  if (!ok || !closed) {
    c->err = "lbm_save: write failed";
    return LBM_ERR_IO;
  }
  return LBM_OK;
}

lbm_status lbm_load(lbm_ctx* c, const char* path) {
  READY(c);
  if (!path) return arg_error(c, "lbm_load: path is NULL");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) {
    c->err = std::string("lbm_load: cannot open ") + path;
    return LBM_ERR_IO;
  }
  CkptHeader h;
  const size_t fb = (size_t)c->set_elems() * elem_bytes(c->storage);
  const size_t sb = sizeof(double) * 9 * c->nbins * c->grid.ny;
  const size_t ub = sizeof(long long) * 2 * MAX_BLOCKS;
  std::vector<unsigned char> payload;
  bool ok = std::fread(&h, sizeof(h), 1, fp) == 1 && std::memcmp(h.magic, "LBMB300\0", 8) == 0 &&
            h.version == 3 && h.storage == (c->storage | (c->aa ? LBM_STORAGE_AA : 0)) &&
            h.nbins == c->nbins &&
            std::memcmp(&h.grid, &c->grid, sizeof(lbm_grid)) == 0 &&
            h.payload_bytes == fb + sb + ub && h.last_grid >= 0 && h.last_grid <= MAX_BLOCKS;
  if (ok) {
    payload.resize(h.payload_bytes);
    ok = std::fread(payload.data(), 1, payload.size(), fp) == payload.size() &&
         fnv1a(payload.data(), payload.size()) == h.checksum;
  }
  std::fclose(fp);
  if (!ok) {
    c->err = "lbm_load: header mismatch, truncated file or checksum error";
    return LBM_ERR_IO;
  }
  CK(c, cudaStreamSynchronize(c->stream));
  CK(c, cudaMemcpy(c->fbuf(0), payload.data(), fb, cudaMemcpyHostToDevice));
  CK(c, cudaMemcpy(c->stats(), payload.data() + fb, sb, cudaMemcpyHostToDevice));
  CK(c, cudaMemcpy(c->ub_part(), payload.data() + fb + sb, ub, cudaMemcpyHostToDevice));
  CK(c, cudaMemset(c->state()->tile_ctr, 0, sizeof(DevState::tile_ctr)));  // fresh tile counters
  c->cur = 0;
  c->steps = h.steps;
  c->stats_samples = h.stats_samples;
  c->stats_on = h.stats_on != 0;
  c->last_grid = h.last_grid;
  return LBM_OK;
}

// ---- field readout without allocation -------------------------------------------------
// lbm_get_macro stages the fields in a device buffer it allocates on first use.
// Callers that must not allocate device memory (a process running inside a
// strict memory budget or a pre-reserved pool, code that may not call
// cudaMalloc while other work is being captured or timed) use this variant:
// the fields go through a file-scope device array of fixed size instead.
namespace {
constexpr long long kNoAllocMaxCells = 262144;  // 64^3 cells; 8 MB of FP64 on every device
__device__ __align__(256) double g_noalloc_fields[4 * kNoAllocMaxCells];
constexpr int kMaxDevices = 64;
// device address of the array, per device; threads that race on the first
// call all store the same value
std::atomic<double*> g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

lbm_status lbm_get_macro_noalloc(lbm_ctx* c, double* rho, double* u, size_t n) {
  READY(c);
  if (!rho || !u || n != (size_t)c->cells) return arg_error(c, "lbm_get_macro_noalloc: wrong size");
  if (c->cells > kNoAllocMaxCells)
    return arg_error(c, "lbm_get_macro_noalloc: the grid has more than 262144 cells, the size of "
                        "its static field buffer; use lbm_get_macro");
  int dev = 0;
  CK(c, cudaGetDevice(&dev));
  if (dev != c->device)
    return arg_error(c, "lbm_get_macro_noalloc: make the context's device the current device");
  if (dev < 0 || dev >= kMaxDevices) return arg_error(c, "lbm_get_macro_noalloc: device id out of range");
  double* buf = g_noalloc_ptr[dev].load();
  if (!buf) {
    // first call on this device: look up the array's device address (the
    // symbol itself is only a host-side stand-in)
    void* ptr = nullptr;
    CK(c, cudaGetSymbolAddress(&ptr, g_noalloc_fields));
    buf = static_cast<double*>(ptr);
    g_noalloc_ptr[dev].store(buf);
  }
  const StepParams p = make_params(c);
  if (c->aa)
    dispatch_s(c, [&](auto s) { KernAA<decltype(s)::value>::macro_d(c->sm_count * 8, c->stream, p, buf); });
  else
    dispatch(c, [&](auto xt, auto s) {
      Kern<decltype(xt)::value, decltype(s)::value>::macro_d(c->sm_count * 8, c->stream, p, buf);
    });
  CK(c, cudaGetLastError());
  lbm_status s = check_device(c);
  if (s != LBM_OK) return s;
  CK(c, cudaMemcpy(rho, buf, sizeof(double) * c->cells, cudaMemcpyDeviceToHost));
  CK(c, cudaMemcpy(u, buf + c->cells, sizeof(double) * 3 * c->cells, cudaMemcpyDeviceToHost));
  return LBM_OK;
}

int64_t lbm_steps_done(const lbm_ctx* c) { return c ? c->steps : -1; }

void lbm_destroy(lbm_ctx* c) {
  if (!c || c->batch) return;  // boxes of an ensemble go with lbm_batch_destroy
  cudaStreamSynchronize(c->stream);
  if (c->macro_buf) cudaFree(c->macro_buf);
  if (c->feat_buf) cudaFree(c->feat_buf);
  if (c->readout) cudaFreeHost(c->readout);
  for (cudaEvent_t e : c->rd_ev)
    if (e) cudaEventDestroy(e);
  if (c->owns_ws && c->ws) cudaFree(c->ws);
  delete c;
}

const char* lbm_last_error(const lbm_ctx* c) {
  if (!c) return "no context";
  return c->err.c_str();
}

const char* lbm_status_string(int32_t s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_OOM: return "out of memory";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_NAN: return "non-finite value in the flow field";
    case LBM_ERR_TIMEOUT: return "device wait timed out";
    case LBM_ERR_STATE: return "context holds an earlier error";
    case LBM_ERR_IO: return "checkpoint I/O error";
    case LBM_ERR_BOUNDS: return "index out of its buffer (checked build)";
    default: return "unknown status";
  }
}

}  // extern "C"

// ---- ensembles of independent boxes ----------------------------------------------------
struct lbm_batch {
  std::vector<lbm_ctx*> boxes;
  int storage = 0, nbins = 1, xt = 0;
  cudaStream_t stream = nullptr;   // the boxes' stream; graphs are launched on it
  cudaStream_t capture = nullptr;  // private stream the graphs are captured on
  cudaStream_t branch[2] = {nullptr, nullptr};  // the second and third chains' launches
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
  char* ws = nullptr;
  bool owns_ws = false;
  std::vector<BatchWork> work;   // in chains of boxes of one chunk width (64, 128, 256)
  int group_off[4] = {0, 0, 0, 0};  // work items of chain g: [group_off[g], group_off[g + 1])
  BatchWork* work_dev = nullptr;
  double tuned_ms = 0.0;
  std::vector<double> tried;      // tuner record: (chunk width, blocks, ms per step) per candidate
  struct Graph {
    int n = 0;
    bool stats = false;
    std::vector<int> cur;         // each box's population set when the graph starts
    StepParams* params = nullptr; // [2][nbox] device parameters, even / odd steps
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<Graph> graphs;      // most recent last
  std::string err;
};

namespace {

// chunk widths the tuner tries: one for every box, or 0: each box its own
// (the size rule of a single domain, chunk_width(nx))
constexpr int kBatchChunks[4] = {64, 128, 256, 0};
constexpr int kChunkWidths[3] = {64, 128, 256};

size_t batch_box_bytes(const lbm_box& b, int storage, int nbins, int xt) {
  return align_up(layout_of(b.grid, storage, nbins, xt).total, kAlign);
}

bool batch_args_ok(int32_t nbox, const lbm_box* boxes, int32_t storage, int32_t nbins) {
  if (nbox < 1 || !boxes || storage < 0 || storage > 2) return false;
  for (int i = 0; i < nbox; i++) {
    if (lbm_workspace_bytes(&boxes[i].grid, storage, nbins) == 0) return false;
    if (boxes[i].forcing.u_bulk_target > 0.0) return false;
    // the ensemble kernel runs the default model on whole boxes
    if (uses_variant(boxes[i].forcing) || boxes[i].grid.x_lo == LBM_BC_HALO) return false;
  }
  return true;
}

void free_streams(lbm_batch* b) {
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->fork) cudaEventDestroy(b->fork);
  for (int j = 0; j < 2; j++) {
    if (b->branch[j]) cudaStreamDestroy(b->branch[j]);
    if (b->join[j]) cudaEventDestroy(b->join[j]);
  }
}

void free_graphs(lbm_batch* b) {
  for (auto& g : b->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.params) cudaFree(g.params);
  }
  b->graphs.clear();
}

void free_boxes(lbm_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_graphs(b);
  for (lbm_ctx* c : b->boxes) {
    if (!c) continue;
    c->batch = nullptr;
    lbm_destroy(c);
  }
  b->boxes.clear();
  if (b->work_dev) cudaFree(b->work_dev);
  b->work_dev = nullptr;
}

// Boxes with chunk width xt in the ensemble's workspace (or their own memory).
lbm_status make_boxes(lbm_batch* b, int32_t nbox, const lbm_box* boxes, double init_perturb,
                      int xt) {
  size_t off = 0;
  for (int i = 0; i < nbox; i++) {
    const lbm_box& x = boxes[i];
    const size_t bytes = batch_box_bytes(x, b->storage, b->nbins, xt);
    lbm_ctx* c = nullptr;
    const lbm_status s =
        create_ctx(&x.grid, x.tau0, x.cs, x.lad, &x.forcing, b->storage, b->nbins, x.seed,
                   init_perturb, b->ws ? b->ws + off : nullptr, b->ws ? bytes : 0, xt, b->stream, &c);
    if (s != LBM_OK) {
      b->err = "lbm_batch_create: box " + std::to_string(i) + ": " + lbm_status_string(s);
      return s;
    }
    c->batch = b;
    b->boxes.push_back(c);
    off += bytes;
  }
  b->xt = xt;
  return LBM_OK;
}

// Work items: every box's tiles cut into runs of about `per` tiles, one run
// per block, in chains (one launch per chain and step): the boxes of one
// chunk width form a chain; when all boxes share one width, alternate boxes
// form two chains, so that the graph's independent chains overlap each
// other's launch tails.
lbm_status make_work(lbm_batch* b, int waves) {
  long long total = 0;
  for (lbm_ctx* c : b->boxes) total += make_params(c).ntiles;
  const lbm_ctx* c0 = b->boxes[0];
  const long long resident = (long long)c0->sm_count * std::max(1, c0->blocks_per_sm);
  const long long per = std::max<long long>(1, (total + waves * resident - 1) / (waves * resident));
  int widths = 0;
  for (int g = 0; g < 3; g++)
    for (const lbm_ctx* c : b->boxes)
      if (c->sh.xt == kChunkWidths[g]) {
        widths++;
        break;
      }
  const int halves = widths == 1 && b->boxes.size() > 1 ? 2 : 1;
  b->work.clear();
  int nch = 0;
  for (int g = 0; g < 3; g++) {
    for (int h = 0; h < halves; h++) {
      b->group_off[nch] = (int)b->work.size();
      int rank = 0;
      for (int i = 0; i < (int)b->boxes.size(); i++) {
        if (b->boxes[i]->sh.xt != kChunkWidths[g] || (rank++ % halves) != h) continue;
        const long long nt = make_params(b->boxes[i]).ntiles;
        const long long items = (nt + per - 1) / per;
        for (long long k = 0; k < items; k++) {
          BatchWork w;
          w.box = i;
          w.t0 = k * nt / items;
          w.ntile = (int)((k + 1) * nt / items - w.t0);
          b->work.push_back(w);
        }
      }
      if ((int)b->work.size() > b->group_off[nch]) nch++;
    }
  }
  for (int g = nch; g < 4; g++) b->group_off[g] = (int)b->work.size();
  if (b->work_dev) cudaFree(b->work_dev);
  b->work_dev = nullptr;
  free_graphs(b);
  if (cudaMalloc(&b->work_dev, sizeof(BatchWork) * b->work.size()) != cudaSuccess) {
    cudaGetLastError();
    b->err = "lbm_batch: cudaMalloc of the work list failed";
    return LBM_ERR_OOM;
  }
  if (cudaMemcpy(b->work_dev, b->work.data(), sizeof(BatchWork) * b->work.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    b->err = "lbm_batch: copy of the work list failed";
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}

// The graph of n launches starting from the boxes' current population sets.
lbm_status batch_graph(lbm_batch* b, int n, bool stats, cudaGraphExec_t* exec) {
  const int nb = (int)b->boxes.size();
  std::vector<int> cur(nb);
  for (int i = 0; i < nb; i++) cur[i] = b->boxes[i]->cur;
  for (auto& g : b->graphs)
    if (g.n == n && g.stats == stats && g.cur == cur) {
      *exec = g.exec;
      return LBM_OK;
    }
  if (b->graphs.size() >= 4) {  // keep the cache small
    if (b->graphs.front().exec) cudaGraphExecDestroy(b->graphs.front().exec);
    if (b->graphs.front().params) cudaFree(b->graphs.front().params);
    b->graphs.erase(b->graphs.begin());
  }
  lbm_batch::Graph g;
  g.n = n;
  g.stats = stats;
  g.cur = cur;
  std::vector<StepParams> hp(2 * (size_t)nb);
  for (int i = 0; i < nb; i++) {
    lbm_ctx* c = b->boxes[i];
    hp[i] = make_params(c);
    c->cur = 1 - c->cur;
    hp[nb + i] = make_params(c);
    c->cur = 1 - c->cur;
  }
  if (cudaMalloc(&g.params, sizeof(StepParams) * hp.size()) != cudaSuccess) {
    cudaGetLastError();
    b->err = "lbm_batch_step: cudaMalloc of the box parameters failed";
    return LBM_ERR_OOM;
  }
  if (cudaMemcpy(g.params, hp.data(), sizeof(StepParams) * hp.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    cudaFree(g.params);
    b->err = "lbm_batch_step: copy of the box parameters failed";
    return LBM_ERR_CUDA;
  }
  // one box of each chain: its kernel form, block shape and stages
  const lbm_ctx* rep[3] = {nullptr, nullptr, nullptr};
  for (int gi = 0; gi < 3; gi++)
    if (b->group_off[gi + 1] > b->group_off[gi]) rep[gi] = b->boxes[b->work[b->group_off[gi]].box];
  cudaGraph_t graph = nullptr;
  cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaError_t e = cudaStreamBeginCapture(b->capture, mode);
  if (e == cudaSuccess) {
    // The chains hold different boxes, so each is a sequence of n launches
    // of its own: the first on the capture stream, the others on branches
    // forked from it and joined at the end, which the graph runs side by side
    // (one chain's launch tail overlaps another chain's launch).
    cudaStream_t sg[3] = {nullptr, nullptr, nullptr};
    int nbr = 0;
    for (int gi = 0; gi < 3; gi++) {
      if (!rep[gi]) continue;
      sg[gi] = nbr == 0 ? b->capture : b->branch[nbr - 1];
      nbr++;
    }
    cudaError_t ef = cudaSuccess;
    if (nbr > 1) {
      ef = cudaEventRecord(b->fork, b->capture);
      for (int j = 0; j + 1 < nbr && ef == cudaSuccess; j++) ef = cudaStreamWaitEvent(b->branch[j], b->fork, 0);
    }
    for (int gi = 0; gi < 3 && ef == cudaSuccess; gi++) {
      const lbm_ctx* cg = rep[gi];
      if (!cg) continue;
      const int off = b->group_off[gi], cnt = b->group_off[gi + 1] - off;
      for (int k = 0; k < n; k++) {
        const StepParams* P = g.params + (k & 1) * nb;
        dispatch(cg, [&](auto xt, auto s) {
          Kern<decltype(xt)::value, decltype(s)::value>::batch_step(
              cnt, cg->block, cg->stage_smem, sg[gi], P, b->work_dev + off, stats);
        });
      }
    }
    for (int j = 0; j + 1 < nbr && ef == cudaSuccess; j++) {
      ef = cudaEventRecord(b->join[j], b->branch[j]);
      if (ef == cudaSuccess) ef = cudaStreamWaitEvent(b->capture, b->join[j], 0);
    }
    e = cudaStreamEndCapture(b->capture, &graph);
    if (e == cudaSuccess && ef != cudaSuccess) e = ef;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g.params);
    b->err = std::string("lbm_batch_step: CUDA graph capture failed: ") + cudaGetErrorString(e);
    return LBM_ERR_CUDA;
  }
  b->graphs.push_back(g);
  *exec = g.exec;
  return LBM_OK;
}

lbm_status batch_run(lbm_batch* b, int n) {
  if (n == 0) return LBM_OK;
  bool stats = b->boxes[0]->stats_on;
  for (lbm_ctx* c : b->boxes) {
    if (c->status != LBM_OK) {
      b->err = "lbm_batch_step: a box holds an earlier error: " + c->err;
      return LBM_ERR_STATE;
    }
    if (c->stats_on != stats) {
      b->err = "lbm_batch_step: statistics must be on for every box or for none";
      return LBM_ERR_ARG;
    }
  }
  cudaGraphExec_t exec = nullptr;
  const lbm_status s = batch_graph(b, n, stats, &exec);
  if (s != LBM_OK) return s;
  if (cudaGraphLaunch(exec, b->stream) != cudaSuccess) {
    b->err = std::string("lbm_batch_step: graph launch failed: ") +
             cudaGetErrorString(cudaGetLastError());
    return LBM_ERR_CUDA;
  }
  for (lbm_ctx* c : b->boxes) {
    if (n & 1) c->cur = 1 - c->cur;
    c->steps += n;
    if (c->stats_on) c->stats_samples += n;
  }
  return LBM_OK;
}

// Milliseconds per step of the current configuration over `steps` steps.
double batch_time(lbm_batch* b, int steps) {
  if (batch_run(b, 2) != LBM_OK) return -1.0;  // warm-up, builds nothing reused
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, b->stream);
  const lbm_status s = batch_run(b, steps);
  cudaEventRecord(e1, b->stream);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  free_graphs(b);
  return s == LBM_OK ? (double)ms / steps : -1.0;
}

}  // namespace

extern "C" {

size_t lbm_batch_workspace_bytes(int32_t nbox, const lbm_box* boxes, int32_t storage,
                                 int32_t stats_xbins) {
  if (!batch_args_ok(nbox, boxes, storage, stats_xbins)) return 0;
  size_t best = 0;
  for (int xt : kBatchChunks) {
    size_t sum = 0;
    for (int i = 0; i < nbox; i++) sum += batch_box_bytes(boxes[i], storage, stats_xbins, xt);
    best = std::max(best, sum);
  }
  return best;
}

lbm_status lbm_batch_create(int32_t nbox, const lbm_box* boxes, int32_t storage,
                            int32_t stats_xbins, double init_perturb, int32_t tune_steps,
                            void* cuda_stream, void* workspace, size_t workspace_bytes,
                            lbm_batch** out) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (!batch_args_ok(nbox, boxes, storage, stats_xbins) || tune_steps < -1 ||
      !std::isfinite(init_perturb))
    return LBM_ERR_ARG;
  const size_t need = lbm_batch_workspace_bytes(nbox, boxes, storage, stats_xbins);
  if (workspace && workspace_bytes < need) return LBM_ERR_OOM;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0) return LBM_ERR_ARG;
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ERR_OOM;
  b->storage = storage;
  b->nbins = stats_xbins;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  auto bail = [&](lbm_status s) {
    free_boxes(b);
    if (b->owns_ws && b->ws) cudaFree(b->ws);
    free_streams(b);
    delete b;
    return s;
  };
  bool made = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) == cudaSuccess;
  if (made) made = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int j = 0; j < 2 && made; j++)
    made = cudaStreamCreateWithFlags(&b->branch[j], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming) == cudaSuccess;
  if (!made) {
    cudaGetLastError();
    return bail(LBM_ERR_CUDA);
  }
  if (workspace) {
    b->ws = static_cast<char*>(workspace);
  } else {
    if (cudaMalloc(&b->ws, need) != cudaSuccess) {
      cudaGetLastError();
      b->ws = nullptr;
      return bail(LBM_ERR_OOM);
    }
    b->owns_ws = true;
  }
  int max_nx = 0;
  for (int i = 0; i < nbox; i++) max_nx = std::max(max_nx, boxes[i].grid.nx);
  // untuned: the widest chunk that does not exceed the longest row, for every
  // box (each box its own width is a tuner candidate: on the 64-box canopy
  // ensemble, nx 96..160, both measured about 0.93 ms per step)
  int best_xt = tune_steps < 0 ? 0 : chunk_width(max_nx), best_waves = 8;
  double best_ms = 0.0;
  if (tune_steps > 0) {
    best_ms = 1e300;
    for (int xt : kBatchChunks) {
      if (xt > 2 * chunk_width(max_nx)) continue;  // (xt = 0: each box its own width)
      lbm_status s = make_boxes(b, nbox, boxes, init_perturb, xt);
      if (s != LBM_OK) return bail(s);
      for (int waves : {2, 4, 8, 16}) {
        if ((s = make_work(b, waves)) != LBM_OK) return bail(s);
        const double ms = batch_time(b, tune_steps);
        b->tried.insert(b->tried.end(), {(double)xt, (double)b->work.size(), ms});
        if (ms > 0.0 && ms < best_ms) {
          best_ms = ms;
          best_xt = xt;
          best_waves = waves;
        }
      }
      free_boxes(b);
    }
  }
  if (best_ms >= 1e300) best_ms = 0.0;  // no candidate could be timed: the size rule stands
  lbm_status s = make_boxes(b, nbox, boxes, init_perturb, best_xt);
  if (s == LBM_OK) s = make_work(b, best_waves);
  if (s != LBM_OK) return bail(s);
  b->tuned_ms = best_ms;
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int32_t n) {
  if (!b || n < 0) return LBM_ERR_ARG;
  return batch_run(b, n);
}

lbm_status lbm_batch_sync(lbm_batch* b) {
  if (!b) return LBM_ERR_ARG;
  for (lbm_ctx* c : b->boxes) {
    const lbm_status s = lbm_sync(c);
    if (s != LBM_OK) {
      b->err = "lbm_batch_sync: " + c->err;
      return s;
    }
  }
  return LBM_OK;
}

lbm_status lbm_batch_stats_reset(lbm_batch* b, int32_t enable) {
  if (!b) return LBM_ERR_ARG;
  for (lbm_ctx* c : b->boxes) {
    const lbm_status s = lbm_stats_reset(c, enable);
    if (s != LBM_OK) return s;
  }
  return LBM_OK;
}

lbm_ctx* lbm_batch_box(lbm_batch* b, int32_t i) {
  if (!b || i < 0 || i >= (int32_t)b->boxes.size()) return nullptr;
  return b->boxes[i];
}

lbm_status lbm_batch_tuning(const lbm_batch* b, int32_t* chunk_width, int32_t* blocks,
                            double* ms_per_step) {
  if (!b) return LBM_ERR_ARG;
  if (chunk_width) *chunk_width = b->xt;
  if (blocks) *blocks = (int32_t)b->work.size();
  if (ms_per_step) *ms_per_step = b->tuned_ms;
  return LBM_OK;
}

int32_t lbm_batch_candidates(const lbm_batch* b, int32_t* chunk_width, int32_t* blocks,
                             double* ms_per_step, int32_t cap) {
  if (!b) return -1;
  const int n = (int)(b->tried.size() / 3);
  for (int k = 0; k < n && k < cap; k++) {
    if (chunk_width) chunk_width[k] = (int32_t)b->tried[3 * k];
    if (blocks) blocks[k] = (int32_t)b->tried[3 * k + 1];
    if (ms_per_step) ms_per_step[k] = b->tried[3 * k + 2];
  }
  return n;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  free_boxes(b);
  if (b->owns_ws && b->ws) cudaFree(b->ws);
  free_streams(b);
  delete b;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"

// ---- learned first-layer correction -------------------------------------------------
namespace {

lbm_status mlp_fail(lbm_mlp* m, lbm_status s, const std::string& what) {
  cudaGetLastError();
  m->err = what;
  return s;
}

// Glorot-uniform weights from SplitMix64 (counter-based), zero biases, unit normalisation.
void mlp_init_host(std::vector<float>& th, uint64_t seed) {
  th.assign(MLP_NP, 0.f);
  const int offs[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4};
  const int fan_in[4] = {MLP_IN, MLP_H, MLP_H, MLP_H}, fan_out[4] = {MLP_H, MLP_H, MLP_H, MLP_OUT};
  uint64_t k = 0;
  for (int l = 0; l < 4; l++) {
    const double r = std::sqrt(6.0 / (fan_in[l] + fan_out[l]));
    for (int e = 0; e < fan_in[l] * fan_out[l]; e++) {
      uint64_t z = seed + (++k) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;  // [-1, 1)
      th[offs[l] + e] = (float)(r * u);
    }
  }
  for (int i = 0; i < MLP_IN; i++) th[OFF_XS + i] = 1.f;
  for (int i = 0; i < MLP_OUT; i++) th[OFF_YS + i] = 1.f;
}

// Training buffers for `rows` samples: H0 (9), H1..H3 (64), D1..D3 (64), D4 (4) per row.
constexpr long long kTrainFloatsPerRow = 9 + 3 * 64 + 3 * 64 + 4;

lbm_status mlp_scratch(lbm_mlp* m, long long rows) {
  if (rows <= m->scratch_rows) return LBM_OK;
  if (m->scratch) cudaFree(m->scratch);
  m->scratch = nullptr;
  m->scratch_rows = 0;
  if (cudaMalloc(&m->scratch, sizeof(float) * kTrainFloatsPerRow * rows) != cudaSuccess)
    return mlp_fail(m, LBM_ERR_OOM, "lbm_mlp: cudaMalloc of the training buffers failed");
  m->scratch_rows = rows;
  return LBM_OK;
}

// Forward, backward and weight gradients of `n` samples (rows idx[0..n) of X,
// Y, or the first n rows when idx is null) into m->grad; the loss is the mean
// over n_total samples and 4 outputs.
void mlp_pass(lbm_mlp* m, const float* X, const float* Y, const int* idx, int n, int n_total) {
  float* H0 = m->scratch;
  float* H1 = H0 + 9ll * n;
  float* H2 = H1 + 64ll * n;
  float* H3 = H2 + 64ll * n;
  float* D1 = H3 + 64ll * n;
  float* D2 = D1 + 64ll * n;
  float* D3 = D2 + 64ll * n;
  float* D4 = D3 + 64ll * n;
  const int blocks = (n + 127) / 128;
  const float scale = 2.0f / (4.0f * (float)n_total);
  mlp_launch_train_fwd(blocks, m->stream, m->theta, X, Y, idx, n, scale, H0, H1, H2, H3, D4,
                       m->sse);
  mlp_launch_train_bwd(blocks, m->stream, m->theta, n, H1, H2, H3, D4, D1, D2, D3);
  cudaMemsetAsync(m->grad, 0, sizeof(float) * MLP_NW, m->stream);
  const int rows_per_slice = 256;
  const int slices = (n + rows_per_slice - 1) / rows_per_slice;
  const float* Ds[4] = {D1, D2, D3, D4};
  const float* Hs[4] = {H0, H1, H2, H3};
  const int nouts[4] = {64, 64, 64, 4}, nins[4] = {9, 64, 64, 64};
  const int offw[4] = {OFF_W1, OFF_W2, OFF_W3, OFF_W4}, offb[4] = {OFF_B1, OFF_B2, OFF_B3, OFF_B4};
  for (int l = 0; l < 4; l++) {
    dim3 grid(slices, (nouts[l] + 3) / 4);
    mlp_launch_train_wgrad(grid, m->stream, Ds[l], nouts[l], Hs[l], nins[l], n, rows_per_slice,
                           m->grad + offw[l], m->grad + offb[l]);
  }
}

}  // namespace

extern "C" {

lbm_status lbm_mlp_create(uint64_t seed, void* cuda_stream, lbm_mlp** out) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  lbm_mlp* m = new (std::nothrow) lbm_mlp();
  if (!m) return LBM_ERR_OOM;
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  std::vector<float> th;
  mlp_init_host(th, seed);
  bool ok = cudaMalloc(&m->theta, sizeof(float) * MLP_NP) == cudaSuccess &&
            cudaMalloc(&m->adam_m, sizeof(float) * MLP_NW) == cudaSuccess &&
            cudaMalloc(&m->adam_v, sizeof(float) * MLP_NW) == cudaSuccess &&
            cudaMalloc(&m->grad, sizeof(float) * MLP_NW) == cudaSuccess &&
            cudaMalloc(&m->sse, sizeof(float)) == cudaSuccess;
  ok = ok && cudaMemcpy(m->theta, th.data(), sizeof(float) * MLP_NP, cudaMemcpyHostToDevice) ==
                 cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    lbm_mlp_destroy(m);
    return LBM_ERR_OOM;
  }
  *out = m;
  return LBM_OK;
}

lbm_status lbm_mlp_params(lbm_mlp* m, float* theta, size_t n) {
  if (!m || !theta || n != (size_t)MLP_NP) return LBM_ERR_ARG;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess ||
      cudaMemcpy(theta, m->theta, sizeof(float) * MLP_NP, cudaMemcpyDeviceToHost) != cudaSuccess)
    return mlp_fail(m, LBM_ERR_CUDA, "lbm_mlp_params: copy failed");
  return LBM_OK;
}

lbm_status lbm_mlp_set_params(lbm_mlp* m, const float* theta, size_t n) {
  if (!m || !theta || n != (size_t)MLP_NP) return LBM_ERR_ARG;
  for (int i = 0; i < MLP_IN; i++)
    if (!(theta[OFF_XS + i] > 0.f)) return LBM_ERR_ARG;
  for (int i = 0; i < MLP_OUT; i++)
    if (!(theta[OFF_YS + i] > 0.f)) return LBM_ERR_ARG;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess ||
      cudaMemcpy(m->theta, theta, sizeof(float) * MLP_NP, cudaMemcpyHostToDevice) != cudaSuccess)
    return mlp_fail(m, LBM_ERR_CUDA, "lbm_mlp_set_params: copy failed");
  m->adam_t = 0;
  return LBM_OK;
}

lbm_status lbm_mlp_forward(lbm_mlp* m, const float* X, int64_t n, float* Y) {
  if (!m || !X || !Y || n < 0 || n > (1ll << 30)) return LBM_ERR_ARG;
  if (n == 0) return LBM_OK;
  float* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(float) * (MLP_IN + MLP_OUT) * n) != cudaSuccess)
    return mlp_fail(m, LBM_ERR_OOM, "lbm_mlp_forward: cudaMalloc failed");
  float* dY = buf + MLP_IN * n;
  cudaMemcpyAsync(buf, X, sizeof(float) * MLP_IN * n, cudaMemcpyHostToDevice, m->stream);
  const long long tiles = (n + 15) / 16;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((tiles + 3) / 4, 4096));
  mlp_launch_infer(blocks, m->stream, m->theta, buf, n, dY);
  cudaMemcpyAsync(Y, dY, sizeof(float) * MLP_OUT * n, cudaMemcpyDeviceToHost, m->stream);
  const cudaError_t e = cudaStreamSynchronize(m->stream);
  cudaFree(buf);
  if (e != cudaSuccess) return mlp_fail(m, LBM_ERR_CUDA, "lbm_mlp_forward: kernel failed");
  return LBM_OK;
}

lbm_status lbm_mlp_gradient(lbm_mlp* m, const float* X, const float* Y, int64_t n, float* grad,
                            size_t ngrad, float* loss) {
  if (!m || !X || !Y || !grad || ngrad != (size_t)MLP_NW || n < 1 || n > (1 << 22))
    return LBM_ERR_ARG;
  lbm_status s = mlp_scratch(m, n);
  if (s != LBM_OK) return s;
  float* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(float) * (MLP_IN + MLP_OUT) * n) != cudaSuccess)
    return mlp_fail(m, LBM_ERR_OOM, "lbm_mlp_gradient: cudaMalloc failed");
  cudaMemcpyAsync(buf, X, sizeof(float) * MLP_IN * n, cudaMemcpyHostToDevice, m->stream);
  cudaMemcpyAsync(buf + MLP_IN * n, Y, sizeof(float) * MLP_OUT * n, cudaMemcpyHostToDevice,
                  m->stream);
  cudaMemsetAsync(m->sse, 0, sizeof(float), m->stream);
  mlp_pass(m, buf, buf + MLP_IN * n, nullptr, (int)n, (int)n);
  float sse = 0.f;
  cudaMemcpyAsync(grad, m->grad, sizeof(float) * MLP_NW, cudaMemcpyDeviceToHost, m->stream);
  cudaMemcpyAsync(&sse, m->sse, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
  const cudaError_t e = cudaStreamSynchronize(m->stream);
  cudaFree(buf);
  if (e != cudaSuccess) return mlp_fail(m, LBM_ERR_CUDA, "lbm_mlp_gradient: kernel failed");
  if (loss) *loss = sse / (4.0f * (float)n);
  return LBM_OK;
}

lbm_status lbm_mlp_train(lbm_mlp* m, const float* X, const float* Y, int64_t n, int32_t epochs,
                         int32_t batch, float lr, uint64_t seed, float* loss_first,
                         float* loss_last) {
  if (!m || !X || !Y || n < 1 || n > (1 << 26) || epochs < 1 || batch < 1 || !(lr > 0.f))
    return LBM_ERR_ARG;
  batch = (int32_t)std::min<int64_t>(batch, n);
  // normalisation from the training set (mean and standard deviation; a
  // constant input or target keeps unit scale)
  std::vector<float> th(MLP_NP);
  if (cudaMemcpy(th.data(), m->theta, sizeof(float) * MLP_NP, cudaMemcpyDeviceToHost) != cudaSuccess)
    return mlp_fail(m, LBM_ERR_CUDA, "lbm_mlp_train: copy failed");
  for (int pass = 0; pass < 2; pass++) {
    const float* D = pass == 0 ? X : Y;
    const int w = pass == 0 ? MLP_IN : MLP_OUT;
    for (int k = 0; k < w; k++) {
      double s1 = 0.0, s2 = 0.0;
      for (int64_t r = 0; r < n; r++) {
        const double v = D[r * w + k];
        s1 += v;
        s2 += v * v;
      }
      const double mean = s1 / n, var = std::max(0.0, s2 / n - mean * mean);
      const double sd = var > 1e-30 * std::max(1.0, mean * mean) ? std::sqrt(var) : 1.0;
      th[(pass == 0 ? OFF_XM : OFF_YM) + k] = (float)mean;
      th[(pass == 0 ? OFF_XS : OFF_YS) + k] = (float)sd;
    }
  }
  if (n > m->data_rows) {
    if (m->data) cudaFree(m->data);
    if (m->perm) cudaFree(m->perm);
    m->data = nullptr;
    m->perm = nullptr;
    m->data_rows = 0;
    if (cudaMalloc(&m->data, sizeof(float) * (MLP_IN + MLP_OUT) * n) != cudaSuccess ||
        cudaMalloc(&m->perm, sizeof(int) * n) != cudaSuccess)
      return mlp_fail(m, LBM_ERR_OOM, "lbm_mlp_train: cudaMalloc of the training set failed");
    m->data_rows = n;
  }
  lbm_status s = mlp_scratch(m, batch);
  if (s != LBM_OK) return s;
  float* dX = m->data;
  float* dY = m->data + MLP_IN * n;
  bool ok = cudaMemcpy(m->theta, th.data(), sizeof(float) * MLP_NP, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(dX, X, sizeof(float) * MLP_IN * n, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(dY, Y, sizeof(float) * MLP_OUT * n, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(m->adam_m, 0, sizeof(float) * MLP_NW) == cudaSuccess &&
            cudaMemset(m->adam_v, 0, sizeof(float) * MLP_NW) == cudaSuccess;
  if (!ok) return mlp_fail(m, LBM_ERR_CUDA, "lbm_mlp_train: upload failed");
  m->adam_t = 0;
  std::vector<int> perm(n);
  for (int64_t r = 0; r < n; r++) perm[r] = (int)r;
  uint64_t draw = 0;
  for (int e = 0; e < epochs; e++) {
    // Fisher-Yates shuffle with SplitMix64 draws
    for (int64_t r = n - 1; r > 0; r--) {
      uint64_t z = seed + (++draw) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      std::swap(perm[r], perm[z % (uint64_t)(r + 1)]);
    }
    cudaMemcpyAsync(m->perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, m->stream);
    cudaMemsetAsync(m->sse, 0, sizeof(float), m->stream);
    for (int64_t b0 = 0; b0 < n; b0 += batch) {
      const int nb = (int)std::min<int64_t>(batch, n - b0);
      mlp_pass(m, dX, dY, m->perm + b0, nb, nb);
      m->adam_t++;
      const double c1 = 1.0 / (1.0 - std::pow(0.9, (double)m->adam_t));
      const double c2 = 1.0 / (1.0 - std::pow(0.999, (double)m->adam_t));
      mlp_launch_adam((MLP_NW + 255) / 256, m->stream, m->theta, m->grad, m->adam_m, m->adam_v,
                      MLP_NW, lr, (float)c1, (float)c2);
    }
    float sse = 0.f;
    cudaMemcpyAsync(&sse, m->sse, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess)
      return mlp_fail(m, LBM_ERR_CUDA, "lbm_mlp_train: kernel failed");
    const float l = sse / (4.0f * (float)n);  // mean over the epoch's batches (pre-update losses)
    if (e == 0 && loss_first) *loss_first = l;
    if (loss_last) *loss_last = l;
  }
  return LBM_OK;
}

void lbm_mlp_destroy(lbm_mlp* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (float* p : {m->theta, m->adam_m, m->adam_v, m->grad, m->sse, m->scratch, m->data})
    if (p) cudaFree(p);
  if (m->perm) cudaFree(m->perm);
  delete m;
}

const char* lbm_mlp_last_error(const lbm_mlp* m) { return m ? m->err.c_str() : "no network"; }

lbm_status lbm_set_correction(lbm_ctx* c, const lbm_mlp* m, double lam) {
  READY(c);
  if (c->batch) return arg_error(c, "lbm_set_correction: not available for ensemble boxes");
  if (c->aa) return arg_error(c, "lbm_set_correction: not available with the AA layout");
  if (m && c->grid.ny < 3) return arg_error(c, "lbm_set_correction: needs ny >= 3");
  if (!std::isfinite(lam)) return arg_error(c, "lbm_set_correction: lam not finite");
  if (m) {
    lbm_status s = ensure_feat_buf(c);
    if (s != LBM_OK) return s;
  }
  c->mlp = m;
  c->lam = (float)lam;
  if (m) {
    CK(c, cudaStreamSynchronize(m->stream));  // the network's parameters are ready
    launch_correction(c, m->theta, c->feat_buf);
    CK(c, cudaGetLastError());
  }
  return LBM_OK;
}

lbm_status lbm_features(lbm_ctx* c, float* X, size_t n) {
  READY(c);
  const size_t cols = (size_t)c->grid.nx * c->grid.nz;
  if (!X || n != cols * MLP_IN) return arg_error(c, "lbm_features: wrong size");
  if (c->aa) return arg_error(c, "lbm_features: not available with the AA layout");
  if (c->grid.ny < 3) return arg_error(c, "lbm_features: needs ny >= 3");
  lbm_status s0 = ensure_feat_buf(c);
  if (s0 != LBM_OK) return s0;
  launch_correction(c, nullptr, c->feat_buf);
  CK(c, cudaGetLastError());
  lbm_status s = check_device(c);
  if (s != LBM_OK) return s;
  CK(c, cudaMemcpy(X, c->feat_buf, sizeof(float) * cols * MLP_IN, cudaMemcpyDeviceToHost));
  return LBM_OK;
}

lbm_status lbm_correction_field(lbm_ctx* c, float* a, size_t n) {
  READY(c);
  const size_t cols = (size_t)c->grid.nx * c->grid.nz;
  if (!a || n != 2 * cols) return arg_error(c, "lbm_correction_field: wrong size");
  if (!c->mlp) return arg_error(c, "lbm_correction_field: no correction in use");
  lbm_status s = check_device(c);
  if (s != LBM_OK) return s;
  CK(c, cudaMemcpy(a, c->accel(), sizeof(float) * 2 * cols, cudaMemcpyDeviceToHost));
  return LBM_OK;
}

}  // extern "C"
