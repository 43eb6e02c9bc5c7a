/*
 * lbm.h -- C ABI of the B300 (sm_103a) D3Q19 LBM-LES library.
 *
 * One call advances a uniform-grid large-eddy simulation by whole time steps
 * of the lattice Boltzmann method of arxiv 2206.15454 (Sec. 2):
 *   stream (pull) -> density and momentum (Eqs. density, momentum)
 *   -> canopy drag F = -C_D a(y) |u| u (Eq. forestForce, Algorithm 1) solved
 *      together with the half-force velocity shift of Eq. momentum
 *   -> equilibrium (Eq. local_eq), non-equilibrium flux (Eq. tensor)
 *   -> Smagorinsky relaxation time (Eqs. nu_t, strain, tau_total)
 *   -> BGK relaxation (Eqs. lbe, bgk) + Guo forcing (Eq. bodyforce) -> store.
 * Everything runs in hand-written CUDA kernels on one GPU; there is no CPU
 * fallback.
 *
 * Conventions
 *   Lattice units (dx = dt = 1, c_s^2 = 1/3).  Direction order:
 *     0:(0,0,0) 1:(+1,0,0) 2:(-1,0,0) 3:(0,+1,0) 4:(0,-1,0) 5:(0,0,+1)
 *     6:(0,0,-1) 7:(+1,+1,0) 8:(-1,-1,0) 9:(+1,-1,0) 10:(-1,+1,0)
 *     11:(+1,0,+1) 12:(-1,0,-1) 13:(+1,0,-1) 14:(-1,0,+1) 15:(0,+1,+1)
 *     16:(0,-1,-1) 17:(0,+1,-1) 18:(0,-1,+1).
 *   Host population arrays (lbm_get_f / lbm_set_f) are FP64, unshifted,
 *   layout f[q][z][y][x] with x fastest, 19*nx*ny*nz values.  The state is
 *   the post-collision population set of the last completed step.
 *   On the device the populations are stored as offsets from the lattice
 *   weights, f_i - w_i, in FP32, FP16 or BF16 (lbm_storage), as a
 *   row-interleaved structure of arrays f[y][z][x-chunk][q][x]: x is cut into
 *   chunks of 64, 128 or 256 cells and each direction row of a chunk starts on
 *   a 128-byte line, with one ghost slot on each side holding the neighbouring
 *   column (previous/next chunk, periodic wrap, inflow equilibrium or
 *   outflow copy).  Two population sets are kept (pull scheme, double
 *   buffered).
 *
 * Errors
 *   Every call returns an lbm_status and never aborts.  An error other than
 *   LBM_ERR_ARG is sticky: the context refuses further work until
 *   lbm_destroy.  lbm_last_error() gives a one-line description.  lbm_step
 *   is asynchronous on the context's stream; device-side failures (a
 *   non-finite density, LBM_ERR_NAN) are reported by the next synchronising
 *   call (lbm_sync, lbm_stats, lbm_mass, lbm_get_f, lbm_get_macro,
 *   lbm_drive, lbm_save).
 *
 * Ownership
 *   Input arrays are copied during the call.  Output arrays are owned by the
 *   caller.  Device memory is either a caller-provided workspace (device
 *   pointer plus size, e.g. from PyTorch's allocator, see
 *   lbm_workspace_bytes) that must outlive the context, or allocated by the
 *   library with cudaMalloc when workspace is NULL.
 */
#ifndef LBM_B300_H
#define LBM_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum lbm_status {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,      /* invalid argument; the context (if any) is unchanged */
    LBM_ERR_OOM = 2,      /* device or host allocation failed / workspace too small */
    LBM_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    LBM_ERR_NAN = 4,      /* a cell produced a non-finite density (a non-finite velocity
                             or population shows as one within a step) */
    LBM_ERR_TIMEOUT = 5,  /* a bounded device wait gave up */
    LBM_ERR_STATE = 6,    /* the context holds an earlier sticky error */
    LBM_ERR_IO = 7,       /* checkpoint file could not be written/read/verified */
    LBM_ERR_BOUNDS = 8    /* checked builds (-DLBM_CHECK_BOUNDS) only: a bulk copy or store
                             of the step fell outside its buffer and was skipped */
} lbm_status;

/* Boundary kinds.  Supported combinations: x periodic, INFLOW(x_lo) with
 * OUTFLOW(x_hi), or HALO at both x faces; y periodic, or BOUNCEBACK at y_lo
 * with BOUNCEBACK, FREESLIP or EQUILIBRIUM at y_hi; z periodic. */
typedef enum lbm_bc {
    LBM_BC_PERIODIC = 0,
    LBM_BC_BOUNCEBACK = 1,  /* halfway bounce-back (no-slip wall half a cell out) */
    LBM_BC_FREESLIP = 2,    /* specular reflection of the wall-normal component */
    LBM_BC_EQUILIBRIUM = 3, /* incoming populations = f_eq(rho = 1, u_top) */
    LBM_BC_INFLOW = 4,      /* incoming populations = f_eq(rho = 1, u_in(y)) */
    LBM_BC_OUTFLOW = 5,     /* incoming populations copied from the last column */
    LBM_BC_HALO = 6         /* x faces of one slab of a larger domain: incoming populations
                               come from the neighbouring slabs through lbm_halo_pack /
                               lbm_halo_unpack (both x faces) */
} lbm_bc;

/* Forcing scheme (lbm_forcing.scheme). */
typedef enum lbm_force_scheme {
    LBM_FORCE_GUO = 0,              /* Eq. bodyforce (Guo), velocity shifted by F/2 (Eq. momentum) */
    LBM_FORCE_EXACT_DIFFERENCE = 1  /* Kupershtokh: relax towards f_eq(rho, u_b), u_b = m/rho,
                                       and add f_eq(rho, u_b + g) - f_eq(rho, u_b) */
} lbm_force_scheme;

typedef enum lbm_storage {
    LBM_F32 = 0,        /* f_i - w_i in FP32: 152 bytes moved per lattice update */
    LBM_F16_SHIFTED = 1,  /* f_i - w_i in FP16 (round to nearest even): 76 B/LUP */
    LBM_BF16_SHIFTED = 2, /* f_i - w_i in BF16 (round to nearest even): 76 B/LUP */
    /* Or-ed into one of the above: AA-pattern in-place storage.  One population
     * set (with a ghost layer one cell wide) instead of two, the same bytes per
     * lattice update.  After an even number of steps f*_i(x) sits in slot
     * opp(i) of cell x, after an odd number in slot i of cell x + c_i; steps
     * alternate between the two, and within a step each location is read and
     * written for one cell only, so the update is in place.  Every boundary
     * kind but LBM_BC_HALO, the model variants and the
     * read-outs work as with two sets; not available: the learned correction
     * (lbm_set_correction, lbm_features), ensembles, lbm_test_withhold_fill. */
    LBM_STORAGE_AA = 0x100
} lbm_storage;

typedef struct lbm_grid {
    int32_t nx, ny, nz;              /* cells; each >= 1, nx*ny*nz < 2^31 */
    int32_t x_lo, x_hi, y_lo, y_hi, z_lo, z_hi;  /* lbm_bc values */
} lbm_grid;

typedef struct lbm_forcing {
    double g[3];            /* driving acceleration; the force density is rho*g
                               (Eq. Body_force gives it as rho u_tau^2 / H) */
    double cd;              /* canopy drag coefficient C_D (Sec. 2.3: 0.15) */
    int32_t x_canopy_begin; /* the canopy covers x in [begin, end) ... */
    int32_t x_canopy_end;   /* ... and the heights where lad[y] > 0 */
    double u_bulk_target;   /* > 0: g[0] is corrected every step by
                               ctrl_gain * (u_bulk_target - U_b), U_b the mean
                               streamwise velocity of the previous step */
    double ctrl_gain;
    double u_top[3];        /* velocity of an EQUILIBRIUM top boundary */
    const double* u_in_profile; /* ny streamwise velocities, or NULL (= 0): the
                                   inflow profile and the initial mean profile */
    /* Model variants (all 0 = the default model).  A context with any of them
     * on runs the variant form of the step kernel; ensembles take the default
     * model only. */
    int32_t drag_streamwise_only; /* 1: the canopy drag acts on u_x alone,
                                     g_c = (-C_D a |u| u_x, 0, 0) (Eq. forestForce read
                                     as a streamwise force, as Sec. 2.3 describes it);
                                     0: on the velocity vector, g_c = -C_D a |u| u */
    int32_t scheme;               /* lbm_force_scheme */
    int32_t sgs_rho_power;        /* 0 or 1: tau_total = (tau0 + sqrt(tau0^2 + 18 sqrt(2)
                                     C_s^2 Q^1/2 / rho)) / 2 (Eq. strain solved for tau);
                                     2: Q^1/2 / rho^2 under the root (the tau_total
                                     equation as printed in Sec. 2.2) */
    int32_t reserved;             /* must be 0 */
} lbm_forcing;

/* Bytes of device workspace lbm_create needs for this grid and storage
 * (an lbm_storage value, optionally or-ed with LBM_STORAGE_AA); 0 on invalid
 * arguments. */
size_t lbm_workspace_bytes(const lbm_grid* grid, int32_t storage, int32_t stats_xbins);

/* Create a domain and initialise it on the device to f = f_eq(1, u0) with
 * u0 = (u_in_profile[y], 0, 0) + init_perturb * (r0, r1, r2), r_a the
 * (3c + a)-th output of SplitMix64 seeded with `seed` mapped to [-1, 1)
 * (c = (z*ny + y)*nx + x).
 *   tau0   molecular relaxation time, > 0.5 (nu_0 = (tau0 - 1/2)/3)
 *   cs     Smagorinsky constant C_s >= 0 (C_smag = C_s^2, filter width 1)
 *   lad    ny leaf-area densities a(y) per lattice length at cell-centre
 *          heights, or NULL for no canopy
 *   stats_xbins  number of equal x-bins the statistics are kept for (>= 1)
 *   workspace, workspace_bytes  caller-owned device memory of at least
 *          lbm_workspace_bytes(), or NULL/0 to let the library allocate.
 * The context uses the legacy default stream until lbm_set_stream. */
lbm_status lbm_create(const lbm_grid* grid, double tau0, double cs, const double* lad,
                      const lbm_forcing* forcing, int32_t storage, int32_t stats_xbins,
                      uint64_t seed, double init_perturb, void* workspace,
                      size_t workspace_bytes, lbm_ctx** out);

/* Use `cuda_stream` (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream)
 * for every later launch and copy. */
lbm_status lbm_set_stream(lbm_ctx* ctx, void* cuda_stream);

/* Enqueue n >= 0 time steps (one fused kernel per step).  Asynchronous. */
lbm_status lbm_step(lbm_ctx* ctx, int32_t n);

/* Wait for the context's stream and report device-side errors. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Test hook for the timeout path: in the next lbm_step (one step) block 0
 * of the step kernel does not issue its `fill`-th tile fill (fills count
 * from 0 per block; an index past the block's fills withholds nothing), so
 * the waits on that stage can only run out.  Every device wait gives up
 * after 2^18 polls of mbarrier.try_wait (about a second on a B300); the step
 * then sets the timeout flag, the next synchronising call returns
 * LBM_ERR_TIMEOUT (sticky), the kernel leaves no copy in flight and the
 * device stays usable.  LBM_ERR_ARG for fill < 0. */
lbm_status lbm_test_withhold_fill(lbm_ctx* ctx, int32_t fill);

/* Zero the statistics accumulators; enable != 0 makes every following step
 * add its velocities to them (Sec. 4: averaged in time, then over x-z planes). */
lbm_status lbm_stats_reset(lbm_ctx* ctx, int32_t enable);

/* Averages since the last reset: out holds 9 blocks of stats_xbins*ny
 * doubles, [quantity][xbin][y]: <u>, <v>, <w>, <u'u'>, <v'v'>, <w'w'>,
 * <u'v'>, <u'w'>, <v'w'> (covariances pooled over time, x and z).
 * n must be >= 9*stats_xbins*ny.  *samples = time steps accumulated. */
lbm_status lbm_stats(lbm_ctx* ctx, double* out, size_t n, int64_t* samples);

/* Pipelined read-out of the same averages, for a caller that reads every
 * step's result without idling the GPU: lbm_stats_begin enqueues, on the
 * context's stream after the work already enqueued, one copy of the
 * accumulators and health flags into a pinned slot of the library (a small
 * kernel writing the slot through its mapped device address, launched as a
 * programmatic dependent so that the steps around it keep their overlap; two
 * slots; LBM_ERR_ARG when both hold a pending read-out; LBM_ERR_CUDA when the
 * pinned slot has no device address) and returns at once;
 * lbm_stats_end waits for the oldest pending read-out and fills `out` and
 * `samples` exactly as lbm_stats would have at the point of the matching
 * begin (LBM_ERR_ARG when none is pending).  A step enqueued between the two
 * calls runs while the host waits.  Device-side errors (LBM_ERR_NAN,
 * LBM_ERR_TIMEOUT) are reported by lbm_stats_end. */
lbm_status lbm_stats_begin(lbm_ctx* ctx);
lbm_status lbm_stats_end(lbm_ctx* ctx, double* out, size_t n, int64_t* samples);

/* Global mass: sum over cells and directions of the stored populations, FP64. */
lbm_status lbm_mass(lbm_ctx* ctx, double* out);

/* Copy the populations out / in (FP64 host array, see Conventions; n must be
 * 19*nx*ny*nz).  lbm_set_f rounds to the storage type. */
lbm_status lbm_get_f(lbm_ctx* ctx, double* host_f, size_t n);
lbm_status lbm_set_f(lbm_ctx* ctx, const double* host_f, size_t n);

/* Density and force-corrected velocity that the next step computes:
 * rho[z][y][x] (n = nx*ny*nz values) and u[3][z][y][x] (3n values). */
lbm_status lbm_get_macro(lbm_ctx* ctx, double* rho, double* u, size_t n);

/* Q-criterion of that velocity field, q[z][y][x] (n = nx*ny*nz values), the
 * quantity whose iso-surfaces show vortical structures (Sec. 4, the
 * turbulent-channel figure): Q = (|Omega|^2 - |S|^2)/2, S and Omega the symmetric and
 * antisymmetric parts of the velocity gradient, differentiated with central
 * differences (periodic wrap; one-sided at the first and last cell of a
 * bounded direction; zero across a direction one cell wide).  FP32 on the
 * device, returned as FP64.  Uses the same device field buffer as
 * lbm_get_macro (allocated on first use). */
lbm_status lbm_get_q(lbm_ctx* ctx, double* q, size_t n);

/* Same output as lbm_get_macro, without allocating device memory.  The paper
 * has no counterpart: this serves callers that must not call cudaMalloc (a
 * fixed memory budget or pre-reserved pool, or code running while other work
 * on the device is captured or timed), whereas lbm_get_macro allocates its
 * staging buffer on first use.  The fields pass through one file-scope device
 * array of 262144 cells x 4 doubles (8 MB, held on every device that loads the
 * library until the process exits); grids with more cells are rejected with
 * LBM_ERR_ARG.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress); make it before any stream capture.  All
 * calls share the array and it keeps the last call's contents: calls that
 * overlap on the GPU (other threads or streams) race.  Synchronises the
 * context's stream. */
lbm_status lbm_get_macro_noalloc(lbm_ctx* ctx, double* rho, double* u, size_t n);

/* ---- x-slab decomposition: halo exchange ----------------------------------------
 * One domain cut along x into slabs, each an lbm_ctx whose x faces are
 * LBM_BC_HALO (no bulk-velocity controller: it needs a global sum).  Per step
 * a face passes on only what streams across it (Eq. lbe): the five
 * populations with c_x = -1 of the slab's first column go to the left
 * neighbour, the five with c_x = +1 of its last column to the right one.
 * After every lbm_step (and once after lbm_create or lbm_set_f, before the
 * first step) each slab calls lbm_halo_pack, the caller moves the faces
 * (cudaMemcpyAsync, NCCL send/receive, ...), and each slab calls
 * lbm_halo_unpack with what it received.
 * Face buffers are caller-owned DEVICE memory of lbm_halo_bytes() bytes each,
 * 16-byte aligned, layout [d][y][z] in the storage type (shifted like the
 * populations), d indexing directions 1, 7, 9, 11, 13 (c_x = +1) or
 * 2, 8, 10, 12, 14 (c_x = -1).  Both calls are asynchronous on the context's
 * stream; LBM_ERR_ARG if the context has no halo faces or a pointer is NULL. */
size_t lbm_halo_bytes(const lbm_ctx* ctx);
/* to_lo <- c_x = -1 populations of column 0; to_hi <- c_x = +1 populations of
 * column nx - 1 (the post-collision state of the last step). */
lbm_status lbm_halo_pack(lbm_ctx* ctx, void* to_lo, void* to_hi);
/* from_lo: the left neighbour's to_hi; from_hi: the right neighbour's to_lo.
 * Written into the ghost slots the next step reads. */
lbm_status lbm_halo_unpack(lbm_ctx* ctx, const void* from_lo, const void* from_hi);

/* Driving acceleration the next step uses and the bulk velocity of the last. */
lbm_status lbm_drive(lbm_ctx* ctx, double g[3], double* u_bulk);

/* Checkpoint: header (grid, parameters, storage, step, statistics) plus the
 * raw device populations, with an FNV-1a checksum; lbm_load verifies it
 * against a context created with the same grid and storage. */
lbm_status lbm_save(lbm_ctx* ctx, const char* path);
lbm_status lbm_load(lbm_ctx* ctx, const char* path);

/* Steps completed since creation (or loaded from a checkpoint). */
int64_t lbm_steps_done(const lbm_ctx* ctx);

/* Release every resource (waits for the stream).  NULL is accepted. */
void lbm_destroy(lbm_ctx* ctx);

const char* lbm_last_error(const lbm_ctx* ctx);
const char* lbm_status_string(int32_t status);

/* ---- learned first-layer correction --------------------------------------------
 * The paper has no learned component.  This is a near-wall/canopy correction
 * of the cells next to the ground at coarse resolution: a network maps, for
 * every first-cell column (x, z), the streamwise velocity u_x, the strain-rate
 * magnitude |S| = sqrt(2 S:S) (from Pi_neq = -2 rho c_s^2 tau_total S) and the
 * leaf-area density of the cells y = 0, 1, 2 (9 inputs) to
 * (du_x, du_z, dtau_x, dtau_z); the next step then drives cell (x, 0, z) with
 * the extra acceleration (lam*du_x - dtau_x, 0, lam*du_z - dtau_z) in its Guo
 * force.  The network is 9-64-64-64-4 with tanh hidden layers, BF16 weights and
 * activations, FP32 accumulation (tensor cores for inference), trained with
 * Adam on the mean squared error of standardised targets.  It is meant to be
 * trained on data the plain method produces on a 2x finer grid, coarsened; the
 * plain step (no correction) stays the fallback.
 *
 * Parameters travel as one FP32 vector of 9246 values, rows = outputs,
 * row-major: W1[64][9] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64]
 * b4[4], then x_mean[9] x_std[9] y_mean[4] y_std[4] (inputs are standardised
 * as (x - x_mean)/x_std, outputs are y_mean + y_std*o).  Feature rows are 9
 * floats in the order above, output rows 4 floats; columns are ordered (z, x). */
typedef struct lbm_mlp lbm_mlp;

/* A network with Glorot-uniform weights drawn from SplitMix64(seed), zero
 * biases and unit normalisation; it works on cuda_stream (NULL = legacy
 * default stream). */
lbm_status lbm_mlp_create(uint64_t seed, void* cuda_stream, lbm_mlp** out);
/* Copy the 9246 parameters out / in (n must be 9246; standard deviations > 0). */
lbm_status lbm_mlp_params(lbm_mlp* m, float* theta, size_t n);
lbm_status lbm_mlp_set_params(lbm_mlp* m, const float* theta, size_t n);
/* Outputs Y[n][4] for host features X[n][9] (the inference path). */
lbm_status lbm_mlp_forward(lbm_mlp* m, const float* X, int64_t n, float* Y);
/* Gradient of the loss over all n samples with respect to the 9220 trainable
 * parameters (the training path, one batch), and the loss itself. */
lbm_status lbm_mlp_gradient(lbm_mlp* m, const float* X, const float* Y, int64_t n, float* grad,
                            size_t ngrad, float* loss);
/* Set the normalisation from the data (means and standard deviations), then
 * train for `epochs` shuffled passes of minibatches of `batch` samples with
 * Adam at learning rate lr.  loss_first / loss_last: mean loss seen during the
 * first / last epoch (either may be NULL). */
lbm_status lbm_mlp_train(lbm_mlp* m, const float* X, const float* Y, int64_t n, int32_t epochs,
                         int32_t batch, float lr, uint64_t seed, float* loss_first,
                         float* loss_last);
/* Release the network; it must not be in use by a context (lbm_set_correction). */
void lbm_mlp_destroy(lbm_mlp* m);
const char* lbm_mlp_last_error(const lbm_mlp* m);

/* Use network m (NULL: none) for the context's first-layer correction with
 * velocity relaxation rate lam: the correction for the next step is computed
 * from the current state now and after every step.  The context keeps a
 * reference: m must stay alive and must not be trained while in use.  Needs
 * ny >= 3; not available for the boxes of an ensemble. */
lbm_status lbm_set_correction(lbm_ctx* ctx, const lbm_mlp* m, double lam);
/* The network inputs of the current state, X[nx*nz][9] (n = 9*nx*nz). */
lbm_status lbm_features(lbm_ctx* ctx, float* X, size_t n);
/* The layer-0 acceleration the next step will apply, a[nx*nz][2] (x, z
 * components; n = 2*nx*nz); LBM_ERR_ARG when no correction is in use. */
lbm_status lbm_correction_field(lbm_ctx* ctx, float* a, size_t n);

/* ---- ensembles of independent boxes ------------------------------------------
 * Many independent domains ("boxes") of uneven sizes and canopy profiles, as in
 * a wind-siting parameter sweep, advanced together.  The paper runs one domain
 * at a time; the ensemble fills the GPU with many small ones: one kernel launch
 * per step covers every box (each block works on one box's tiles with that
 * box's parameters), and lbm_batch_step(n) replays n such launches as one CUDA
 * graph.  The block shape (chunk width, hence the device layout) and the number
 * of work items per launch are chosen by timing candidates at creation
 * (tune_steps > 0), or by a size rule (tune_steps = 0).
 *
 * Every box is an ordinary lbm_ctx owned by the ensemble: lbm_batch_box()
 * returns it for the readouts (lbm_get_f, lbm_get_macro, lbm_stats, lbm_mass,
 * lbm_drive, lbm_save, lbm_load, lbm_set_f, lbm_sync), and even lbm_step on
 * one box alone works; lbm_destroy on a box is a no-op (lbm_batch_destroy
 * releases them).  The boxes use the ensemble's stream. */
typedef struct lbm_batch lbm_batch;

typedef struct lbm_box {
    lbm_grid grid;          /* any of the supported boundary combinations */
    double tau0, cs;        /* as in lbm_create */
    const double* lad;      /* ny leaf-area densities, or NULL */
    lbm_forcing forcing;    /* u_bulk_target must be <= 0: no controller in an ensemble */
    uint64_t seed;          /* initial perturbation seed of this box */
} lbm_box;

/* Device workspace an ensemble needs (the largest over the chunk widths the
 * tuner may pick); 0 on invalid arguments. */
size_t lbm_batch_workspace_bytes(int32_t nbox, const lbm_box* boxes, int32_t storage,
                                 int32_t stats_xbins);

/* Create nbox >= 1 boxes, all with the same storage type and statistics bins,
 * initialised as lbm_create does with their own seed and the common
 * init_perturb.  tune_steps > 0 times every candidate launch configuration over
 * that many steps (the boxes are then re-initialised); tune_steps = 0 takes the
 * chunk width of the longest row for every box, tune_steps = -1 each box in its
 * own (as lbm_create would), both untimed; LBM_ERR_ARG below -1.  cuda_stream
 * NULL = legacy default stream.  workspace/workspace_bytes as in lbm_create. */
lbm_status lbm_batch_create(int32_t nbox, const lbm_box* boxes, int32_t storage,
                            int32_t stats_xbins, double init_perturb, int32_t tune_steps,
                            void* cuda_stream, void* workspace, size_t workspace_bytes,
                            lbm_batch** out);

/* Enqueue n >= 0 steps of every box: one CUDA graph of n launches (built on
 * first use for this n and reused).  Asynchronous.  Statistics must be on for
 * all boxes or for none (lbm_batch_stats_reset). */
lbm_status lbm_batch_step(lbm_batch* b, int32_t n);

/* Wait for the stream and report device-side errors of any box. */
lbm_status lbm_batch_sync(lbm_batch* b);

/* lbm_stats_reset on every box. */
lbm_status lbm_batch_stats_reset(lbm_batch* b, int32_t enable);

/* Box i (0 <= i < nbox) as a context handle owned by the ensemble; NULL if out
 * of range. */
lbm_ctx* lbm_batch_box(lbm_batch* b, int32_t i);

/* The launch configuration in use: chunk width (cells; 0 = every box in the
 * width a single domain of its x-length takes: 64 up to 64 cells, 128 up to
 * 128, else 256, one launch per width and step), blocks per launch and the measured
 * milliseconds per step of the chosen candidate (0 if untuned; untuned, the
 * chunk width is the one the longest row takes). */
lbm_status lbm_batch_tuning(const lbm_batch* b, int32_t* chunk_width, int32_t* blocks,
                            double* ms_per_step);

/* The tuner's record: for each candidate it timed (at most cap are written),
 * its chunk width (0: each box its own, as above), blocks per launch and
 * milliseconds per step (negative if it failed).  Returns the number of candidates timed (0 when untuned), -1 for
 * b == NULL. */
int32_t lbm_batch_candidates(const lbm_batch* b, int32_t* chunk_width, int32_t* blocks,
                             double* ms_per_step, int32_t cap);

void lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

#ifdef __cplusplus
}
#endif
#endif
