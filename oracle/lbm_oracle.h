/*
 * lbm_oracle.h -- FP64 CPU oracle for the D3Q19 BGK-Smagorinsky LBM-LES step
 * with Guo body forcing and a forest-canopy drag (arxiv 2206.15454,
 * Sec. 2.1-2.3, Eqs. lbe, bgk, local_eq, bodyforce, density, momentum,
 * tensor, nu_t, the tau_total equation, forestForce; Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library; the two
 * are written independently from the paper.
 *
 * Conventions (fixed here, restated independently by the CUDA library):
 *   lattice units dx = dt = 1, c_s^2 = 1/3;
 *   direction order  0:(0,0,0) 1:(+1,0,0) 2:(-1,0,0) 3:(0,+1,0) 4:(0,-1,0)
 *                    5:(0,0,+1) 6:(0,0,-1) 7:(+1,+1,0) 8:(-1,-1,0)
 *                    9:(+1,-1,0) 10:(-1,+1,0) 11:(+1,0,+1) 12:(-1,0,-1)
 *                    13:(+1,0,-1) 14:(-1,0,+1) 15:(0,+1,+1) 16:(0,-1,-1)
 *                    17:(0,+1,-1) 18:(0,-1,+1);
 *   public population layout f[q][z][y][x], x fastest, FP64, unshifted;
 *   the stored state after a step is the post-collision population set.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* boundary kinds (same numeric values as the CUDA library's public enum) */
enum {
    OBC_PERIODIC = 0,
    OBC_BOUNCEBACK = 1,   /* halfway bounce-back, wall half a cell outside */
    OBC_FREESLIP = 2,     /* specular reflection of the wall-normal component */
    OBC_EQUILIBRIUM = 3,  /* incoming populations = f_eq(rho=1, u_top) */
    OBC_INFLOW = 4,       /* x = 0: incoming populations = f_eq(1, u_in(y)) */
    OBC_OUTFLOW = 5       /* x = nx-1: zero-gradient copy of post-collision values */
};

typedef struct olbm_params {
    int32_t nx, ny, nz;
    int32_t bc_x_lo, bc_x_hi, bc_y_lo, bc_y_hi, bc_z_lo, bc_z_hi;
    double tau0;          /* molecular relaxation time tau_0 */
    double cs;            /* Smagorinsky constant C_s; C_smag = C_s^2, filter width 1 */
    double g[3];          /* driving acceleration (lattice units) */
    double cd;            /* canopy drag coefficient C_D */
    int32_t canopy_x0, canopy_x1;  /* canopy occupies x in [x0, x1) */
    double u_bulk_target; /* > 0: x-acceleration controlled towards this bulk velocity */
    double ctrl_gain;     /* controller gain (1/steps) */
    double u_top[3];      /* velocity of the equilibrium top boundary */
    int32_t stats_xbins;  /* statistics are kept per (x-bin, y); >= 1 */
    int32_t pad0;
    uint64_t seed;        /* seed of the initial velocity perturbation */
    double init_perturb;  /* amplitude of the uniform initial perturbation */
    /* model variants (0 = default) */
    int32_t drag_streamwise_only; /* 1: the canopy drag acts on u_x only */
    int32_t forcing_scheme;       /* OLBM_GUO or OLBM_EXACT_DIFFERENCE */
    int32_t sgs_rho_power;        /* 0/1: Q^1/2 / rho under the root of tau_total; 2: / rho^2 */
    int32_t pad1;
} olbm_params;

enum { OLBM_GUO = 0, OLBM_EXACT_DIFFERENCE = 1 };

typedef struct olbm olbm;

/* Create a domain.  lad: ny entries, leaf area density per lattice length at
 * cell-centre heights (NULL = no canopy).  u_profile: ny entries, streamwise
 * velocity used as the initial mean profile and the inflow profile (NULL = 0).
 * Returns NULL on invalid arguments. */
olbm* olbm_create(const olbm_params* p, const double* lad, const double* u_profile);
void olbm_destroy(olbm* s);
/* Advance n time steps (stream + collide, Algorithm 1). */
void olbm_step(olbm* s, int n);
/* Copy the stored post-collision populations out / in, [q][z][y][x]. */
void olbm_get_f(const olbm* s, double* f);
void olbm_set_f(olbm* s, const double* f);
/* Density and force-corrected velocity that the next step would compute,
 * rho[z][y][x] and u[3][z][y][x]. */
void olbm_macro(const olbm* s, double* rho, double* u);
/* Density, velocity and strain-rate magnitude |S| = sqrt(2 S:S) that the
 * next step computes, per cell [z][y][x] (u: [3][z][y][x]); |S| follows from
 * the non-equilibrium momentum flux, Pi_neq = -2 rho c_s^2 tau_total S.
 * Any output may be NULL.  The layer-0 correction is not included. */
void olbm_fields(const olbm* s, double* rho, double* u, double* strain);
/* Learned first-layer correction: an extra driving acceleration (x and z
 * components, [z][x][2]) of the cells at y = 0 in every following step;
 * NULL switches it off.  Returns 0, or -1 if memory ran out. */
int olbm_set_layer0_accel(olbm* s, const double* a);
/* Global mass, sum over cells and directions of the stored populations. */
double olbm_mass(const olbm* s);
/* Statistics window: reset (and enable) accumulation, read averages.
 * out: 9 blocks of xbins*ny doubles: <u>,<v>,<w>, <u'u'>,<v'v'>,<w'w'>,
 * <u'v'>,<u'w'>,<v'w'>.  Returns the number of time samples. */
void olbm_stats_reset(olbm* s, int enable);
int64_t olbm_stats(const olbm* s, double* out);
/* Current driving acceleration (after the controller) and last bulk velocity. */
void olbm_drive(const olbm* s, double g[3], double* u_bulk);
int64_t olbm_steps_done(const olbm* s);

/* ---- building blocks, exposed for the closed-form checks ---- */
void olbm_lattice(int32_t c[57], double w[19]);
void olbm_feq(double rho, const double u[3], double feq[19]);
void olbm_guo(double tau, const double u[3], const double F[3], double Fi[19]);
double olbm_tau_total(double tau0, double cs, double rho, const double pineq[6]);
void olbm_canopy_velocity(const double v[3], double k, double u[3]);
/* One full collision of a single cell from its post-streaming populations;
 * g_drive is the driving acceleration, k = C_D * a(y) the local drag factor. */
void olbm_collide_cell(const double fin[19], const double g_drive[3], double k,
                       double tau0, double cs, double fout[19],
                       double* rho_out, double u_out[3]);
/* ---- model variants ---- */
/* Streamwise-only drag: u_y = v_y, u_z = v_z and u_x the root of
 * u_x (1 + (k/2) |u|) = v_x, |u|^2 = u_x^2 + v_y^2 + v_z^2 (by bisection). */
void olbm_canopy_velocity_x(const double v[3], double k, double u[3]);
/* tau_total with Q^1/2 / rho^p under the root, p = 1 or 2. */
double olbm_tau_total_p(double tau0, double cs, double rho, const double pineq[6], int p);
/* Exact-difference force term f_eq(rho, u + g) - f_eq(rho, u). */
void olbm_edm_force(double rho, const double u[3], const double g[3], double Fi[19]);
/* olbm_collide_cell with the variants: drag_x_only, scheme (OLBM_GUO or
 * OLBM_EXACT_DIFFERENCE), rho_power (1 or 2).  u_out is the physical
 * (force-corrected) velocity. */
void olbm_collide_cell_model(const double fin[19], const double g_drive[3], double k,
                             double tau0, double cs, int drag_x_only, int scheme,
                             int rho_power, double fout[19], double* rho_out,
                             double u_out[3]);
/* Counter-based uniform draw in [-1, 1): n-th output of splitmix64 seeded
 * with seed, mapped through the top 53 bits. */
double olbm_uniform(uint64_t seed, uint64_t n);
/* The raw n-th SplitMix64 output behind olbm_uniform. */
uint64_t olbm_splitmix64(uint64_t seed, uint64_t n);

#ifdef __cplusplus
}
#endif
#endif
