/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the D3Q19 LBM-LES time step
 * (arxiv 2206.15454, Sec. 2 "Methodology" and Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY: slow, unblocked, obviously correct.  It is the
 * reference the CUDA library is compared with and shares nothing with it.
 *
 * One time step, per cell, in the paper's order (Algorithm 1):
 *   1. stream: pull the post-collision populations of the neighbours,
 *      f_i(x) <- f*_i(x - c_i), with the boundary rules of pull_population();
 *   2. moments: rho = sum f_i (Eq. density), m = sum f_i c_i;
 *   3. forest cell: velocity, drag force (Eq. forestForce) and the corrected
 *      velocity.  The drag depends on the velocity and the velocity on the
 *      force through Eq. momentum, rho u = m + F/2; the pair is solved exactly
 *      (canopy_velocity());
 *   4. collide with the total body force: BGK relaxation (Eqs. lbe, bgk)
 *      towards f_eq (Eq. local_eq) with the Smagorinsky relaxation time
 *      tau_total (tau_total equation), plus the Guo term (Eq. bodyforce).
 *
 * Readings of points the paper leaves open (each restated in the design
 * notes): collision sign = standard BGK relaxation towards f_eq; F in Eqs.
 * bodyforce/momentum is the force density rho*g; the Guo prefactor uses the
 * local tau_total; C_smag = C_s^2 with filter width 1; tau_total carries
 * 1/rho under the root (the form that follows from Eq. strain); Pi_neq is
 * built from post-streaming populations and f_eq at the force-corrected
 * velocity; the canopy drag acts on the full velocity vector.  Variants
 * (olbm_params): the drag on the streamwise component only, exact-difference
 * forcing (Kupershtokh) instead of Guo's, Q^1/2 / rho^2 under the root of
 * tau_total (the tau_total equation as printed).
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* D3Q19 velocities in the public order (see the header). */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
};

static const double CS2 = 1.0 / 3.0;  /* lattice speed of sound squared */

/* D3Q19 weights: 1/3 at rest, 1/18 along the axes, 1/36 along the edges
 * (standard values; the paper does not print them). */
static double weight(int i)
{
    int n = abs(CV[i][0]) + abs(CV[i][1]) + abs(CV[i][2]);
    if (n == 0) return 1.0 / 3.0;
    if (n == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* index of the direction with velocity (cx, cy, cz) */
static int find_dir(int cx, int cy, int cz)
{
    for (int i = 0; i < Q; i++)
        if (CV[i][0] == cx && CV[i][1] == cy && CV[i][2] == cz) return i;
    return -1;
}

static int opposite(int i) { return find_dir(-CV[i][0], -CV[i][1], -CV[i][2]); }
static int mirror_y(int i) { return find_dir(CV[i][0], -CV[i][1], CV[i][2]); }

struct olbm {
    olbm_params p;
    size_t n;          /* cells */
    double* f;         /* stored post-collision populations [q][z][y][x] */
    double* ftmp;      /* second population set (double-population scheme) */
    double* lad;       /* a(y), ny entries */
    double* uprof;     /* inflow / initial streamwise profile, ny entries */
    double* cell_rho;  /* per-cell density of the last step */
    double* cell_u;    /* per-cell velocity of the last step [3][n] */
    double g_now[3];   /* driving acceleration of the next step */
    double ub_last;    /* bulk velocity measured in the last step */
    int have_ub;
    int64_t steps;
    int stats_on;
    int64_t stats_samples;
    double* acc;       /* [9][xbins][ny]: sums of u,v,w,uu,vv,ww,uv,uw,vw */
    double* cnt;       /* [xbins][ny] number of cell samples */
    double* accel0;    /* [z][x][2] extra (x, z) acceleration of the cells at y = 0, or NULL */
};

static size_t cell_index(const olbm* s, int x, int y, int z)
{
    return ((size_t)z * (size_t)s->p.ny + (size_t)y) * (size_t)s->p.nx + (size_t)x;
}

/* ---------------------------------------------------------------------- */
/* building blocks                                                         */
/* ---------------------------------------------------------------------- */

void olbm_lattice(int32_t c[57], double w[19])
{
    for (int i = 0; i < Q; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = CV[i][a];
        w[i] = weight(i);
    }
}

/* Eq. local_eq: second-order equilibrium. */
void olbm_feq(double rho, const double u[3], double feq[19])
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; i++) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        feq[i] = weight(i) * rho *
                 (1.0 + cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. bodyforce: Guo forcing term for the force density F and relaxation
 * time tau. */
void olbm_guo(double tau, const double u[3], const double F[3], double Fi[19])
{
    for (int i = 0; i < Q; i++) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        double s = 0.0;
        for (int a = 0; a < 3; a++) {
            double term = (CV[i][a] - u[a]) / CS2 + cu * CV[i][a] / (CS2 * CS2);
            s += term * F[a];
        }
        Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * weight(i) * s;
    }
}

/* Smagorinsky model (Eqs. smogrinsky_model, nu_t, strain, tau_total):
 * Q^(1/2) = sqrt(Pi_neq : Pi_neq) and
 * tau_total = (tau0 + sqrt(tau0^2 + 18 sqrt(2) C_smag Q^(1/2) / rho)) / 2,
 * C_smag = C_s^2, filter width 1.  pineq = (xx, yy, zz, xy, xz, yz). */
double olbm_tau_total(double tau0, double cs, double rho, const double pineq[6])
{
    return olbm_tau_total_p(tau0, cs, rho, pineq, 1);
}

/* The same with Q^(1/2) / rho^p under the root: p = 1 follows from Eq. strain
 * solved for tau; p = 2 is the tau_total equation of Sec. 2.2 as printed
 * ((tau0 rho c)^2 under the root, divided by 2 rho c, c = 1). */
double olbm_tau_total_p(double tau0, double cs, double rho, const double pineq[6], int p)
{
    double qq = pineq[0] * pineq[0] + pineq[1] * pineq[1] + pineq[2] * pineq[2] +
                2.0 * (pineq[3] * pineq[3] + pineq[4] * pineq[4] + pineq[5] * pineq[5]);
    double q12 = sqrt(qq);
    double csmag = cs * cs;
    double rp = (p == 2) ? rho * rho : rho;
    return 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * sqrt(2.0) * csmag * q12 / rp));
}

/* Forest cell (Algorithm 1, Eqs. forestForce and momentum): the velocity u
 * and the drag acceleration g_c = -k |u| u satisfy u = v + g_c / 2, where v
 * already holds the momentum and half of the driving force.  Hence u is
 * parallel to v and |u| is the positive root of (k/2) s^2 + s - |v| = 0,
 * written as 2|v| / (1 + sqrt(1 + 2 k |v|)) to avoid cancellation. */
void olbm_canopy_velocity(const double v[3], double k, double u[3])
{
    double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double scale = 2.0 / (1.0 + sqrt(1.0 + 2.0 * k * vn));
    for (int a = 0; a < 3; a++) u[a] = scale * v[a];
}

/* Streamwise-only forest drag (Eq. forestForce read as acting on the
 * streamwise velocity component alone): g_c = (-k |u| u_x, 0, 0).  With
 * u = v + g_c / 2, the cross-stream components are those of v and u_x solves
 * phi(u_x) = u_x (1 + (k/2) sqrt(u_x^2 + s^2)) - v_x = 0, s^2 = v_y^2 + v_z^2.
 * phi is increasing and changes sign between 0 and v_x, so bisection on that
 * interval finds the root; it runs until the interval stops shrinking. */
void olbm_canopy_velocity_x(const double v[3], double k, double u[3])
{
    double s2 = v[1] * v[1] + v[2] * v[2];
    double lo = 0.0, hi = fabs(v[0]);
    for (int it = 0; it < 2000; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double phi = mid * (1.0 + 0.5 * k * sqrt(mid * mid + s2)) - fabs(v[0]);
        if (phi > 0.0) hi = mid;
        else lo = mid;
    }
    double ux = 0.5 * (lo + hi);
    u[0] = v[0] < 0.0 ? -ux : ux;
    u[1] = v[1];
    u[2] = v[2];
}

/* Exact-difference forcing (Kupershtokh): the force enters as the change of
 * the equilibrium when the velocity is raised by g (one time step of the
 * acceleration), f_eq(rho, u + g) - f_eq(rho, u). */
void olbm_edm_force(double rho, const double u[3], const double g[3], double Fi[19])
{
    double ug[3] = {u[0] + g[0], u[1] + g[1], u[2] + g[2]};
    double a[Q], b[Q];
    olbm_feq(rho, ug, a);
    olbm_feq(rho, u, b);
    for (int i = 0; i < Q; i++) Fi[i] = a[i] - b[i];
}

/* One collision with the model variants.  Both forcing schemes share the
 * physical velocity: u solves rho u = m + rho g_total / 2 (Eq. momentum) with
 * the drag in g_total.  Guo (Eq. bodyforce) relaxes towards f_eq(rho, u);
 * the exact-difference scheme relaxes towards f_eq(rho, u_b) at the bare
 * velocity u_b = m / rho and adds f_eq(rho, u_b + g_total) - f_eq(rho, u_b);
 * Pi_neq and tau_total are taken against the equilibrium the scheme relaxes
 * towards. */
void olbm_collide_cell_model(const double fin[19], const double g_drive[3], double k,
                             double tau0, double cs, int drag_x_only, int scheme,
                             int rho_power, double fout[19], double* rho_out,
                             double u_out[3])
{
    /* Eq. density and the first moment */
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; i++) {
        rho += fin[i];
        for (int a = 0; a < 3; a++) m[a] += fin[i] * CV[i][a];
    }
    /* Eq. momentum with the driving force, then the forest correction
     * (Algorithm 1; drag of Eq. forestForce) */
    double v[3], u[3];
    for (int a = 0; a < 3; a++) v[a] = (m[a] + 0.5 * rho * g_drive[a]) / rho;
    if (drag_x_only) olbm_canopy_velocity_x(v, k, u);
    else olbm_canopy_velocity(v, k, u);
    double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double g[3];
    for (int a = 0; a < 3; a++) g[a] = g_drive[a];
    if (drag_x_only) g[0] -= k * un * u[0];
    else
        for (int a = 0; a < 3; a++) g[a] -= k * un * u[a];

    /* Eq. local_eq at the velocity the scheme relaxes towards, and the
     * non-equilibrium momentum flux (Eq. tensor) */
    double urel[3];
    for (int a = 0; a < 3; a++) urel[a] = (scheme == OLBM_EXACT_DIFFERENCE) ? m[a] / rho : u[a];
    double feq[Q];
    olbm_feq(rho, urel, feq);
    double pineq[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < Q; i++) {
        double d = fin[i] - feq[i];
        pineq[0] += CV[i][0] * CV[i][0] * d;
        pineq[1] += CV[i][1] * CV[i][1] * d;
        pineq[2] += CV[i][2] * CV[i][2] * d;
        pineq[3] += CV[i][0] * CV[i][1] * d;
        pineq[4] += CV[i][0] * CV[i][2] * d;
        pineq[5] += CV[i][1] * CV[i][2] * d;
    }
    double tau = olbm_tau_total_p(tau0, cs, rho, pineq, rho_power);
    /* Eqs. lbe + bgk (relaxation towards f_eq) plus the forcing term */
    double Fi[Q];
    if (scheme == OLBM_EXACT_DIFFERENCE) {
        olbm_edm_force(rho, urel, g, Fi);
    } else {
        double F[3] = {rho * g[0], rho * g[1], rho * g[2]};
        olbm_guo(tau, u, F, Fi);
    }
    for (int i = 0; i < Q; i++) fout[i] = fin[i] - (fin[i] - feq[i]) / tau + Fi[i];
    *rho_out = rho;
    for (int a = 0; a < 3; a++) u_out[a] = u[a];
}

/* The default model: vector drag, Guo forcing, Q^1/2 / rho in tau_total. */
void olbm_collide_cell(const double fin[19], const double g_drive[3], double k,
                       double tau0, double cs, double fout[19],
                       double* rho_out, double u_out[3])
{
    olbm_collide_cell_model(fin, g_drive, k, tau0, cs, 0, OLBM_GUO, 1, fout, rho_out, u_out);
}

uint64_t olbm_splitmix64(uint64_t seed, uint64_t n)
{
    /* n-th output (n = 0, 1, ...) of Steele-Lea-Flood's SplitMix64 seeded
     * with `seed`: the state advances by the golden gamma before mixing. */
    uint64_t z = seed + (n + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

double olbm_uniform(uint64_t seed, uint64_t n)
{
    double r01 = (double)(olbm_splitmix64(seed, n) >> 11) * (1.0 / 9007199254740992.0);
    return 2.0 * r01 - 1.0;
}

/* ---------------------------------------------------------------------- */
/* streaming with boundaries                                                */
/* ---------------------------------------------------------------------- */

/* Post-collision value of direction j at (x, y, z) where y is inside the
 * domain and x, z may lie one cell outside: periodic wrap, inflow
 * equilibrium at x < 0, zero-gradient outflow at x >= nx. */
static double post_value(const olbm* s, const double* src, int j, int x, int y, int z)
{
    const olbm_params* p = &s->p;
    if (x < 0) {
        if (p->bc_x_lo == OBC_INFLOW) {
            double uin[3] = {s->uprof[y], 0.0, 0.0};
            double feq[Q];
            olbm_feq(1.0, uin, feq);
            return feq[j];
        }
        x += p->nx;
    } else if (x >= p->nx) {
        if (p->bc_x_hi == OBC_OUTFLOW) x = p->nx - 1;
        else x -= p->nx;
    }
    if (z < 0) z += p->nz;
    else if (z >= p->nz) z -= p->nz;
    return src[(size_t)j * s->n + cell_index(s, x, y, z)];
}

/* Stream step of Algorithm 1: population i arriving at (x, y, z). */
static double pull_population(const olbm* s, const double* src, int i, int x, int y, int z)
{
    const olbm_params* p = &s->p;
    int ys = y - CV[i][1];
    if (ys < 0 || ys >= p->ny) {
        int bc = (ys < 0) ? p->bc_y_lo : p->bc_y_hi;
        if (bc == OBC_PERIODIC) {
            ys = (ys < 0) ? ys + p->ny : ys - p->ny;
        } else if (bc == OBC_BOUNCEBACK) {
            /* halfway bounce-back: the population that left this cell
             * towards the wall comes back reversed */
            return src[(size_t)opposite(i) * s->n + cell_index(s, x, y, z)];
        } else if (bc == OBC_FREESLIP) {
            /* specular reflection: the wall-normal component flips */
            return post_value(s, src, mirror_y(i), x - CV[i][0], y, z - CV[i][2]);
        } else { /* OBC_EQUILIBRIUM */
            double feq[Q];
            olbm_feq(1.0, p->u_top, feq);
            return feq[i];
        }
    }
    return post_value(s, src, i, x - CV[i][0], ys, z - CV[i][2]);
}

/* Driving acceleration for the next step: constant, or a proportional
 * controller on the bulk velocity measured in the previous step. */
static void drive_for_next_step(const olbm* s, double g[3])
{
    for (int a = 0; a < 3; a++) g[a] = s->p.g[a];
    if (s->p.u_bulk_target > 0.0 && s->have_ub)
        g[0] = s->p.g[0] + s->p.ctrl_gain * (s->p.u_bulk_target - s->ub_last);
}

/* The collision of the domain's model (variants from the parameters). */
static void collide(const olbm* s, const double fin[Q], const double g[3], double k,
                    double fout[Q], double* rho, double u[3])
{
    const olbm_params* p = &s->p;
    olbm_collide_cell_model(fin, g, k, p->tau0, p->cs, p->drag_streamwise_only,
                            p->forcing_scheme, p->sgs_rho_power == 2 ? 2 : 1, fout, rho, u);
}

static double drag_factor(const olbm* s, int x, int y)
{
    if (s->lad == NULL) return 0.0;
    if (x < s->p.canopy_x0 || x >= s->p.canopy_x1) return 0.0;
    return s->p.cd * s->lad[y];
}

/* ---------------------------------------------------------------------- */
/* public API                                                               */
/* ---------------------------------------------------------------------- */

olbm* olbm_create(const olbm_params* p, const double* lad, const double* u_profile)
{
    if (p == NULL || p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    if (p->tau0 <= 0.5 || p->stats_xbins < 1 || p->stats_xbins > p->nx) return NULL;
    if (p->drag_streamwise_only < 0 || p->drag_streamwise_only > 1 ||
        (p->forcing_scheme != OLBM_GUO && p->forcing_scheme != OLBM_EXACT_DIFFERENCE) ||
        p->sgs_rho_power < 0 || p->sgs_rho_power > 2)
        return NULL;
    int xper = p->bc_x_lo == OBC_PERIODIC && p->bc_x_hi == OBC_PERIODIC;
    int xio = p->bc_x_lo == OBC_INFLOW && p->bc_x_hi == OBC_OUTFLOW;
    int yper = p->bc_y_lo == OBC_PERIODIC && p->bc_y_hi == OBC_PERIODIC;
    int ywall = p->bc_y_lo == OBC_BOUNCEBACK &&
                (p->bc_y_hi == OBC_BOUNCEBACK || p->bc_y_hi == OBC_FREESLIP ||
                 p->bc_y_hi == OBC_EQUILIBRIUM);
    int zper = p->bc_z_lo == OBC_PERIODIC && p->bc_z_hi == OBC_PERIODIC;
    if (!(xper || xio) || !(yper || ywall) || !zper) return NULL;

    olbm* s = (olbm*)calloc(1, sizeof(olbm));
    if (!s) return NULL;
    s->p = *p;
    s->n = (size_t)p->nx * p->ny * p->nz;
    s->f = (double*)malloc(sizeof(double) * Q * s->n);
    s->ftmp = (double*)malloc(sizeof(double) * Q * s->n);
    s->uprof = (double*)calloc((size_t)p->ny, sizeof(double));
    s->cell_rho = (double*)malloc(sizeof(double) * s->n);
    s->cell_u = (double*)malloc(sizeof(double) * 3 * s->n);
    s->acc = (double*)calloc((size_t)9 * p->stats_xbins * p->ny, sizeof(double));
    s->cnt = (double*)calloc((size_t)p->stats_xbins * p->ny, sizeof(double));
    if (lad) {
        s->lad = (double*)malloc(sizeof(double) * p->ny);
        if (s->lad) memcpy(s->lad, lad, sizeof(double) * p->ny);
    }
    if (!s->f || !s->ftmp || !s->uprof || !s->cell_rho || !s->cell_u || !s->acc || !s->cnt ||
        (lad && !s->lad)) {
        olbm_destroy(s);
        return NULL;
    }
    if (u_profile) memcpy(s->uprof, u_profile, sizeof(double) * p->ny);

    /* initial state: equilibrium at rho = 1 and the mean profile plus a
     * seeded uniform perturbation per velocity component */
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                size_t c = cell_index(s, x, y, z);
                double u0[3] = {s->uprof[y], 0.0, 0.0};
                for (int a = 0; a < 3; a++)
                    u0[a] += p->init_perturb * olbm_uniform(p->seed, 3 * (uint64_t)c + a);
                double feq[Q];
                olbm_feq(1.0, u0, feq);
                for (int i = 0; i < Q; i++) s->f[(size_t)i * s->n + c] = feq[i];
            }
    for (int a = 0; a < 3; a++) s->g_now[a] = p->g[a];
    return s;
}

void olbm_destroy(olbm* s)
{
    if (!s) return;
    free(s->f);
    free(s->ftmp);
    free(s->lad);
    free(s->uprof);
    free(s->cell_rho);
    free(s->cell_u);
    free(s->acc);
    free(s->cnt);
    free(s->accel0);
    free(s);
}

static void one_step(olbm* s)
{
    const olbm_params* p = &s->p;
    double g[3];
    drive_for_next_step(s, g);
    for (int a = 0; a < 3; a++) s->g_now[a] = g[a];

#pragma omp parallel for schedule(static)
    for (int z = 0; z < p->nz; z++) {
        for (int y = 0; y < p->ny; y++) {
            for (int x = 0; x < p->nx; x++) {
                double fin[Q], fout[Q], rho, u[3];
                for (int i = 0; i < Q; i++) fin[i] = pull_population(s, s->f, i, x, y, z);
                /* the learned first-layer correction enters as extra driving
                 * acceleration of the cells at y = 0 */
                double gc[3] = {g[0], g[1], g[2]};
                if (y == 0 && s->accel0) {
                    const double* a = s->accel0 + 2 * ((size_t)z * p->nx + x);
                    gc[0] += a[0];
                    gc[2] += a[1];
                }
                collide(s, fin, gc, drag_factor(s, x, y), fout, &rho, u);
                size_t c = cell_index(s, x, y, z);
                for (int i = 0; i < Q; i++) s->ftmp[(size_t)i * s->n + c] = fout[i];
                s->cell_rho[c] = rho;
                for (int a = 0; a < 3; a++) s->cell_u[(size_t)a * s->n + c] = u[a];
            }
        }
    }
    double* t = s->f;
    s->f = s->ftmp;
    s->ftmp = t;

    /* bulk velocity for the controller: mean streamwise velocity */
    double sum_u = 0.0;
    for (size_t c = 0; c < s->n; c++) sum_u += s->cell_u[c];
    s->ub_last = sum_u / (double)s->n;
    s->have_ub = 1;

    /* plane statistics, averaged over time, x (per bin) and z */
    if (s->stats_on) {
        size_t nb = (size_t)p->stats_xbins * p->ny;
        for (int z = 0; z < p->nz; z++)
            for (int y = 0; y < p->ny; y++)
                for (int x = 0; x < p->nx; x++) {
                    size_t c = cell_index(s, x, y, z);
                    int b = (int)(((int64_t)x * p->stats_xbins) / p->nx);
                    size_t k = (size_t)b * p->ny + y;
                    double u = s->cell_u[c], v = s->cell_u[s->n + c], w = s->cell_u[2 * s->n + c];
                    double q[9] = {u, v, w, u * u, v * v, w * w, u * v, u * w, v * w};
                    for (int m = 0; m < 9; m++) s->acc[m * nb + k] += q[m];
                    s->cnt[k] += 1.0;
                }
        s->stats_samples++;
    }
    s->steps++;
}

void olbm_step(olbm* s, int n)
{
    for (int k = 0; k < n; k++) one_step(s);
}

void olbm_get_f(const olbm* s, double* f) { memcpy(f, s->f, sizeof(double) * Q * s->n); }

void olbm_set_f(olbm* s, const double* f) { memcpy(s->f, f, sizeof(double) * Q * s->n); }

void olbm_macro(const olbm* s, double* rho_out, double* u_out)
{
    const olbm_params* p = &s->p;
    double g[3];
    drive_for_next_step(s, g);
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                double fin[Q], fout[Q], rho, u[3];
                for (int i = 0; i < Q; i++) fin[i] = pull_population(s, s->f, i, x, y, z);
                collide(s, fin, g, drag_factor(s, x, y), fout, &rho, u);
                size_t c = cell_index(s, x, y, z);
                rho_out[c] = rho;
                for (int a = 0; a < 3; a++) u_out[(size_t)a * s->n + c] = u[a];
            }
}

void olbm_fields(const olbm* s, double* rho_out, double* u_out, double* strain_out)
{
    const olbm_params* p = &s->p;
    double g[3];
    drive_for_next_step(s, g);
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                double fin[Q];
                for (int i = 0; i < Q; i++) fin[i] = pull_population(s, s->f, i, x, y, z);
                /* the same moments, velocity and non-equilibrium flux as the
                 * collision of the next step (Eqs. density, momentum, tensor) */
                double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < Q; i++) {
                    rho += fin[i];
                    for (int a = 0; a < 3; a++) m[a] += fin[i] * CV[i][a];
                }
                double v[3], u[3];
                for (int a = 0; a < 3; a++) v[a] = (m[a] + 0.5 * rho * g[a]) / rho;
                double k = drag_factor(s, x, y);
                if (p->drag_streamwise_only) olbm_canopy_velocity_x(v, k, u);
                else olbm_canopy_velocity(v, k, u);
                /* the equilibrium the collision relaxes towards: at u, or at
                 * the bare velocity m / rho with exact-difference forcing */
                double urel[3];
                for (int a = 0; a < 3; a++)
                    urel[a] = p->forcing_scheme == OLBM_EXACT_DIFFERENCE ? m[a] / rho : u[a];
                double feq[Q];
                olbm_feq(rho, urel, feq);
                double pi[6] = {0, 0, 0, 0, 0, 0};
                for (int i = 0; i < Q; i++) {
                    double d = fin[i] - feq[i];
                    pi[0] += CV[i][0] * CV[i][0] * d;
                    pi[1] += CV[i][1] * CV[i][1] * d;
                    pi[2] += CV[i][2] * CV[i][2] * d;
                    pi[3] += CV[i][0] * CV[i][1] * d;
                    pi[4] += CV[i][0] * CV[i][2] * d;
                    pi[5] += CV[i][1] * CV[i][2] * d;
                }
                double q = sqrt(pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2] +
                                2.0 * (pi[3] * pi[3] + pi[4] * pi[4] + pi[5] * pi[5]));
                double tau = olbm_tau_total_p(p->tau0, p->cs, rho, pi, p->sgs_rho_power == 2 ? 2 : 1);
                /* Pi_neq = -2 rho c_s^2 tau S (Chapman-Enskog, the relation
                 * behind Eq. strain), so |S| = sqrt(2 S:S) = sqrt(2) Q^1/2 / (2 rho c_s^2 tau) */
                size_t c = cell_index(s, x, y, z);
                if (rho_out) rho_out[c] = rho;
                if (u_out)
                    for (int a = 0; a < 3; a++) u_out[(size_t)a * s->n + c] = u[a];
                if (strain_out) strain_out[c] = sqrt(2.0) * q / (2.0 * rho * CS2 * tau);
            }
}

int olbm_set_layer0_accel(olbm* s, const double* a)
{
    if (a == NULL) {
        free(s->accel0);
        s->accel0 = NULL;
        return 0;
    }
    size_t m = 2 * (size_t)s->p.nx * s->p.nz;
    if (!s->accel0) s->accel0 = (double*)malloc(sizeof(double) * m);
    if (!s->accel0) return -1;
    memcpy(s->accel0, a, sizeof(double) * m);
    return 0;
}

double olbm_mass(const olbm* s)
{
    double m = 0.0;
    for (size_t k = 0; k < (size_t)Q * s->n; k++) m += s->f[k];
    return m;
}

void olbm_stats_reset(olbm* s, int enable)
{
    size_t nb = (size_t)s->p.stats_xbins * s->p.ny;
    memset(s->acc, 0, sizeof(double) * 9 * nb);
    memset(s->cnt, 0, sizeof(double) * nb);
    s->stats_samples = 0;
    s->stats_on = enable;
}

int64_t olbm_stats(const olbm* s, double* out)
{
    size_t nb = (size_t)s->p.stats_xbins * s->p.ny;
    for (size_t k = 0; k < nb; k++) {
        double n = s->cnt[k] > 0 ? s->cnt[k] : 1.0;
        double mu = s->acc[0 * nb + k] / n, mv = s->acc[1 * nb + k] / n,
               mw = s->acc[2 * nb + k] / n;
        out[0 * nb + k] = mu;
        out[1 * nb + k] = mv;
        out[2 * nb + k] = mw;
        out[3 * nb + k] = s->acc[3 * nb + k] / n - mu * mu;
        out[4 * nb + k] = s->acc[4 * nb + k] / n - mv * mv;
        out[5 * nb + k] = s->acc[5 * nb + k] / n - mw * mw;
        out[6 * nb + k] = s->acc[6 * nb + k] / n - mu * mv;
        out[7 * nb + k] = s->acc[7 * nb + k] / n - mu * mw;
        out[8 * nb + k] = s->acc[8 * nb + k] / n - mv * mw;
    }
    return s->stats_samples;
}

void olbm_drive(const olbm* s, double g[3], double* u_bulk)
{
    drive_for_next_step(s, g);
    *u_bulk = s->ub_last;
}

int64_t olbm_steps_done(const olbm* s) { return s->steps; }
