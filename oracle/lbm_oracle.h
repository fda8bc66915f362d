/*
 * Oracle for the coupled LBM-MEM method of Werner, Rettinger & Ruede,
 * "Coupling fully resolved light particles with the Lattice Boltzmann
 * method on adaptively refined grids" (arXiv 2103.10882).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
 * the method, written from the paper's equations so that the CUDA library
 * can be checked against it.  It shares no code with the CUDA library and
 * neither side includes or links the other.  Only tests/, the smoke check
 * of __graft_entry__ and the CPU-baseline leg of bench.py may load it.
 *
 * Conventions (each side defines them on its own; they are an interface
 * both must agree on, like a file format):
 *   - D3Q19, q = 0 rest, 1..6 faces (+x,-x,+y,-y,+z,-z), 7..18 edges
 *     (+x+y,-x-y,+x-y,-x+y,+x+z,-x-z,+x-z,-x+z,+y+z,-y-z,+y-z,-y+z);
 *     the opposite of q >= 1 is q+1 for odd q and q-1 for even q.
 *   - populations are kept as deviations g_q = f_q - w_q, array layout
 *     [q][z][y][x], cell (i,j,k) has its centre at (i+1/2, j+1/2, k+1/2);
 *   - the stored state between steps is the post-collision field.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    int periodic[3];      /* 1: periodic axis; 0: stationary no-slip walls half-way outside both ends */
    double tau;           /* s+ = 1/tau (Sec. 2.1: nu = c_s^2 (1/s_nu - 1/2)) */
    double magic;         /* TRT magic parameter Lambda (Sec. 2.1) */
    double body_force[3]; /* fluid body force per unit volume (0 disables the source term) */
    int boundary;         /* 0 = CLI (Eq. of Sec. 2.3), 1 = simple bounce-back (delta = 1/2) */
    int force_average;    /* 1 = average hydrodynamic force/torque over two steps (Algorithm 1) */
    int plain_mem;        /* 1 = particle update of Sec. 2.2 without the virtual-mass terms */
    double bulk;          /* MRT bulk factor Lambda_b (Sec. 2.1); 0 or 1 = TRT */
    int refill;           /* uncovered cells: 0 = equilibrium, 1 = Grad's approximation (Sec. 2.3) */
} orc_params;

typedef struct orc_sim orc_sim;

orc_sim* orc_create(const orc_params* p);
void orc_destroy(orc_sim* s);

/* One sphere per simulation. fixed != 0 keeps position and velocity unchanged. */
int orc_add_sphere(orc_sim* s, const double pos[3], double diameter, double density_ratio,
                   double cv, double cv_omega, int fixed);
void orc_set_particle_velocity(orc_sim* s, const double u[3], const double w[3]);
void orc_set_gravity(orc_sim* s, const double g[3]);
/* Held degrees of freedom of the sphere from the next step on: 0 none, 1
 * translation and rotation, 2 translation only (rotation free).  A held
 * group keeps its velocity and has zero acceleration; a released group
 * starts its kick-drift-kick afresh.  -1 without a sphere or for another
 * value.  (orc_add_sphere's `fixed` takes the same values.) */
int orc_set_particle_fixed(orc_sim* s, int fixed);
/* Velocity of the no-slip domain wall on the low (side 0) or high (side 1)
 * face of a non-periodic axis (bounce-back with Ladd's moving-wall term,
 * the CLI rule at delta = 1/2); -1 for a periodic axis. */
int orc_set_wall_velocity(orc_sim* s, int axis, int side, const double u[3]);

/* Test geometry: two moving plane walls normal to `axis` at coordinates lo < hi.
 * Cells whose centre lies outside [lo, hi] are solid; links use CLI with the
 * exact sub-grid distance. */
int orc_set_planes(orc_sim* s, int axis, double lo, double hi, const double v_lo[3], const double v_hi[3]);

/* Equilibrium initialisation of every fluid cell; u_field ([3][ncells]) may be NULL. */
void orc_init_equilibrium(orc_sim* s, double rho, const double u[3], const double* u_field);
void orc_set_populations(orc_sim* s, const double* g);
void orc_get_populations(const orc_sim* s, double* g);
void orc_get_flags(const orc_sim* s, uint8_t* flags);
void orc_moments(const orc_sim* s, double* rho, double* u);

void orc_step(orc_sim* s, int n);

/* Boundary links (x fluid, x + c_q solid) in (cell, q) order. Returns the count. */
int64_t orc_get_links(const orc_sim* s, int64_t* cell, int32_t* q, double* delta, int64_t cap);

/* Particle record, 24 doubles:
 * [0:3] F_hyd of the last step, [3:6] T_hyd, [6:9] x_p, [9:12] u_p (wall velocity, u at t+1/2),
 * [12:15] omega_p, [15:18] a_p (last), [18:21] beta_p (last), [21:24] F_p total (last). */
void orc_get_particle(const orc_sim* s, double out[24]);
/* Per-step history: 15 doubles per step: F_hyd, T_hyd, x_p, u_p, omega_p. */
int64_t orc_get_history(const orc_sim* s, double* out, int64_t cap_steps);
/* Momentum exchanged with the planes during the last step (test geometry only). */
void orc_get_plane_force(const orc_sim* s, double out[3]);

/* Particle update alone (Algorithm 1, the steps after the LBM step), with a
 * given hydrodynamic force and torque instead of the fluid's. No remap. */
void orc_particle_only_step(orc_sim* s, const double F_hyd[3], const double T_hyd[3]);

/* Threads for the per-cell loops (results do not depend on it). Returns the count in use. */
int orc_set_threads(int n);

/* ------------------------------------------------------------------------
 * Tangent-linear model of the mean drag on a fixed sphere, tangent.cpp.
 * Periodic box, sphere at rest at pos, CLI (boundary 0) or simple
 * bounce-back (1), fluid started at the equilibrium of u0 ([3][cells] with
 * x fastest, NULL = rest).  Returns J = (1/nsteps) sum_n F_axis^n of the
 * momentum-exchange force; *dJ receives its derivative along (dtau, dforce,
 * du0) (dforce or du0 NULL = 0), force_out ([nsteps][3], may be NULL) the
 * force of every step.
 */
typedef struct {
    int nx, ny, nz;
    double tau, magic;
    double body_force[3];
    int boundary;
    double pos[3];
    double diameter;
} orc_drag_params;
double orc_drag_tangent(const orc_drag_params* p, const double* u0, int nsteps, double dtau, const double dforce[3],
                        const double* du0, int axis, double* dJ, double* force_out);

/* ------------------------------------------------------------------------
 * Refined (block-structured) grid, refined.cpp.  Levels 0..levels-1, blocks
 * of 16^3 cells, nx, ny, nz = level-0 cells (multiples of 16), positions and
 * diameters in finest-level lattice units, tau of the finest level.
 */
typedef struct {
    int nx, ny, nz;
    int levels;
    int periodic[3];
    double tau;
    double magic;
    int boundary;
    int force_average;
    int plain_mem;
    int rescale;          /* 1: rescale non-equilibrium parts of cells that change level in a regrid */
    double bulk;          /* MRT bulk factor Lambda_b (Sec. 2.1); 0 or 1 = TRT */
    int refill;           /* uncovered cells: 0 = equilibrium, 1 = Grad's approximation (Sec. 2.3) */
} orc_amr_params;
/* Grad's post-collision non-equilibrium part for relaxation time tau and
 * strain rate S (row major) into out[19] (test helper). */
void orc_grad_noneq(double tau, const double S[9], double out[19]);
typedef struct orc_amr orc_amr;
orc_amr* orc_amr_create(const orc_amr_params* p);
void orc_amr_destroy(orc_amr* a);
/* Refines the finest-level blocks intersecting [lo, hi) (and regrids). */
int orc_amr_refine_box(orc_amr* a, const double lo[3], const double hi[3]);
int orc_amr_add_sphere(orc_amr* a, const double pos[3], double diameter, double density_ratio, double cv,
                       double cv_omega, int fixed);
void orc_amr_set_gravity(orc_amr* a, const double g[3]);
void orc_amr_set_particle_velocity(orc_amr* a, const double u[3], const double w[3]);
/* Rebuilds the hierarchy for the sphere (and box); with the flow sensor on,
 * also for the sensor's wishes of every real block (Sec. 4.2.2). */
int orc_amr_regrid(orc_amr* a);
/* Flow sensor: refine a block whose scaled curl exceeds sigma, coarsen below
 * c sigma; sigma = 0 turns it off.  -1 unless 0 < c < 2^-1.5. */
int orc_amr_set_sensor(orc_amr* a, double sigma, double c);
/* Scaled curl of every real block of a level (position order); returns the
 * number of real blocks, -1 for a bad level. */
int64_t orc_amr_block_sensor(const orc_amr* a, int level, double* out, int64_t cap);
/* Equilibrium everywhere with the linear velocity u0 + A (x - x0), A row
 * major, x the cell centre in finest-level units. */
void orc_amr_init_linear(orc_amr* a, double rho, const double u0[3], const double A[9], const double x0[3]);
/* Equilibrium everywhere with velocity u + amp sin(2 pi x_axis / L_axis) e_dir. */
void orc_amr_init_equilibrium(orc_amr* a, double rho, const double u[3], double amp, int dir, int axis);
/* n coarse (level-0) steps; returns 0 or an error code (1: missing source, 2: sphere not on the finest level). */
int orc_amr_step(orc_amr* a, int n);
int orc_amr_error(const orc_amr* a);
void orc_amr_level_shape(const orc_amr* a, int level, int out[3]);
/* Block-position map of a level: >= 0 real block (position order), -2 ghost block, -1 none. */
int64_t orc_amr_block_map(const orc_amr* a, int level, int32_t* out, int64_t cap);
/* Dense [19][cells of the level] deviations, NaN where the level has no real cell. */
void orc_amr_level_populations(const orc_amr* a, int level, double* out);
/* Real cells of a level in block-position order then local (x fastest)
 * order: coordinates [n][3] and deviations [n][19].  Returns n. */
int64_t orc_amr_real_cells(const orc_amr* a, int level, int32_t* xyz, double* g, int64_t cap);
/* Flags of the finest level's real cells in orc_amr_real_cells order: 1
 * inside the sphere, 2 fluid with a D3Q19 neighbour inside it, 0 otherwise.
 * Returns the number of cells (nothing written if cap is too small). */
int64_t orc_amr_get_flags(const orc_amr* a, uint8_t* out, int64_t cap);
/* Boundary links of the finest level: fluid cell (linear index over the
 * whole finest level, x fastest), direction q with x + c_q inside the
 * sphere, and the wall distance delta in [0, 1] (Sec. 2.3), cells in
 * orc_amr_real_cells order and q ascending.  Returns the number of links. */
int64_t orc_amr_get_links(const orc_amr* a, int64_t* cell, int32_t* q, double* delta, int64_t cap);
/* sum over real cells of (rho, rho u) times the cell volume in finest units. */
void orc_amr_mass(const orc_amr* a, double out[4]);
void orc_amr_get_particle(const orc_amr* a, double out[24]);
int64_t orc_amr_get_history(const orc_amr* a, double* out, int64_t cap_steps);

#ifdef __cplusplus
}
#endif
#endif
