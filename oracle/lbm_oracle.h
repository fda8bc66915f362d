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
} orc_params;

typedef struct orc_sim orc_sim;

orc_sim* orc_create(const orc_params* p);
void orc_destroy(orc_sim* s);

/* One sphere per simulation. fixed != 0 keeps position and velocity unchanged. */
int orc_add_sphere(orc_sim* s, const double pos[3], double diameter, double density_ratio,
                   double cv, double cv_omega, int fixed);
void orc_set_particle_velocity(orc_sim* s, const double u[3], const double w[3]);
void orc_set_gravity(orc_sim* s, const double g[3]);
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

#ifdef __cplusplus
}
#endif
#endif
