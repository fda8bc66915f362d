/*
 * lbmp.h -- C ABI of the GB300 library for the coupled lattice Boltzmann /
 * momentum exchange method of Werner, Rettinger & Ruede, "Coupling fully
 * resolved light particles with the Lattice Boltzmann method on adaptively
 * refined grids" (arXiv 2103.10882).
 *
 * One handle holds one simulation on one GPU: a D3Q19 TRT fluid on a
 * periodic/walled box (Sec. 2.1), one sphere coupled by the momentum exchange
 * method with the CLI boundary (Sec. 2.3), and the virtual-mass rigid-body
 * update (Sec. 3.3, Algorithm 1).  All work runs in CUDA kernels on the
 * stream given in the configuration; nothing falls back to the CPU.
 *
 * General rules
 *   - Every call returns an lbmp_status; nothing throws across the ABI.
 *   - Units are lattice units of the finest level: dx = dt = rho_0 = 1
 *     (Sec. 2.1).  Cell (i,j,k) has its centre at (i+1/2, j+1/2, k+1/2).
 *   - Populations cross the ABI as FP64 deviations g_q = f_q - w_q in the
 *     layout [q][z][y][x]; q = 0 rest, 1..6 faces (+x,-x,+y,-y,+z,-z),
 *     7..18 edges (+x+y,-x-y,+x-y,-x+y,+x+z,-x-z,+x-z,-x+z,+y+z,-y-z,+y-z,-y+z).
 *     The opposite of q >= 1 is q+1 for odd q and q-1 for even q.
 *   - Host pointers passed in are read during the call only; output buffers
 *     are owned by the caller.  "cap" arguments give the capacity of an
 *     output buffer in elements; passing cap = 0 (and out = NULL) returns
 *     the required size in *n where the call has one.
 *   - A handle is not thread-safe.  All device work is ordered on
 *     config.cuda_stream; calls that return host data synchronise it.
 *   - After a failed call lbmp_last_error() describes the failure.
 */
#ifndef LBMP_H
#define LBMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbmp_handle lbmp_handle;

typedef enum {
    LBMP_OK = 0,
    LBMP_ERR_INVALID_ARG = 1,   /* bad size, pointer, parameter or state */
    LBMP_ERR_OOM = 2,           /* device allocation failed */
    LBMP_ERR_CUDA = 3,          /* a CUDA call failed (message in lbmp_last_error) */
    LBMP_ERR_UNSTABLE = 4,      /* NaN/Inf or |u| > 0.3 in the fluid, or a particle moved > 0.5 cell in one step */
    LBMP_ERR_PARTICLE_NOT_FINEST = 5,
    LBMP_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    LBMP_ERR_UNSUPPORTED = 7    /* valid request this build does not implement */
} lbmp_status;

enum { LBMP_PERIODIC = 0, LBMP_NOSLIP = 1 };
enum { LBMP_FP64 = 0, LBMP_FP32 = 1, LBMP_FP16 = 2 };
enum { LBMP_CLI = 0, LBMP_SBB = 1 };
enum { LBMP_REFILL_EQUILIBRIUM = 0, LBMP_REFILL_GRAD = 1 };

/* Optional device allocator (e.g. a framework's caching allocator). Both
 * NULL: cudaMalloc / cudaFree.  alloc returns NULL on failure. */
typedef void* (*lbmp_alloc_fn)(size_t bytes, void* ctx);
typedef void (*lbmp_free_fn)(void* ptr, size_t bytes, void* ctx);

typedef struct {
    int nx, ny, nz;          /* cells along x, y, z (each >= 1) */
    int levels;              /* grid levels; 1 = uniform grid */
    int bc[3];               /* LBMP_PERIODIC or LBMP_NOSLIP per axis (no-slip: bounce-back walls half-way outside) */
    int precision;           /* population storage: LBMP_FP64, LBMP_FP32 (deviations), LBMP_FP16 (scaled deviations, FP32 math) */
    double tau;              /* relaxation time of the symmetric part, s+ = 1/tau, nu = (tau - 1/2)/3 (Sec. 2.1) */
    double magic;            /* TRT magic parameter Lambda (Sec. 2.1); 3/16 by default */
    int boundary;            /* LBMP_CLI (Sec. 2.3) or LBMP_SBB (delta = 1/2 on every link) */
    int force_average;       /* 1: average F/T over two steps (Algorithm 1) */
    int rescale_noneq;       /* refined grids: rescale the non-equilibrium parts of cells that change level in a regrid (default 0) */
    int regrid_interval;     /* refined grids: coarse steps between regrids, 0 = manual */
    int history_capacity;    /* particle history records kept on the device (ring) */
    int fp16_scale_log2;     /* LBMP_FP16: deviations are stored times 2^fp16_scale_log2 */
    uintptr_t cuda_stream;   /* cudaStream_t to run on; 0 = legacy default stream */
    lbmp_alloc_fn alloc;
    lbmp_free_fn free;
    void* alloc_ctx;
    double bulk_factor;      /* MRT bulk factor Lambda_b (Sec. 2.1): the bulk mode and the isotropic fourth-order
                                mode relax at s_b with (1/s_b - 1/2) = Lambda_b (1/s_nu - 1/2); 1 (default) is TRT,
                                the paper's runs use 100.  Must be > 0.  Not with rescale_noneq or the drag adjoint. */
    int refill;              /* cells the sphere uncovers (Sec. 2.3): LBMP_REFILL_EQUILIBRIUM (default) sets the
                                equilibrium at the mean density of the neighbours that stay fluid and the rigid-body
                                velocity; LBMP_REFILL_GRAD adds Grad's non-equilibrium part, -3 w_q (1 - s+)/s+ Q_q:S
                                with Q_q = c_q c_q - I/3 and the strain rate S from the velocities of the six face
                                neighbours (central differences, one-sided against the wall velocity) - the paper's
                                choice (Dorschner et al.'s approach, read as Grad's approximation) */
} lbmp_config;

/* Fills *cfg with defaults: 32^3 periodic, 1 level, FP32, tau 0.6,
 * Lambda 3/16, CLI, force averaging on, history 4096, fp16 scale 2^11. */
lbmp_status lbmp_config_default(lbmp_config* cfg);

/* Creates a simulation: allocates its device memory and initialises the
 * fluid at rest (rho = 1, u = 0).  On success *out owns everything. */
lbmp_status lbmp_create(const lbmp_config* cfg, lbmp_handle** out);
/* Frees everything the handle owns. NULL is accepted. */
lbmp_status lbmp_destroy(lbmp_handle* h);

/* Adds the sphere (Sec. 2.2-2.3): centre pos (lattice units), diameter d_p,
 * density ratio pi_p = rho_p / rho_f, virtual-mass coefficients C_v and
 * C_v,omega (Sec. 3.3; 0 gives plain MEM).  Maps it into the grid (solid
 * flags, boundary links) and zeroes the populations it covers.  One sphere
 * per handle: a second call returns LBMP_ERR_UNSUPPORTED.  *id receives 0. */
lbmp_status lbmp_add_sphere(lbmp_handle* h, const double pos[3], double diameter, double density_ratio,
                            double cv, double cv_omega, int* id);
/* Translational and angular velocity of the sphere (the wall velocity the
 * fluid sees in the next step). */
lbmp_status lbmp_set_particle_velocity(lbmp_handle* h, int id, const double u[3], const double omega[3]);
/* Held degrees of freedom of the sphere (forces are still computed):
 * fixed = 0 none, 1 translation and rotation (the sphere keeps its place
 * and velocities), 2 translation only, the rotation free (the rotating
 * virtual-mass test of Sec. 3.4).  A held group keeps its velocity and
 * records zero acceleration, so the virtual force or torque of Sec. 3.3
 * after it is zero; a group released at a step starts its kick-drift-kick
 * there (no half kick completing an earlier step).  Other values:
 * LBMP_ERR_INVALID_ARG. */
lbmp_status lbmp_set_particle_fixed(lbmp_handle* h, int id, int fixed);
/* Velocity u (lattice units, |u_i| < 0.3) of the no-slip domain wall on the
 * low (side 0) or high (side 1) face of a non-periodic axis: the wall sits
 * half-way between cells and a link crossing it takes bounce-back plus
 * Ladd's term 2 w_q rho_0 c_q.u / c_s^2, the CLI rule of Sec. 2.3 at
 * delta = 1/2 (the moving upper wall of the Couette flow in Sec. 3.4).
 * Uniform grids only (refined and batched: LBMP_ERR_UNSUPPORTED); a
 * periodic axis: LBMP_ERR_INVALID_ARG.  Walls start at rest. */
lbmp_status lbmp_set_wall_velocity(lbmp_handle* h, int axis, int side, const double u[3]);

/* Galileo number relation (Sec. 3.1, Eq. Ga): u_g = sqrt(|pi_p - 1| g d_p),
 * Ga = u_g d_p / nu.  Pure host arithmetic: returns nu, |g| and tau. */
lbmp_status lbmp_ga_parameters(double ga, double u_g, double diameter, double density_ratio,
                               double* nu, double* g, double* tau);
/* Applies lbmp_ga_parameters for the handle's sphere: sets tau and gravity
 * |g| along the unit vector dir (normalised here). */
lbmp_status lbmp_set_ga(lbmp_handle* h, double ga, double u_g, const double dir[3]);
lbmp_status lbmp_set_tau(lbmp_handle* h, double tau);
/* Gravitational acceleration acting on the sphere (F_g = (rho_p - rho_f) g V). */
lbmp_status lbmp_set_gravity(lbmp_handle* h, const double g[3]);
/* Body force density acting on the fluid (Guo-type source term). */
lbmp_status lbmp_set_body_force(lbmp_handle* h, const double f[3]);

/* Equilibrium initialisation of every fluid cell with density rho and
 * velocity u, or the velocity field u_field ([3][nz][ny][nx] FP64) when
 * non-NULL; u_field_on_device says whether it is a device or host pointer. */
lbmp_status lbmp_init_fluid(lbmp_handle* h, double rho, const double u[3], const double* u_field,
                            int u_field_on_device);
/* Whole population field in/out as FP64 deviations (host memory, 19*cells). */
lbmp_status lbmp_set_populations(lbmp_handle* h, const double* g, size_t cap);
lbmp_status lbmp_get_populations(lbmp_handle* h, double* g, size_t cap);

/* Gathers the populations of n cells (linear indices i + nx*(j + ny*k),
 * host array) into out[n][19] (FP64 deviations, host memory). */
lbmp_status lbmp_gather_populations(lbmp_handle* h, const int64_t* cells, size_t n, double* out);

/* Advances n coupled steps (Algorithm 1): stream + collide with CLI and
 * momentum-exchange forces, force averaging, gravity, virtual force and
 * Velocity Verlet, then the remap with equilibrium refill.  Asynchronous on
 * the handle's stream except for a status check every call, which also
 * brings the particle record back (a following lbmp_get_particle then needs
 * no second synchronisation).  Refined grids replay level-0 steps from CUDA
 * graphs of one or two steps. */
lbmp_status lbmp_step(lbmp_handle* h, int n);
/* Same as lbmp_step but does not read the device status word (fully
 * asynchronous); lbmp_check_status reads it later. */
lbmp_status lbmp_step_async(lbmp_handle* h, int n);
lbmp_status lbmp_check_status(lbmp_handle* h);
lbmp_status lbmp_synchronize(lbmp_handle* h);

/* Particle record, 24 doubles: F_hyd of the last step [0:3], T_hyd [3:6],
 * position [6:9], velocity u(t+1/2) [9:12], angular velocity [12:15],
 * acceleration a_p [15:18], angular acceleration [18:21], total force F_p [21:24]. */
lbmp_status lbmp_get_particle(lbmp_handle* h, int id, double out[24]);
/* Per-step history, 15 doubles per step (F_hyd, T_hyd, x_p, u_p, omega_p),
 * oldest first; at most max_steps records (the last ones kept in the ring). */
lbmp_status lbmp_get_history(lbmp_handle* h, int id, double* out, int max_steps, int* n);

/* Cell flags (0 fluid, 1 particle solid), one byte per cell. */
lbmp_status lbmp_get_flags(lbmp_handle* h, uint8_t* out, size_t cap);
/* Boundary links (x fluid, x + c_q solid) with their wall distance delta_q
 * (Sec. 2.3); order unspecified.  *n receives the number of links. */
lbmp_status lbmp_get_links(lbmp_handle* h, int64_t* cell, int32_t* q, double* delta, size_t cap, size_t* n);

/* ------------------------------------------------------------------------
 * Refined (block-structured) grids, config.levels > 1 (Sec. 4.1, 4.2.1).
 * nx, ny, nz are level-0 cells (multiples of 16, blocks of 16^3 cells);
 * level l has cells half the size of level l-1; positions, diameters and
 * tau are those of the finest level; lbmp_step advances level-0 steps, each
 * made of 2^l steps of level l.  Interface transfer: explosion into ghost
 * cells and coalescence of ghost cells into the coarser cells next to the
 * finer region (Rohde's scheme named in Sec. 4.1).  These transfers move
 * populations between cell centres 1.5 fine cells apart, which to first
 * order in Chapman-Enskog carries the non-equilibrium part from one
 * level's form to the other's, so they are not rescaled.  Cells that change
 * level in place in a regrid are: with config.rescale_noneq, each TRT part
 * of a refined cell's non-equilibrium part is scaled by
 * (tau_f - 1) / (2 (tau_c - 1)) and a coarsened cell's by the inverse
 * (otherwise they are copied, which conserves mass exactly).  The sphere and the
 * blocks around it stay on the finest level: its blocks and their 26
 * neighbours are finest, every coarser level adds the 26 neighbours of the
 * next finer level's parents (2:1 balance), and the hierarchy is rebuilt
 * every config.regrid_interval level-0 steps (0: only on lbmp_regrid).
 * Uniform-grid-only calls (populations, gather, flags) return
 * LBMP_ERR_UNSUPPORTED on refined grids; lbmp_get_level_cells replaces them.
 */

/* Equilibrium with velocity u + amp sin(2 pi (x_axis + 1/2) / L_axis) e_dir,
 * x and L in finest-level cells; works on both grid kinds. */
lbmp_status lbmp_init_fluid_wave(lbmp_handle* h, double rho, const double u[3], double amp, int dir, int axis);
/* Refines the finest-level blocks intersecting [lo, hi) (finest units), in
 * addition to the sphere's blocks, and rebuilds the hierarchy now. */
lbmp_status lbmp_refine_box(lbmp_handle* h, const double lo[3], const double hi[3]);
/* Rebuilds the hierarchy for the sphere's current position (regrid); with
 * the flow sensor on, also for the sensor's reading of every real block. */
lbmp_status lbmp_regrid(lbmp_handle* h);
/* Flow-based refinement sensor (Sec. 4.2.2, Eq. "sensor_curl"): per cell
 * phi_c = |curl u| s^((r+1)/r) with r = 2, s the cell size and derivatives
 * in finest-level units; u = sum_q g_q c_q of the stored deviations;
 * central differences inside a block, one-sided on its faces.  A real block
 * of level l whose largest phi_c exceeds sigma_c asks for level l+1 (at most
 * the finest), below c sigma_c for level l-1, else for level l; eight
 * siblings coarsen only together, and the 2:1 balance and the sphere's
 * blocks come on top.  Consulted by lbmp_regrid and the periodic regrid
 * (which then runs even without a sphere), not by lbmp_create,
 * lbmp_add_sphere or lbmp_refine_box.  sigma_c = 0 turns it off (default).
 * Errors: LBMP_ERR_INVALID_ARG unless sigma_c >= 0 and, for sigma_c > 0,
 * 0 < c < 2^-1.5 (the bound that keeps a coarsened block from refining
 * again at once); LBMP_ERR_UNSUPPORTED on a one-level or batched handle. */
lbmp_status lbmp_set_refinement_sensor(lbmp_handle* h, double sigma_c, double c);
/* Largest phi_c of every real block of a level (the sensor above), in block
 * order, computed now on the device from the current populations: out[cap]
 * caller-owned host memory, *n = real blocks of the level (cap = 0 or
 * out = NULL queries).  Errors: LBMP_ERR_INVALID_ARG for a bad level,
 * LBMP_ERR_UNSUPPORTED on a one-level or batched handle. */
lbmp_status lbmp_get_block_sensor(lbmp_handle* h, int level, double* out, size_t cap, size_t* n);
/* Cells of a level across the domain. */
lbmp_status lbmp_level_shape(lbmp_handle* h, int level, int out[3]);
/* Block-position map of a level (x fastest): real block index in position
 * order (>= 0), -2 ghost block, -1 no block of this level.  *n = positions. */
lbmp_status lbmp_get_block_map(lbmp_handle* h, int level, int32_t* out, size_t cap, size_t* n);
/* Real cells of a level in block order (x fastest within a block): global
 * level coordinates xyz[n][3] and FP64 deviations g[n][19].  *n = cells;
 * pass cap = 0 to query. */
lbmp_status lbmp_get_level_cells(lbmp_handle* h, int level, int32_t* xyz, double* g, size_t cap, size_t* n);
/* Cell flags of a level's real cells, in lbmp_get_level_cells order (the
 * remap of Sec. 2.3 on the finest level): 1 centre inside the sphere, 2
 * fluid with a D3Q19 neighbour inside it (the cells whose links take the
 * boundary rule), 0 other fluid; every cell of the coarser levels, and of
 * a grid without a sphere, is 0.  out: host array of cap bytes (caller
 * owned); *n receives the number of cells (nothing is written when cap is
 * smaller).  Refined grids only (uniform grids: lbmp_get_flags). */
lbmp_status lbmp_get_level_flags(lbmp_handle* h, int level, uint8_t* out, size_t cap, size_t* n);
/* Cell updates and kernel launches of one (level-0) step. */
lbmp_status lbmp_updates_per_step(lbmp_handle* h, int64_t* updates, int32_t* launches);

/* ------------------------------------------------------------------------
 * Batched sweep: n independent uniform periodic simulations of different
 * sizes (the (density ratio, Ga) parameter study of Sec. 5 run as one job).
 * Each simulation is a cubic box of `edge` cells (a multiple of 16) with
 * one sphere; relaxation time and gravity are per simulation (set them from
 * Ga with lbmp_ga_parameters).  cfg supplies precision, magic parameter,
 * boundary scheme, force averaging, history capacity, stream and allocator;
 * its grid fields are ignored.  The fluid starts at rest.  lbmp_step
 * advances every simulation; lbmp_get_particle / lbmp_get_history take the
 * simulation index as id.  Every phase of a step is one launch for all
 * simulations; two steps are replayed from a CUDA graph.
 */
typedef struct {
    int edge;                 /* cells per side (multiple of 16, >= 16) */
    double pos[3];            /* sphere centre */
    double diameter;
    double density_ratio;
    double cv, cv_omega;      /* virtual-mass coefficients (Sec. 3.3) */
    double tau;               /* relaxation time of this simulation */
    double gravity[3];
} lbmp_batch_sim;

lbmp_status lbmp_batch_create(const lbmp_config* cfg, const lbmp_batch_sim* sims, int n, lbmp_handle** out);
/* Times the candidate stream-collide tile shapes on the batch (reps launches
 * each, without advancing the simulations) and keeps the fastest. */
lbmp_status lbmp_batch_autotune(lbmp_handle* h, int reps);
/* [0] simulations, [1] cells, [2] threads per tile, [3] cells per thread
 * along z, [4..7] measured ns per launch of the four candidate shapes. */
lbmp_status lbmp_batch_info(lbmp_handle* h, int64_t out[8]);
/* FP64 deviations [19][edge^3] of one simulation (host memory). */
lbmp_status lbmp_batch_get_populations(lbmp_handle* h, int sim, double* out, size_t cap);

/* Counters: [0] steps, [1] cell updates (MLUPS numerator), [2] kernel
 * launches, [3] host-to-device bytes, [4] device-to-host bytes copied by
 * the library since the handle was created. */
lbmp_status lbmp_get_counters(lbmp_handle* h, int64_t out[5]);
/* Per-phase timing with CUDA events recorded on the handle's stream
 * (enable != 0 starts a new measurement, 0 stops recording).  While
 * enabled every step records events around its stream-collide kernel. */
lbmp_status lbmp_profile(lbmp_handle* h, int enable);
/* Results since the last lbmp_profile(h, 1): [0] total ms in the
 * stream-collide kernels, [1] their launches, [2] total ms of the whole
 * steps, [3] steps, [4] algorithmic bytes of those launches (19 reads and
 * 19 writes of a stored population per real cell updated), [5] cell
 * updates of those launches.  Synchronises the stream. */
lbmp_status lbmp_get_profile(lbmp_handle* h, double out[6]);
/* Boundary cells of one sphere, computed without allocating any memory.
 * (No counterpart in the paper: this is a service for callers that cannot
 * call cudaMalloc, such as a loop that must not risk the device
 * synchronisation an allocation may cause, or a process whose device
 * memory belongs to another allocator.  The call launches kernels through
 * the CUDA runtime, so it must not be made from a host function enqueued
 * on a stream, where CUDA forbids runtime calls.)
 *   flags       device array of nx*ny*nz bytes, 0 = fluid, nonzero = solid
 *   periodic    per axis, nonzero for a periodic axis
 *   center      sphere centre (host), diameter in cells
 *   list        device array of `capacity` ints: receives the linear indices
 *               of the fluid cells in the sphere's box (half width
 *               ceil(d/2) + 3 cells) that have a solid D3Q19 neighbour, in
 *               box order -- the same cells and order as the coupled step's
 *               own boundary list
 *   count       device int: the number of such cells (may exceed capacity;
 *               only the first `capacity` are written)
 *   cuda_stream stream to run on (asynchronous; nothing is synchronised)
 * Scratch lives in one fixed device array of 266240 bytes per device, held
 * until the process exits: boxes larger than 64^3 cells (diameters above 56
 * cells) are rejected with LBMP_ERR_INVALID_ARG.  The first call on a
 * device looks up that array's address and launches the kernels for the
 * first time, which may load the library's module and synchronise the
 * device: make one warm-up call before any stream capture and outside any
 * loop that must not synchronise.  The address is kept for the life of the
 * process, so the call must not be used after cudaDeviceReset.  All calls
 * share the array, so calls that overlap on the GPU race: the caller
 * serialises them.  Errors are reported by lbmp_last_error(NULL). */
lbmp_status lbmp_boundary_cells_noalloc(const uint8_t* flags, int nx, int ny, int nz, const int periodic[3],
                                        const double center[3], double diameter, int* list, int capacity,
                                        int* count, uintptr_t cuda_stream);

/* Checkpoint and resume (the paper describes none; long refined runs need
 * them).  lbmp_save writes the handle's state to the file `path`: the grid
 * description, tau, the body force, the step count, the sphere's record and
 * history, the populations (storage type, as held) and flags, and on refined
 * grids the block coverage of every level, the level-0 step count, the
 * refinement sensor and the refined box.  The byte order is the host's.
 * lbmp_load restores such a file into a handle created with the same grid,
 * levels, precision and boundary conditions (other config fields come from
 * the handle); a handle without a sphere gets the saved one.  Stepping on
 * after a load continues the saved run bit for bit.  Errors:
 * LBMP_ERR_INVALID_ARG for a missing file, another format or a different
 * grid (or a handle with a sphere of another diameter);
 * LBMP_ERR_UNSUPPORTED for batched handles.  Both synchronise the stream. */
lbmp_status lbmp_save(lbmp_handle* h, const char* path);
lbmp_status lbmp_load(lbmp_handle* h, const char* path);

/* Message of the last failure on this handle (or of the last failed create
 * when h is NULL).  Never NULL. */
const char* lbmp_last_error(const lbmp_handle* h);

/* ------------------------------------------------------------------------
 * Differentiation.  (No counterpart in the paper, which only runs the
 * forward method: a reverse-mode derivative of its uniform-grid step.)
 * Objective: the mean drag J = (1/nsteps) sum_{n=1..nsteps} F_axis^n of the
 * momentum-exchange force (Sec. 2.3) on the handle's sphere, held fixed at
 * rest (lbmp_set_particle_fixed, zero velocity) in a periodic box, with the
 * fluid started at the incompressible equilibrium (rho = 1) of the velocity
 * field u0 and the handle's tau, magic parameter and body force
 * (lbmp_set_tau, lbmp_set_body_force).  FP32 or FP64 storage; the adjoint
 * runs in the storage's arithmetic.
 *
 * lbmp_drag_forward runs the nsteps steps (the handle's populations end at
 * the last one) and keeps every checkpoint_interval-th field for the reverse
 * pass (ceil(nsteps / interval) + interval fields of device memory).
 *   u0      device array [3][nz][ny][nx] of doubles (x fastest), read during the call
 *   J       device double, receives J
 *   forces  device array [nsteps][3] of doubles receiving the force of every
 *           step (may be NULL)
 * lbmp_drag_backward then forms, by the adjoint of the step with checkpoint
 * and recompute, the derivatives of J times the device scalar dJ:
 *   grad_tau    device double, dJ * dJ/dtau               (may be NULL)
 *   grad_force  device double[3], dJ * dJ/dF (body force)  (may be NULL)
 *   grad_u0     device array like u0, dJ * dJ/du0          (may be NULL)
 * It needs the preceding forward call with the same tau and body force.
 * Both calls are asynchronous on the handle's stream except for one
 * synchronisation on the first forward call after the geometry is set.
 * Errors: LBMP_ERR_UNSUPPORTED for a refined or batched handle, FP16
 * storage, walls, or a sphere that moves; LBMP_ERR_INVALID_ARG for bad
 * arguments or a backward call without its forward call; LBMP_ERR_OOM. */
lbmp_status lbmp_drag_forward(lbmp_handle* h, const double* u0, int nsteps, int checkpoint_interval, int axis,
                              double* J, double* forces);
lbmp_status lbmp_drag_backward(lbmp_handle* h, const double* dJ, double* grad_tau, double* grad_force,
                               double* grad_u0);

#ifdef __cplusplus
}
#endif
#endif /* LBMP_H */
