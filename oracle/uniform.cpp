/*
 * Oracle, uniform grid: D3Q19 TRT lattice Boltzmann step with the momentum
 * exchange coupling of one sphere and the virtual-mass particle update.
 *
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).  Plain loops, FP64, built
 * with -O2 -ffp-contract=off.  Every function names the passage it follows.
 * The OpenMP pragmas only split independent per-cell loops; the force sums
 * stay serial, so a threaded build gives bit-identical results.
 */
#include "lbm_oracle.h"
#include "common.h"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

using namespace orc;

namespace {

struct Planes {
    bool present = false;
    int axis = 1;
    double lo = 0, hi = 0;
    double v_lo[3] = {0, 0, 0}, v_hi[3] = {0, 0, 0};
};

}  // namespace

struct orc_sim {
    orc_params p;
    long n = 0;
    std::vector<double> g, g_new;   // [19][n]
    std::vector<uint8_t> flag;      // per cell
    Particle part;
    Planes planes;
    double gravity[3] = {0, 0, 0};
    double sp = 0, sm = 0;          // s+ and s-
    double sb = 0;                  // bulk rate s_b of the MRT model (used when bulk != 1)
    double bulk = 1.0;              // bulk factor Lambda_b (1: TRT)
    std::vector<double> history;    // 15 per step
    double plane_force[3] = {0, 0, 0};
    std::vector<uint8_t> has_link;  // per cell: some source of the pull is solid
    double wall_u[3][2][3] = {};    // velocity of the domain wall [axis][0 low, 1 high] (non-periodic axes)
};

namespace {

long cell_index(const orc_sim* s, int i, int j, int k) {
    return (long)i + (long)s->p.nx * ((long)j + (long)s->p.ny * (long)k);
}

int extent(const orc_sim* s, int a) { return a == 0 ? s->p.nx : (a == 1 ? s->p.ny : s->p.nz); }

// Neighbour of (i,j,k) displaced by sign*c_q. Returns false when it leaves the
// domain through a wall axis.
bool neighbour(const orc_sim* s, int i, int j, int k, int q, int sign, long* out) {
    int c[3] = {i + sign * C[q][0], j + sign * C[q][1], k + sign * C[q][2]};
    for (int a = 0; a < 3; ++a) {
        int L = extent(s, a);
        if (c[a] < 0 || c[a] >= L) {
            if (!s->p.periodic[a]) return false;
            c[a] = (c[a] + L) % L;
        }
    }
    *out = cell_index(s, c[0], c[1], c[2]);
    return true;
}

// Minimum-image difference along axis a for periodic axes.
double wrap_diff(const orc_sim* s, int a, double d) {
    if (!s->p.periodic[a]) return d;
    double L = (double)extent(s, a);
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

// Sec. 2.3: a cell is solid when its centre lies inside the sphere (closed ball).
bool inside_sphere(const orc_sim* s, int i, int j, int k) {
    const Particle& P = s->part;
    double dx = wrap_diff(s, 0, (i + 0.5) - P.x[0]);
    double dy = wrap_diff(s, 1, (j + 0.5) - P.x[1]);
    double dz = wrap_diff(s, 2, (k + 0.5) - P.x[2]);
    double d2 = ((dx * dx) + (dy * dy)) + (dz * dz);
    return d2 <= P.r * P.r;
}

uint8_t geometry_flag(const orc_sim* s, int i, int j, int k) {
    if (s->planes.present) {
        int idx[3] = {i, j, k};
        double xc = idx[s->planes.axis] + 0.5;
        if (xc < s->planes.lo || xc > s->planes.hi) return SOLID_PLANE;
    }
    if (s->part.present && inside_sphere(s, i, j, k)) return SOLID_PARTICLE;
    return FLUID;
}

// Sec. 2.3: delta_q = distance fraction from the fluid cell centre x to the
// wall along c_q, i.e. the root s in (0,1] of |x + s c_q - x_p|^2 = r^2.
double sphere_delta(const orc_sim* s, int i, int j, int k, int q) {
    const Particle& P = s->part;
    double d[3] = {wrap_diff(s, 0, (i + 0.5) - P.x[0]), wrap_diff(s, 1, (j + 0.5) - P.x[1]),
                   wrap_diff(s, 2, (k + 0.5) - P.x[2])};
    double cc = 0, dc = 0, dd = 0;
    for (int a = 0; a < 3; ++a) {
        cc += (double)(C[q][a] * C[q][a]);
        dc += d[a] * C[q][a];
        dd += d[a] * d[a];
    }
    double disc = dc * dc - cc * (dd - P.r * P.r);
    if (disc < 0) disc = 0;
    double root = (-dc - std::sqrt(disc)) / cc;
    if (root < 0) root = 0;
    if (root > 1) root = 1;
    return root;
}

double plane_delta(const orc_sim* s, int i, int j, int k, int q) {
    int idx[3] = {i, j, k};
    int a = s->planes.axis;
    double xc = idx[a] + 0.5;
    return C[q][a] > 0 ? (s->planes.hi - xc) : (xc - s->planes.lo);
}

// Moments, Eq. (rho_f, rho_0 u_f), with half the body force added to the
// velocity for the forced case.
void cell_moments(const orc_sim* s, const std::vector<double>& g, long x, double* drho, double u[3]) {
    double r = 0;
    u[0] = u[1] = u[2] = 0;
    for (int q = 0; q < 19; ++q) {
        double v = g[(size_t)q * s->n + x];
        r += v;
        u[0] += v * C[q][0];
        u[1] += v * C[q][1];
        u[2] += v * C[q][2];
    }
    for (int a = 0; a < 3; ++a) u[a] += 0.5 * s->p.body_force[a];
    *drho = r;
}

// TRT collision (Sec. 2.1: MRT with Lambda_b = 1), written on the symmetric
// and antisymmetric parts of each pair (q, qbar).  Body force: Guo-type source
// term split the same way (its reading is listed in the design notes).
void collide_cell(orc_sim* s, long x) {
    std::vector<double>& g = s->g_new;
    double drho, u[3];
    cell_moments(s, g, x, &drho, u);
    const double* F = s->p.body_force;
    bool forced = (F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0);
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    if (s->bulk != 1.0) {   // MRT with the bulk factor Lambda_b (Sec. 2.1)
        double gi[19], ge[19], src[19], out[19];
        for (int q = 0; q < 19; ++q) {
            gi[q] = g[(size_t)q * s->n + x];
            ge[q] = geq(q, drho, u);
            const double cu = C[q][0] * u[0] + C[q][1] * u[1] + C[q][2] * u[2];
            const double cF = C[q][0] * F[0] + C[q][1] * F[1] + C[q][2] * F[2];
            src[q] = W[q] * (3.0 * cF - 3.0 * uF + 9.0 * cu * cF);   // Guo source (reading in the design notes)
        }
        mrt_collide(gi, ge, forced ? src : nullptr, s->sp, s->sm, s->sb, out);
        for (int q = 0; q < 19; ++q) g[(size_t)q * s->n + x] = out[q];
        return;
    }
    double out[19];
    // rest population: purely symmetric
    {
        double e = geq(0, drho, u);
        double gq = g[x];
        out[0] = gq - s->sp * (gq - e);
        if (forced) out[0] += (1.0 - 0.5 * s->sp) * W[0] * (-3.0 * uF);
    }
    for (int q = 1; q < 19; q += 2) {
        int qb = q + 1;
        double gq = g[(size_t)q * s->n + x], gb = g[(size_t)qb * s->n + x];
        double eq = geq(q, drho, u), eb = geq(qb, drho, u);
        double gp = 0.5 * (gq + gb), gm = 0.5 * (gq - gb);
        double ep = 0.5 * (eq + eb), em = 0.5 * (eq - eb);
        double dp = s->sp * (gp - ep), dm = s->sm * (gm - em);
        out[q] = gq - dp - dm;
        out[qb] = gb - dp + dm;
        if (forced) {
            double cu = C[q][0] * u[0] + C[q][1] * u[1] + C[q][2] * u[2];
            double cF = C[q][0] * F[0] + C[q][1] * F[1] + C[q][2] * F[2];
            double Sp = W[q] * (9.0 * cu * cF - 3.0 * uF);
            double Sm = W[q] * (3.0 * cF);
            out[q] += (1.0 - 0.5 * s->sp) * Sp + (1.0 - 0.5 * s->sm) * Sm;
            out[qb] += (1.0 - 0.5 * s->sp) * Sp - (1.0 - 0.5 * s->sm) * Sm;
        }
    }
    for (int q = 0; q < 19; ++q) g[(size_t)q * s->n + x] = out[q];
}

// Stream (Eq. LBE, pull form) with domain walls, and the CLI boundary of
// Sec. 2.3 on particle and plane links; accumulates the momentum-exchange
// force and torque of Sec. 2.3 (Galilean-invariant form) in (cell, q) order.
void stream_and_boundaries(orc_sim* s, double F[3], double T[3]) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    const long n = s->n;
    const std::vector<double>& gt = s->g;   // post-collision, time t
    std::vector<double>& gn = s->g_new;     // pre-collision, time t+1
    for (int a = 0; a < 3; ++a) F[a] = T[a] = s->plane_force[a] = 0.0;
    const Particle& P = s->part;

#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long x = cell_index(s, i, j, k);
                if (s->flag[x] != FLUID) {
                    for (int q = 0; q < 19; ++q) gn[(size_t)q * n + x] = 0.0;
                    s->has_link[x] = 0;
                    continue;
                }
                uint8_t any = 0;
                for (int q = 0; q < 19; ++q) {
                    long src;
                    if (!neighbour(s, i, j, k, q, -1, &src)) {
                        // no-slip domain wall half-way between cells: bounce-back with
                        // Ladd's moving-wall term 2 w_q rho_0 c_q.u_w / c_s^2 (the CLI
                        // rule of Sec. 2.3 at delta = 1/2), summed over the faces the
                        // link crosses
                        double mw = 0.0;
                        const int ijk[3] = {i, j, k};
                        for (int a = 0; a < 3; ++a) {
                            const int c = ijk[a] - C[q][a];
                            if (s->p.periodic[a] || (c >= 0 && c < extent(s, a))) continue;
                            const double* uw = s->wall_u[a][c < 0 ? 0 : 1];
                            mw += 2.0 * W[q] * (C[q][0] * uw[0] + C[q][1] * uw[1] + C[q][2] * uw[2]) / CS2;
                        }
                        gn[(size_t)q * n + x] = gt[(size_t)opposite(q) * n + x] + mw;
                    } else if (s->flag[src] == FLUID) {
                        gn[(size_t)q * n + x] = gt[(size_t)q * n + src];
                    } else {
                        any = 1;   // solid source: filled in the serial link pass below
                    }
                }
                s->has_link[x] = any;
            }

    // Link pass, serial in (cell, q) order so the force sum is reproducible.
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long x = cell_index(s, i, j, k);
                if (s->flag[x] != FLUID || !s->has_link[x]) continue;
                for (int qin = 1; qin < 19; ++qin) {
                    long src;
                    if (!neighbour(s, i, j, k, qin, -1, &src)) continue;
                    uint8_t fs = s->flag[src];
                    if (fs == FLUID) continue;
                    // Paper's notation: q points from x into the solid, the
                    // unknown is f_qbar(x, t+1) with qbar = qin.
                    int q = opposite(qin);
                    int qb = qin;
                    bool is_particle = (fs == SOLID_PARTICLE);
                    double delta;
                    if (s->p.boundary == 1) delta = 0.5;
                    else delta = is_particle ? sphere_delta(s, i, j, k, q) : plane_delta(s, i, j, k, q);
                    // cell x - c_q (one further away from the wall) must be fluid for CLI
                    long far;
                    bool far_ok = neighbour(s, i, j, k, q, -1, &far) && s->flag[far] == FLUID;
                    if (!far_ok) delta = 0.5;   // fall back to simple bounce-back
                    double kappa0 = (1.0 - 2.0 * delta) / (1.0 + 2.0 * delta);
                    double alpha = 4.0 / (1.0 + 2.0 * delta);
                    // wall velocity at x_b = x + delta c_q
                    double xc[3] = {i + 0.5, j + 0.5, k + 0.5};
                    double vb[3] = {0, 0, 0};
                    double arm[3] = {0, 0, 0};
                    if (is_particle) {
                        for (int a = 0; a < 3; ++a)
                            arm[a] = wrap_diff(s, a, xc[a] - P.x[a]) + delta * C[q][a];
                        double wr[3];
                        cross(P.w, arm, wr);
                        for (int a = 0; a < 3; ++a) vb[a] = P.u[a] + wr[a];
                    } else {
                        const double* v = (C[q][s->planes.axis] > 0) ? s->planes.v_hi : s->planes.v_lo;
                        for (int a = 0; a < 3; ++a) vb[a] = v[a];
                    }
                    double vc = vb[0] * C[q][0] + vb[1] * C[q][1] + vb[2] * C[q][2];
                    // full populations f = w + g (Sec. 2.3 works on f)
                    double ft_q = W[q] + gt[(size_t)q * n + x];
                    double ft_qb = W[qb] + gt[(size_t)qb * n + x];
                    double ft_q_far = far_ok ? (W[q] + gt[(size_t)q * n + far]) : 0.0;
                    // CLI (Sec. 2.3) with the moving-wall term alpha w_q / c_s^2 rho_0 v.c_q
                    double f_new = ft_q + kappa0 * ft_q_far - kappa0 * ft_qb - alpha * (W[q] / CS2) * 1.0 * vc;
                    gn[(size_t)qb * n + x] = f_new - W[qb];
                    // link force (Sec. 2.3): (c_q - v) ft_q(x,t) - (c_qbar - v) f_qbar(x,t+1)
                    double Fl[3];
                    for (int a = 0; a < 3; ++a)
                        Fl[a] = (C[q][a] - vb[a]) * ft_q - (C[qb][a] - vb[a]) * f_new;
                    if (is_particle) {
                        double Tl[3];
                        cross(arm, Fl, Tl);
                        for (int a = 0; a < 3; ++a) {
                            F[a] += Fl[a];
                            T[a] += Tl[a];
                        }
                    } else {
                        for (int a = 0; a < 3; ++a) s->plane_force[a] += Fl[a];
                    }
                }
            }
}

void collide_all(orc_sim* s) {
    const long n = s->n;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < n; ++x)
        if (s->flag[x] == FLUID) collide_cell(s, x);
}

// Particle update of Algorithm 1 (see common.h).
void particle_update(orc_sim* s, const double Fh[3], const double Th[3]) {
    const double ext[3] = {(double)s->p.nx, (double)s->p.ny, (double)s->p.nz};
    particle_advance(s->part, Fh, Th, s->gravity, s->p.force_average != 0, s->p.plain_mem != 0, s->p.periodic, ext,
                     s->history);
}

// Sec. 2.3: new solid flags after the particle moved; cells the sphere
// uncovers are refilled (equilibrium with the mean density of neighbours
// that are fluid before and after, and the local rigid-body velocity);
// cells it covers drop their populations.
void remap(orc_sim* s) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    const long n = s->n;
    std::vector<uint8_t> nf(n);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) nf[cell_index(s, i, j, k)] = geometry_flag(s, i, j, k);
    const Particle& P = s->part;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                long x = cell_index(s, i, j, k);
                bool was_fluid = s->flag[x] == FLUID, is_fluid = nf[x] == FLUID;
                if (!was_fluid && is_fluid) {
                    double rsum = 0;
                    int cnt = 0;
                    for (int q = 1; q < 19; ++q) {
                        long y;
                        if (!neighbour(s, i, j, k, q, +1, &y)) continue;
                        if (s->flag[y] != FLUID || nf[y] != FLUID) continue;
                        double r = 1.0;
                        for (int p = 0; p < 19; ++p) r += s->g[(size_t)p * n + y];
                        rsum += r;
                        cnt += 1;
                    }
                    double rho = cnt > 0 ? rsum / cnt : 1.0;
                    double d[3] = {wrap_diff(s, 0, (i + 0.5) - P.x[0]), wrap_diff(s, 1, (j + 0.5) - P.x[1]),
                                   wrap_diff(s, 2, (k + 0.5) - P.x[2])};
                    double wr[3];
                    cross(P.w, d, wr);
                    double u[3] = {P.u[0] + wr[0], P.u[1] + wr[1], P.u[2] + wr[2]};
                    double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                    if (s->p.refill == 1) {   // face neighbours fluid before and after the move
                        double up[3][3], um[3][3];
                        bool okp[3], okm[3];
                        for (int a = 0; a < 3; ++a)
                            for (int sgn = 0; sgn < 2; ++sgn) {
                                const int q = 1 + 2 * a + sgn;   // +e_a, then -e_a
                                long y;
                                bool ok = neighbour(s, i, j, k, q, +1, &y) && s->flag[y] == FLUID && nf[y] == FLUID;
                                double* uu = sgn == 0 ? up[a] : um[a];
                                uu[0] = uu[1] = uu[2] = 0.0;
                                if (ok)
                                    for (int p = 0; p < 19; ++p)
                                        for (int b = 0; b < 3; ++b) uu[b] += s->g[(size_t)p * n + y] * C[p][b];
                                (sgn == 0 ? okp : okm)[a] = ok;
                            }
                        refill_strain(up, okp, um, okm, u, S);
                    }
                    for (int q = 0; q < 19; ++q)
                        s->g[(size_t)q * n + x] = geq(q, rho - 1.0, u) + (s->p.refill == 1 ? grad_noneq(q, s->sp, S) : 0.0);
                } else if (was_fluid && !is_fluid) {
                    for (int q = 0; q < 19; ++q) s->g[(size_t)q * n + x] = 0.0;
                }
            }
    s->flag.swap(nf);
}

void compute_flags(orc_sim* s) {
    for (int k = 0; k < s->p.nz; ++k)
        for (int j = 0; j < s->p.ny; ++j)
            for (int i = 0; i < s->p.nx; ++i) s->flag[cell_index(s, i, j, k)] = geometry_flag(s, i, j, k);
    for (long x = 0; x < s->n; ++x)
        if (s->flag[x] != FLUID)
            for (int q = 0; q < 19; ++q) s->g[(size_t)q * s->n + x] = 0.0;
}

}  // namespace

extern "C" {

orc_sim* orc_create(const orc_params* p) {
    if (!p || p->nx <= 0 || p->ny <= 0 || p->nz <= 0 || p->tau <= 0.5) return nullptr;
    orc_sim* s = new orc_sim();
    s->p = *p;
    s->n = (long)p->nx * p->ny * p->nz;
    s->g.assign((size_t)19 * s->n, 0.0);
    s->g_new.assign((size_t)19 * s->n, 0.0);
    s->flag.assign(s->n, FLUID);
    s->has_link.assign(s->n, 0);
    // Sec. 2.1: s+ = s_nu = 1/tau; Lambda = (1/s+ - 1/2)(1/s- - 1/2)
    s->sp = 1.0 / p->tau;
    s->sm = 1.0 / (0.5 + p->magic / (p->tau - 0.5));
    s->bulk = p->bulk > 0.0 ? p->bulk : 1.0;
    s->sb = 1.0 / (0.5 + s->bulk * (p->tau - 0.5));   // Lambda_b = (1/s_b - 1/2) / (1/s_nu - 1/2)
    return s;
}

void orc_grad_noneq(double tau, const double S[9], double out[19]) {
    for (int q = 0; q < 19; ++q) out[q] = grad_noneq(q, 1.0 / tau, S);
}

void orc_destroy(orc_sim* s) { delete s; }

int orc_add_sphere(orc_sim* s, const double pos[3], double diameter, double density_ratio, double cv,
                   double cv_omega, int fixed) {
    if (s->part.present || diameter <= 0 || density_ratio <= 0) return -1;
    Particle& P = s->part;
    P = Particle();
    P.present = true;
    if (fixed < 0 || fixed > 2) return -1;
    P.fixed = P.prev_fixed = fixed;
    for (int a = 0; a < 3; ++a) P.x[a] = pos[a];
    P.D = diameter;
    P.r = 0.5 * diameter;
    P.rho_p = density_ratio;   // rho_f = rho_0 = 1 in lattice units
    P.cv = cv;
    P.cvw = cv_omega;
    P.V = M_PI * diameter * diameter * diameter / 6.0;
    compute_flags(s);
    return 0;
}

void orc_set_particle_velocity(orc_sim* s, const double u[3], const double w[3]) {
    for (int a = 0; a < 3; ++a) {
        s->part.u[a] = u[a];
        s->part.w[a] = w[a];
    }
}

void orc_set_gravity(orc_sim* s, const double g[3]) {
    for (int a = 0; a < 3; ++a) s->gravity[a] = g[a];
}

int orc_set_planes(orc_sim* s, int axis, double lo, double hi, const double v_lo[3], const double v_hi[3]) {
    if (axis < 0 || axis > 2 || !(lo < hi)) return -1;
    s->planes.present = true;
    s->planes.axis = axis;
    s->planes.lo = lo;
    s->planes.hi = hi;
    for (int a = 0; a < 3; ++a) {
        s->planes.v_lo[a] = v_lo[a];
        s->planes.v_hi[a] = v_hi[a];
    }
    compute_flags(s);
    return 0;
}

void orc_init_equilibrium(orc_sim* s, double rho, const double u[3], const double* u_field) {
    const long n = s->n;
    for (long x = 0; x < n; ++x) {
        double ux[3] = {u[0], u[1], u[2]};
        if (u_field)
            for (int a = 0; a < 3; ++a) ux[a] = u_field[(size_t)a * n + x];
        for (int q = 0; q < 19; ++q)
            s->g[(size_t)q * n + x] = (s->flag[x] == FLUID) ? geq(q, rho - 1.0, ux) : 0.0;
    }
}

void orc_set_populations(orc_sim* s, const double* g) {
    std::memcpy(s->g.data(), g, sizeof(double) * 19 * (size_t)s->n);
}

void orc_get_populations(const orc_sim* s, double* g) {
    std::memcpy(g, s->g.data(), sizeof(double) * 19 * (size_t)s->n);
}

void orc_get_flags(const orc_sim* s, uint8_t* flags) { std::memcpy(flags, s->flag.data(), (size_t)s->n); }

void orc_moments(const orc_sim* s, double* rho, double* u) {
    const long n = s->n;
    for (long x = 0; x < n; ++x) {
        double r = 1.0, m[3] = {0, 0, 0};
        for (int q = 0; q < 19; ++q) {
            double v = s->g[(size_t)q * n + x];
            r += v;
            for (int a = 0; a < 3; ++a) m[a] += v * C[q][a];
        }
        rho[x] = r;
        for (int a = 0; a < 3; ++a) u[(size_t)a * n + x] = m[a];
    }
}

void orc_step(orc_sim* s, int nsteps) {
    for (int it = 0; it < nsteps; ++it) {
        double F[3], T[3];
        stream_and_boundaries(s, F, T);
        collide_all(s);
        s->g.swap(s->g_new);
        if (s->part.present) {
            particle_update(s, F, T);
            remap(s);
        }
    }
}

int64_t orc_get_links(const orc_sim* s, int64_t* cell, int32_t* qout, double* delta, int64_t cap) {
    int64_t cnt = 0;
    for (int k = 0; k < s->p.nz; ++k)
        for (int j = 0; j < s->p.ny; ++j)
            for (int i = 0; i < s->p.nx; ++i) {
                long x = cell_index(s, i, j, k);
                if (s->flag[x] != FLUID) continue;
                for (int q = 1; q < 19; ++q) {
                    long y;
                    if (!neighbour(s, i, j, k, q, +1, &y)) continue;
                    if (s->flag[y] != SOLID_PARTICLE) continue;
                    if (cnt < cap) {
                        cell[cnt] = x;
                        qout[cnt] = q;
                        delta[cnt] = sphere_delta(s, i, j, k, q);
                    }
                    ++cnt;
                }
            }
    return cnt;
}

void orc_get_particle(const orc_sim* s, double out[24]) {
    const Particle& P = s->part;
    for (int a = 0; a < 3; ++a) {
        out[a] = P.Fh[a];
        out[3 + a] = P.Th[a];
        out[6 + a] = P.x[a];
        out[9 + a] = P.u[a];
        out[12 + a] = P.w[a];
        out[15 + a] = P.a[a];
        out[18 + a] = P.b[a];
        out[21 + a] = P.Fp[a];
    }
}

int64_t orc_get_history(const orc_sim* s, double* out, int64_t cap_steps) {
    int64_t steps = (int64_t)(s->history.size() / 15);
    int64_t m = steps < cap_steps ? steps : cap_steps;
    if (out && m > 0) std::memcpy(out, s->history.data(), sizeof(double) * 15 * (size_t)m);
    return steps;
}

void orc_get_plane_force(const orc_sim* s, double out[3]) {
    for (int a = 0; a < 3; ++a) out[a] = s->plane_force[a];
}

int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_set_particle_fixed(orc_sim* s, int fixed) {
    if (!s->part.present || fixed < 0 || fixed > 2) return -1;
    s->part.fixed = fixed;
    return 0;
}

int orc_set_wall_velocity(orc_sim* s, int axis, int side, const double u[3]) {
    if (axis < 0 || axis > 2 || side < 0 || side > 1 || s->p.periodic[axis]) return -1;
    for (int a = 0; a < 3; ++a) s->wall_u[axis][side][a] = u[a];
    return 0;
}

void orc_particle_only_step(orc_sim* s, const double F_hyd[3], const double T_hyd[3]) {
    particle_update(s, F_hyd, T_hyd);
}

}  // extern "C"
