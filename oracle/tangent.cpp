/*
 * Oracle, tangent-linear model of the mean drag on a fixed sphere.
 *
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).  Plain loops, FP64.
 *
 * Setting: periodic box, one sphere held fixed (zero wall velocity), CLI
 * links of Sec. 2.3, constant fluid body force, fluid started at the
 * incompressible equilibrium of a velocity field u0.  Objective: the mean
 * over N steps of one component of the momentum-exchange force,
 * J = (1/N) sum_{n=1..N} F_a^n.
 *
 * The step of uniform.cpp (pull streaming with CLI links, link force on full
 * populations, TRT collision with the Guo-type source) is written here once
 * more over a dual number (value, derivative along one direction of the
 * inputs tau, body force and u0), so the derivative part is the exact
 * forward-mode derivative of the same arithmetic.  The geometry (solid flags
 * and wall distances) is taken from uniform.cpp through its C interface.
 * The source term is always applied: it adds exact zeros to the value when
 * the body force is zero, and its derivative is what d/dF needs there.
 */
#include "lbm_oracle.h"
#include "common.h"

#include <cmath>
#include <cstring>
#include <vector>

using namespace orc;

namespace {

// value and derivative along the chosen direction
struct Dual {
    double v = 0.0, d = 0.0;
    Dual() = default;
    Dual(double value) : v(value), d(0.0) {}
    Dual(double value, double deriv) : v(value), d(deriv) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual& operator+=(Dual& a, Dual b) { return a = a + b; }

Dual geq_dual(int q, Dual drho, const Dual u[3]) {
    Dual cu = Dual(C[q][0]) * u[0] + Dual(C[q][1]) * u[1] + Dual(C[q][2]) * u[2];
    Dual uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return Dual(W[q]) * (drho + Dual(3.0) * cu + Dual(4.5) * cu * cu - Dual(1.5) * uu);
}

struct Tlm {
    int nx, ny, nz;
    long n;
    std::vector<uint8_t> flag;
    std::vector<double> delta;   // [19][n] wall distance of link (x, q into the solid), -1 where none
    std::vector<Dual> g, gn;     // [19][n]
    Dual sp, sm, F[3];
    int boundary;

    long idx(int i, int j, int k) const { return (long)i + (long)nx * ((long)j + (long)ny * (long)k); }
    long shifted(int i, int j, int k, int q, int sign) const {
        int a = (i + sign * C[q][0] + nx) % nx, b = (j + sign * C[q][1] + ny) % ny, c = (k + sign * C[q][2] + nz) % nz;
        return idx(a, b, c);
    }
};

// Pull streaming with the CLI rule of Sec. 2.3 on sphere links (wall at
// rest), and the link force (c_q - v) f~_q(x) - (c_qbar - v) f_qbar(x, t+1)
// summed in (cell, incoming direction) order.
void stream(Tlm& T, Dual Fsum[3]) {
    const long n = T.n;
    for (int a = 0; a < 3; ++a) Fsum[a] = Dual(0.0);
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < T.nz; ++k)
        for (int j = 0; j < T.ny; ++j)
            for (int i = 0; i < T.nx; ++i) {
                const long x = T.idx(i, j, k);
                if (T.flag[x] != FLUID) {
                    for (int q = 0; q < 19; ++q) T.gn[(size_t)q * n + x] = Dual(0.0);
                    continue;
                }
                for (int q = 0; q < 19; ++q) {
                    const long src = T.shifted(i, j, k, q, -1);
                    if (T.flag[src] == FLUID) T.gn[(size_t)q * n + x] = T.g[(size_t)q * n + src];
                }
            }
    for (int k = 0; k < T.nz; ++k)
        for (int j = 0; j < T.ny; ++j)
            for (int i = 0; i < T.nx; ++i) {
                const long x = T.idx(i, j, k);
                if (T.flag[x] != FLUID) continue;
                for (int qin = 1; qin < 19; ++qin) {
                    const long src = T.shifted(i, j, k, qin, -1);
                    if (T.flag[src] == FLUID) continue;
                    const int q = opposite(qin);   // from x into the solid
                    double delta = T.boundary == 1 ? 0.5 : T.delta[(size_t)q * n + x];
                    const long far = T.shifted(i, j, k, q, -1);
                    const bool far_ok = T.flag[far] == FLUID;
                    if (!far_ok) delta = 0.5;
                    const Dual kappa0 = Dual((1.0 - 2.0 * delta) / (1.0 + 2.0 * delta));
                    const Dual ft_q = Dual(W[q]) + T.g[(size_t)q * n + x];
                    const Dual ft_qb = Dual(W[qin]) + T.g[(size_t)qin * n + x];
                    const Dual ft_far = far_ok ? Dual(W[q]) + T.g[(size_t)q * n + far] : Dual(0.0);
                    const Dual f_new = ft_q + kappa0 * ft_far - kappa0 * ft_qb;
                    T.gn[(size_t)qin * n + x] = f_new - Dual(W[qin]);
                    for (int a = 0; a < 3; ++a)
                        Fsum[a] += Dual(C[q][a]) * ft_q - Dual(C[qin][a]) * f_new;
                }
            }
}

// TRT collision with the Guo-type source of uniform.cpp (Sec. 2.1).
void collide(Tlm& T) {
    const long n = T.n;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < n; ++x) {
        if (T.flag[x] != FLUID) continue;
        Dual drho(0.0), u[3] = {Dual(0.0), Dual(0.0), Dual(0.0)};
        for (int q = 0; q < 19; ++q) {
            const Dual v = T.gn[(size_t)q * n + x];
            drho += v;
            for (int a = 0; a < 3; ++a) u[a] += v * Dual(C[q][a]);
        }
        for (int a = 0; a < 3; ++a) u[a] += Dual(0.5) * T.F[a];
        const Dual uF = u[0] * T.F[0] + u[1] * T.F[1] + u[2] * T.F[2];
        Dual out[19];
        {
            const Dual e = geq_dual(0, drho, u);
            const Dual gq = T.gn[x];
            out[0] = gq - T.sp * (gq - e);
            out[0] += (Dual(1.0) - Dual(0.5) * T.sp) * Dual(W[0]) * (Dual(-3.0) * uF);
        }
        for (int q = 1; q < 19; q += 2) {
            const int qb = q + 1;
            const Dual gq = T.gn[(size_t)q * n + x], gb = T.gn[(size_t)qb * n + x];
            const Dual eq = geq_dual(q, drho, u), eb = geq_dual(qb, drho, u);
            const Dual gp = Dual(0.5) * (gq + gb), gm = Dual(0.5) * (gq - gb);
            const Dual ep = Dual(0.5) * (eq + eb), em = Dual(0.5) * (eq - eb);
            const Dual dp = T.sp * (gp - ep), dm = T.sm * (gm - em);
            out[q] = gq - dp - dm;
            out[qb] = gb - dp + dm;
            const Dual cu = Dual(C[q][0]) * u[0] + Dual(C[q][1]) * u[1] + Dual(C[q][2]) * u[2];
            const Dual cF = Dual(C[q][0]) * T.F[0] + Dual(C[q][1]) * T.F[1] + Dual(C[q][2]) * T.F[2];
            const Dual Sp = Dual(W[q]) * (Dual(9.0) * cu * cF - Dual(3.0) * uF);
            const Dual Sm = Dual(W[q]) * (Dual(3.0) * cF);
            out[q] += (Dual(1.0) - Dual(0.5) * T.sp) * Sp + (Dual(1.0) - Dual(0.5) * T.sm) * Sm;
            out[qb] += (Dual(1.0) - Dual(0.5) * T.sp) * Sp - (Dual(1.0) - Dual(0.5) * T.sm) * Sm;
        }
        for (int q = 0; q < 19; ++q) T.gn[(size_t)q * n + x] = out[q];
    }
}

}  // namespace

extern "C" {

double orc_drag_tangent(const orc_drag_params* p, const double* u0, int nsteps, double dtau, const double dforce[3],
                        const double* du0, int axis, double* dJ, double* force_out) {
    if (!p || nsteps <= 0 || axis < 0 || axis > 2) return NAN;
    // geometry from the uniform oracle: flags and link distances
    orc_params op;
    std::memset(&op, 0, sizeof(op));
    op.nx = p->nx;
    op.ny = p->ny;
    op.nz = p->nz;
    op.periodic[0] = op.periodic[1] = op.periodic[2] = 1;
    op.tau = p->tau;
    op.magic = p->magic;
    op.boundary = p->boundary;
    orc_sim* s = orc_create(&op);
    if (!s) return NAN;
    orc_add_sphere(s, p->pos, p->diameter, 1.0, 0.0, 0.0, 1);
    Tlm T;
    T.nx = p->nx;
    T.ny = p->ny;
    T.nz = p->nz;
    T.n = (long)T.nx * T.ny * T.nz;
    T.boundary = p->boundary;
    T.flag.resize(T.n);
    orc_get_flags(s, T.flag.data());
    const int64_t nl = orc_get_links(s, nullptr, nullptr, nullptr, 0);
    std::vector<int64_t> lc(nl);
    std::vector<int32_t> lq(nl);
    std::vector<double> ld(nl);
    orc_get_links(s, lc.data(), lq.data(), ld.data(), nl);
    orc_destroy(s);
    T.delta.assign((size_t)19 * T.n, -1.0);
    for (int64_t i = 0; i < nl; ++i) T.delta[(size_t)lq[i] * T.n + lc[i]] = ld[i];

    // parameters as dual numbers: s+ = 1/tau, s- from the magic parameter (Sec. 2.1)
    const Dual tau(p->tau, dtau);
    T.sp = Dual(1.0) / tau;
    T.sm = Dual(1.0) / (Dual(0.5) + Dual(p->magic) / (tau - Dual(0.5)));
    for (int a = 0; a < 3; ++a) T.F[a] = Dual(p->body_force[a], dforce ? dforce[a] : 0.0);

    // initial state: equilibrium of u0 on fluid cells (drho = 0)
    const long n = T.n;
    T.g.assign((size_t)19 * n, Dual(0.0));
    T.gn.assign((size_t)19 * n, Dual(0.0));
    for (long x = 0; x < n; ++x) {
        if (T.flag[x] != FLUID) continue;
        Dual u[3];
        for (int a = 0; a < 3; ++a)
            u[a] = Dual(u0 ? u0[(size_t)a * n + x] : 0.0, du0 ? du0[(size_t)a * n + x] : 0.0);
        for (int q = 0; q < 19; ++q) T.g[(size_t)q * n + x] = geq_dual(q, Dual(0.0), u);
    }

    Dual J(0.0);
    for (int it = 0; it < nsteps; ++it) {
        Dual Fs[3];
        stream(T, Fs);
        collide(T);
        T.g.swap(T.gn);
        J += Fs[axis];
        if (force_out)
            for (int a = 0; a < 3; ++a) force_out[(size_t)it * 3 + a] = Fs[a].v;
    }
    J = J / Dual((double)nsteps);
    if (dJ) *dJ = J.d;
    return J.v;
}

}  // extern "C"
