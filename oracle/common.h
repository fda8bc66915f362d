/*
 * Oracle, pieces shared by the uniform and the refined grid restatements:
 * the D3Q19 lattice, the incompressible equilibrium and the particle update
 * of Algorithm 1.  TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).
 */
#ifndef LBM_ORACLE_COMMON_H
#define LBM_ORACLE_COMMON_H
#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

namespace orc {

// ---------------------------------------------------------------- lattice
// D3Q19 velocity set (Sec. 2.1 names D3Q19; the set and weights are the
// standard ones: w0 = 1/3, faces 1/18, edges 1/36, c_s^2 = 1/3).
inline constexpr int C[19][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1},
    {1, 0, -1}, {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
inline constexpr double W[19] = {1.0 / 3.0,
                      1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                      1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                      1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
inline constexpr double CS2 = 1.0 / 3.0;

inline int opposite(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }

enum : uint8_t { FLUID = 0, SOLID_PARTICLE = 1, SOLID_PLANE = 2 };

struct Particle {
    bool present = false;
    int fixed = 0;        // held degrees of freedom: 0 none, 1 translation and rotation, 2 translation only
    int prev_fixed = 0;   // the value of fixed in the previous step
    double x[3] = {0, 0, 0};
    double u[3] = {0, 0, 0};   // wall velocity seen by the fluid (u at t + 1/2)
    double w[3] = {0, 0, 0};
    double a[3] = {0, 0, 0};   // acceleration of the previous step (a_{p,t-1})
    double b[3] = {0, 0, 0};   // angular acceleration of the previous step
    double Fh[3] = {0, 0, 0}, Th[3] = {0, 0, 0};        // hydrodynamic, this step
    double Fh_old[3] = {0, 0, 0}, Th_old[3] = {0, 0, 0};  // previous step
    double Fp[3] = {0, 0, 0};
    double D = 0, r = 0, rho_p = 1, cv = 0, cvw = 0, V = 0;
    long steps = 0;
};

// Incompressible equilibrium deviation (He & Luo form cited in Sec. 2.1,
// rho_0 = 1): f_eq - w = w (drho + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u).
inline double geq(int q, double drho, const double u[3]) {
    double cu = C[q][0] * u[0] + C[q][1] * u[1] + C[q][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W[q] * (drho + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

// ------------------------------------------------------------ MRT (Sec. 2.1)
// Moment basis of the D3Q19 MRT model the paper uses (transformation matrix
// of Duenweg et al. 2007): row k of M is the polynomial e_k evaluated at
// c_q.  Rows 0-3: density and momentum; 4: |c|^2 - 1 (bulk); 5-9: the five
// shear components; 10-15: six odd third-order modes; 16: 3|c|^4 - 6|c|^2 + 1
// (isotropic fourth order); 17-18: two anisotropic fourth-order modes.  The
// rows are orthogonal under the lattice weights.
inline double mrt_basis(int k, int q) {
    const double x = C[q][0], y = C[q][1], z = C[q][2];
    const double c2 = x * x + y * y + z * z;
    switch (k) {
        case 0: return 1.0;
        case 1: return x;
        case 2: return y;
        case 3: return z;
        case 4: return c2 - 1.0;
        case 5: return 3.0 * x * x - c2;
        case 6: return y * y - z * z;
        case 7: return x * y;
        case 8: return y * z;
        case 9: return z * x;
        case 10: return (3.0 * c2 - 5.0) * x;
        case 11: return (3.0 * c2 - 5.0) * y;
        case 12: return (3.0 * c2 - 5.0) * z;
        case 13: return (y * y - z * z) * x;
        case 14: return (z * z - x * x) * y;
        case 15: return (x * x - y * y) * z;
        case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
        case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
        default: return (2.0 * c2 - 3.0) * (y * y - z * z);
    }
}

// Relaxation rate of moment k (Sec. 2.1): 0 for the conserved moments,
// s_b for the bulk and the isotropic fourth-order mode, s_nu for the shear
// modes and the two anisotropic fourth-order modes, s_nu^- for the six odd
// modes (the counts of the paper's relaxation matrix: 4 zeros, 2 s_b, 7
// s_nu, 6 s_nu^-).
inline double mrt_rate(int k, double s_nu, double s_minus, double s_b) {
    if (k < 4) return 0.0;
    if (k == 4 || k == 16) return s_b;
    if (k >= 10 && k <= 15) return s_minus;
    return s_nu;
}

// M^-1 by Gauss-Jordan elimination with partial pivoting (computed once).
inline const double* mrt_inverse() {
    static const std::vector<double> inv = [] {
        double a[19][38];
        for (int k = 0; k < 19; ++k)
            for (int q = 0; q < 38; ++q) a[k][q] = q < 19 ? mrt_basis(k, q) : (q - 19 == k ? 1.0 : 0.0);
        for (int col = 0; col < 19; ++col) {
            int piv = col;
            for (int r = col + 1; r < 19; ++r)
                if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
            for (int q = 0; q < 38; ++q) std::swap(a[col][q], a[piv][q]);
            const double d = a[col][col];
            for (int q = 0; q < 38; ++q) a[col][q] /= d;
            for (int r = 0; r < 19; ++r) {
                if (r == col) continue;
                const double f = a[r][col];
                if (f != 0.0)
                    for (int q = 0; q < 38; ++q) a[r][q] -= f * a[col][q];
            }
        }
        std::vector<double> m(19 * 19);
        for (int r = 0; r < 19; ++r)
            for (int q = 0; q < 19; ++q) m[(size_t)r * 19 + q] = a[r][19 + q];
        return m;
    }();
    return inv.data();
}

// MRT collision of one cell's deviations g (Sec. 2.1, C = M^-1 S M):
// m = M g, m_eq = M g_eq, m' = m - S (m - m_eq) + (I - S/2) M src, g' = M^-1 m'.
// src (may be NULL): the velocity-space body-force source of the cell.
inline void mrt_collide(const double g[19], const double geq_dev[19], const double* src, double s_nu,
                        double s_minus, double s_b, double out[19]) {
    const double* Minv = mrt_inverse();
    double m[19];
    for (int k = 0; k < 19; ++k) {
        double mk = 0.0, mq = 0.0, ms = 0.0;
        for (int q = 0; q < 19; ++q) {
            mk += mrt_basis(k, q) * g[q];
            mq += mrt_basis(k, q) * geq_dev[q];
            if (src) ms += mrt_basis(k, q) * src[q];
        }
        const double s = mrt_rate(k, s_nu, s_minus, s_b);
        m[k] = mk - s * (mk - mq) + (1.0 - 0.5 * s) * ms;
    }
    for (int q = 0; q < 19; ++q) {
        double v = 0.0;
        for (int k = 0; k < 19; ++k) v += Minv[(size_t)q * 19 + k] * m[k];
        out[q] = v;
    }
}

// ------------------------------------------------ Grad refill (Sec. 2.3)
// The paper refills uncovered cells with the approach of Dorschner et al.
// (2015), Grad's approximation using local velocity gradients.  Reading:
// equilibrium at the mean density of the neighbours and the wall velocity,
// plus Grad's non-equilibrium part from the strain rate S.  The refilled
// state is a post-collision state, so the first-order Chapman-Enskog stress
// enters after one collision: -3 w_q (1 - s+)/s+ Q_q:S, Q_q = c_q c_q - I/3.
inline double grad_noneq(int q, double sp, const double S[9]) {
    double qs = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) qs += (C[q][a] * C[q][b] - (a == b ? 1.0 / 3.0 : 0.0)) * S[3 * a + b];
    return -3.0 * W[q] * (1.0 - sp) / sp * qs;
}

// Strain rate at an uncovered cell from the velocities of its six face
// neighbours (up[a]: at x + e_a, um[a]: at x - e_a, each used only where
// that neighbour is fluid) and the wall velocity uw at the cell: central
// differences where both are fluid, one-sided against uw where one is,
// zero where neither is.  S = (grad u + grad u^T) / 2, row major.
inline void refill_strain(const double up[3][3], const bool okp[3], const double um[3][3], const bool okm[3],
                          const double uw[3], double S[9]) {
    double G[3][3];   // G[a][b] = d u_b / d x_a
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            if (okp[a] && okm[a]) G[a][b] = 0.5 * (up[a][b] - um[a][b]);
            else if (okp[a]) G[a][b] = up[a][b] - uw[b];
            else if (okm[a]) G[a][b] = uw[b] - um[a][b];
            else G[a][b] = 0.0;
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[3 * a + b] = 0.5 * (G[a][b] + G[b][a]);
}

inline void cross(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

// Sec. 2.2 and Sec. 3.3 (Algorithm 1): average the hydrodynamic force and
// torque over two steps, add gravity/buoyancy and the virtual force/torque
// (built from the previous accelerations), and advance with Velocity Verlet
// using the virtually increased mass and moment of inertia.  The paper's
// position and velocity updates are taken in kick-drift-kick order: the
// first step has no preceding half kick.
inline void particle_advance(Particle& P, const double Fh[3], const double Th[3], const double gravity[3],
                             bool force_average, bool plain_mem, const int periodic[3], const double extent[3],
                             std::vector<double>& history) {
    double Fbar[3], Tbar[3];
    for (int a = 0; a < 3; ++a) {
        if (force_average && P.steps > 0) {
            Fbar[a] = 0.5 * (Fh[a] + P.Fh_old[a]);
            Tbar[a] = 0.5 * (Th[a] + P.Th_old[a]);
        } else {
            Fbar[a] = Fh[a];
            Tbar[a] = Th[a];
        }
        P.Fh[a] = Fh[a];
        P.Th[a] = Th[a];
        P.Fh_old[a] = Fh[a];
        P.Th_old[a] = Th[a];
    }
    const double V = P.V, r = P.r;
    double Fp[3], Tp[3], m, I;
    if (plain_mem) {
        // Sec. 2.2: F_p = F_g + F_hyd, T_p = T_hyd, m = rho_p V, I = 2/5 m r^2
        m = P.rho_p * V;
        I = 0.4 * P.rho_p * V * r * r;
        for (int a = 0; a < 3; ++a) {
            double Fg = (P.rho_p - 1.0) * gravity[a] * V;
            Fp[a] = Fbar[a] + Fg;
            Tp[a] = Tbar[a];
        }
    } else {
        // Sec. 3.3: F_v = C_v rho_f V a_{t-1}, T_v = 2/5 C_vw rho_f V r^2 beta_{t-1},
        // m = (rho_p + C_v rho_f) V, I = 2/5 (rho_p + C_vw rho_f) V r^2, rho_f = 1
        m = (P.rho_p + P.cv) * V;
        I = 0.4 * (P.rho_p + P.cvw) * V * r * r;
        for (int a = 0; a < 3; ++a) {
            double Fg = (P.rho_p - 1.0) * gravity[a] * V;
            double Fv = P.cv * V * P.a[a];
            double Tv = 0.4 * P.cvw * V * r * r * P.b[a];
            Fp[a] = Fbar[a] + Fg + Fv;
            Tp[a] = Tbar[a] + Tv;
        }
    }
    for (int a = 0; a < 3; ++a) P.Fp[a] = Fp[a];
    // A held group (translation, rotation) keeps its velocity and has zero
    // acceleration, so the virtual force or torque of the next step is zero;
    // a group released in this step starts its kick-drift-kick afresh (no
    // half kick completing a previous step).
    const bool tfree = P.fixed == 0, rfree = P.fixed != 1;
    const bool tprev = P.steps > 0 && P.prev_fixed == 0, rprev = P.steps > 0 && P.prev_fixed != 1;
    for (int a = 0; a < 3; ++a) {
        if (tfree) {
            if (tprev) P.u[a] += Fp[a] / (2.0 * m);   // second half kick of the previous step completes u(t)
            P.a[a] = Fp[a] / m;
            P.u[a] += Fp[a] / (2.0 * m);              // first half kick, then drift with u(t + 1/2)
            P.x[a] += P.u[a];
            if (periodic[a]) {
                double L = extent[a];
                if (P.x[a] >= L) P.x[a] -= L;
                else if (P.x[a] < 0.0) P.x[a] += L;
            }
        } else {
            P.a[a] = 0.0;
        }
        if (rfree) {
            if (rprev) P.w[a] += Tp[a] / (2.0 * I);
            P.b[a] = Tp[a] / I;
            P.w[a] += Tp[a] / (2.0 * I);
        } else {
            P.b[a] = 0.0;
        }
    }
    P.prev_fixed = P.fixed;
    P.steps += 1;
    double rec[15];
    for (int a = 0; a < 3; ++a) {
        rec[a] = Fh[a];
        rec[3 + a] = Th[a];
        rec[6 + a] = P.x[a];
        rec[9 + a] = P.u[a];
        rec[12 + a] = P.w[a];
    }
    history.insert(history.end(), rec, rec + 15);
}

}  // namespace orc

#endif
