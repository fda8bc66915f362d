// Device arithmetic shared by the uniform and the refined-grid kernels:
// TRT collision on deviations (Sec. 2.1) and the sphere-link geometry of
// the CLI boundary (Sec. 2.3).
#pragma once

#include "internal.h"

namespace lbmp {

// Minimum-image difference for periodic axes.
__device__ __forceinline__ double wrap_diff(double d, int n, int periodic) {
    if (!periodic) return d;
    double L = (double)n;
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

// Wall distance fraction along c_q from the fluid cell centre (Sec. 2.3):
// smallest root in (0,1] of |d + s c|^2 = r^2.
__device__ __forceinline__ double link_delta(const double d[3], int q, double r) {
    double c0 = cx(q), c1 = cy(q), c2 = cz(q);
    double cc = c0 * c0 + c1 * c1 + c2 * c2;
    double dc = d[0] * c0 + d[1] * c1 + d[2] * c2;
    double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double disc = dc * dc - cc * (dd - r * r);
    disc = disc < 0.0 ? 0.0 : disc;
    double s = (-dc - sqrt(disc)) / cc;
    return s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
}

// TRT collision on deviations (Sec. 2.1, Lambda_b = 1): the symmetric part of
// each pair relaxes with s+, the antisymmetric part with s-; incompressible
// equilibrium with rho_0 = 1; optional Guo-type source split the same way.
template <typename A, bool FORCED>
__device__ __forceinline__ void trt_collide(A (&g)[19], const CollideParams<A>& P, int* status) {
    A drho = A(0), jx = A(0), jy = A(0), jz = A(0);
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        drho += g[q];
        if (cx(q) == 1) jx += g[q];
        if (cx(q) == -1) jx -= g[q];
        if (cy(q) == 1) jy += g[q];
        if (cy(q) == -1) jy -= g[q];
        if (cz(q) == 1) jz += g[q];
        if (cz(q) == -1) jz -= g[q];
    }
    A ux = jx, uy = jy, uz = jz;
    if (FORCED) {
        ux += A(0.5) * P.F[0];
        uy += A(0.5) * P.F[1];
        uz += A(0.5) * P.F[2];
    }
    const A uu = ux * ux + uy * uy + uz * uz;
    if (!(uu <= A(0.09))) atomicOr(status, STATUS_UNSTABLE_FLUID);
    const A sp = P.sp, sm = P.sm;
    {
        const A e0 = wgt<A>(0) * (drho - A(1.5) * uu);
        A o = g[0] - sp * (g[0] - e0);
        if (FORCED) {
            const A uF = ux * P.F[0] + uy * P.F[1] + uz * P.F[2];
            o += (A(1) - A(0.5) * sp) * wgt<A>(0) * (A(-3) * uF);
        }
        g[0] = o;
    }
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        const A cu = A(cx(q)) * ux + A(cy(q)) * uy + A(cz(q)) * uz;
        const A w = wgt<A>(q);
        const A ep = w * (drho + A(4.5) * cu * cu - A(1.5) * uu);
        const A em = w * (A(3) * cu);
        const A gp = A(0.5) * (g[q] + g[q + 1]);
        const A gm = A(0.5) * (g[q] - g[q + 1]);
        const A dp = sp * (gp - ep);
        const A dm = sm * (gm - em);
        A a = g[q] - dp - dm;
        A b = g[q + 1] - dp + dm;
        if (FORCED) {
            const A cF = A(cx(q)) * P.F[0] + A(cy(q)) * P.F[1] + A(cz(q)) * P.F[2];
            const A uF = ux * P.F[0] + uy * P.F[1] + uz * P.F[2];
            const A Sp = (A(1) - A(0.5) * sp) * w * (A(9) * cu * cF - A(3) * uF);
            const A Sm = (A(1) - A(0.5) * sm) * w * (A(3) * cF);
            a += Sp + Sm;
            b += Sp - Sm;
        }
        g[q] = a;
        g[q + 1] = b;
    }
}

}  // namespace lbmp

namespace lbmp {

// Warp-cooperative TRT collision: lane q (< 19) holds population q of one
// cell; lanes 19..31 hold 0 and take part in the shuffles.  Returns the
// post-collision value of the lane's population (same arithmetic as
// trt_collide, reduced across the warp).
template <typename A>
__device__ __forceinline__ A warp_sum(A v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ int lane_c(int lane, int axis) {
    // c_q components for q = lane < 19 (0 for idle lanes)
    const int q = lane < 19 ? lane : 0;
    switch (axis) {
        case 0: return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
                     : ((q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0);
        case 1: return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
                     : ((q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0);
        default: return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
                      : ((q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0);
    }
}

template <typename A, bool FORCED>
__device__ __forceinline__ A warp_trt_collide(A gq, int lane, const CollideParams<A>& P, int* status) {
    const int c0 = lane_c(lane, 0), c1 = lane_c(lane, 1), c2 = lane_c(lane, 2);
    const A drho = warp_sum<A>(gq);
    A ux = warp_sum<A>(A(c0) * gq), uy = warp_sum<A>(A(c1) * gq), uz = warp_sum<A>(A(c2) * gq);
    if (FORCED) {
        ux += A(0.5) * P.F[0];
        uy += A(0.5) * P.F[1];
        uz += A(0.5) * P.F[2];
    }
    const A uu = ux * ux + uy * uy + uz * uz;
    if (lane == 0 && !(uu <= A(0.09))) atomicOr(status, STATUS_UNSTABLE_FLUID);
    const int partner = lane == 0 ? 0 : (lane < 19 ? ((lane & 1) ? lane + 1 : lane - 1) : lane);
    const A gb = __shfl_sync(0xffffffffu, gq, partner);
    const A w = lane == 0 ? A(1) / A(3) : (lane <= 6 ? A(1) / A(18) : A(1) / A(36));
    const A cu = A(c0) * ux + A(c1) * uy + A(c2) * uz;
    const A ep = w * (drho + A(4.5) * cu * cu - A(1.5) * uu);
    const A em = w * (A(3) * cu);
    const A gp = A(0.5) * (gq + gb), gm = A(0.5) * (gq - gb);
    A out = gq - P.sp * (gp - ep) - P.sm * (gm - em);
    if (FORCED) {
        const A cF = A(c0) * P.F[0] + A(c1) * P.F[1] + A(c2) * P.F[2];
        const A uF = ux * P.F[0] + uy * P.F[1] + uz * P.F[2];
        out += (A(1) - A(0.5) * P.sp) * w * (A(9) * cu * cF - A(3) * uF) + (A(1) - A(0.5) * P.sm) * w * (A(3) * cF);
    }
    return lane < 19 ? out : A(0);
}

// CLI link of Sec. 2.3 for the fluid cell at distance d from the sphere
// centre, incoming direction q (k = opp(q) points into the solid):
// returns the new deviation g_q and adds the link's momentum-exchange force
// and torque (FP64, on full populations).
template <typename A>
__device__ __forceinline__ A cli_link(int q, const double d[3], double r, double delta, A gt_k, A gt_q, A gt_far,
                                      const ParticleState& Pp, double F[3], double T[3]) {
    const int k = opp(q);
    const int ck[3] = {lane_c(k, 0), lane_c(k, 1), lane_c(k, 2)};
    const double kappa0 = (1.0 - 2.0 * delta) / (1.0 + 2.0 * delta);
    const double alpha = 4.0 / (1.0 + 2.0 * delta);
    const double arm[3] = {d[0] + delta * ck[0], d[1] + delta * ck[1], d[2] + delta * ck[2]};
    const double vb[3] = {Pp.u[0] + (Pp.w[1] * arm[2] - Pp.w[2] * arm[1]),
                          Pp.u[1] + (Pp.w[2] * arm[0] - Pp.w[0] * arm[2]),
                          Pp.u[2] + (Pp.w[0] * arm[1] - Pp.w[1] * arm[0])};
    const double vc = vb[0] * ck[0] + vb[1] * ck[1] + vb[2] * ck[2];
    const double wk = k == 0 ? 1.0 / 3.0 : (k <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    const A gnew = gt_k + A(kappa0) * gt_far - A(kappa0) * gt_q - A(alpha * 3.0 * wk * vc);
    const double ftk = wk + (double)gt_k;
    const double fnew = wk + (double)gnew;
    const double Fl[3] = {(ck[0] + vb[0]) * fnew + (ck[0] - vb[0]) * ftk,
                          (ck[1] + vb[1]) * fnew + (ck[1] - vb[1]) * ftk,
                          (ck[2] + vb[2]) * fnew + (ck[2] - vb[2]) * ftk};
    F[0] += Fl[0];
    F[1] += Fl[1];
    F[2] += Fl[2];
    T[0] += arm[1] * Fl[2] - arm[2] * Fl[1];
    T[1] += arm[2] * Fl[0] - arm[0] * Fl[2];
    T[2] += arm[0] * Fl[1] - arm[1] * Fl[0];
    return gnew;
}

}  // namespace lbmp

namespace lbmp {

// Source coordinate x - c along one axis; -1 when it leaves through a wall.
__device__ __forceinline__ int src_coord(int x, int c, int n, int periodic) {
    int s = x - c;
    if (s < 0) return periodic ? s + n : -1;
    if (s >= n) return periodic ? s - n : -1;
    return s;
}

// Cell centre inside the closed ball.  Explicit round-to-nearest products and
// sums (no contraction) so the predicate is evaluated exactly as written.
__device__ __forceinline__ bool inside_ball(int i, int j, int k, const GridDesc& G, const ParticleState& P) {
    double dx = wrap_diff(__dsub_rn((double)i + 0.5, P.x[0]), G.nx, G.periodic[0]);
    double dy = wrap_diff(__dsub_rn((double)j + 0.5, P.x[1]), G.ny, G.periodic[1]);
    double dz = wrap_diff(__dsub_rn((double)k + 0.5, P.x[2]), G.nz, G.periodic[2]);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 <= __dmul_rn(P.r, P.r);
}

// Algorithm 1 after the LBM step, on the staged particle record.
__device__ __forceinline__ void particle_advance(ParticleState& P, const double FT[6], const GridDesc& G,
                                                 double* __restrict__ history, int hist_cap,
                                                 int* __restrict__ status) {
    const double Fh[3] = {FT[0], FT[1], FT[2]};
    const double Th[3] = {FT[3], FT[4], FT[5]};
    const double V = P.V, r = P.r;
    const double m = (P.rho_p + P.cv) * V;
    const double I = 0.4 * (P.rho_p + P.cvw) * V * r * r;
    const double inv_m = 1.0 / m, inv_I = 1.0 / I;
    const bool avg = P.force_average && P.steps > 0;
    double xold[3];
    for (int a = 0; a < 3; ++a) {
        const double Fbar = avg ? 0.5 * (Fh[a] + P.Fh_old[a]) : Fh[a];
        const double Tbar = avg ? 0.5 * (Th[a] + P.Th_old[a]) : Th[a];
        P.Fh[a] = Fh[a];
        P.Th[a] = Th[a];
        P.Fh_old[a] = Fh[a];
        P.Th_old[a] = Th[a];
        const double Fg = (P.rho_p - 1.0) * P.g[a] * V;
        const double Fv = P.cv * V * P.a[a];
        const double Tv = 0.4 * P.cvw * V * r * r * P.b[a];
        const double Fp = Fbar + Fg + Fv;
        const double Tp = Tbar + Tv;
        P.Fp[a] = Fp;
        xold[a] = P.x[a];
        const double acc = Fp * inv_m, bet = Tp * inv_I;
        if (!P.fixed) {
            if (P.steps > 0) {   // second half kick of the previous step completes u(t)
                P.u[a] += 0.5 * acc;
                P.w[a] += 0.5 * bet;
            }
            P.a[a] = acc;
            P.b[a] = bet;
            P.u[a] += 0.5 * acc;   // first half kick, then drift with u(t + 1/2)
            P.w[a] += 0.5 * bet;
            P.x[a] += P.u[a];
        } else {
            P.a[a] = acc;
            P.b[a] = bet;
        }
    }
    const int n3[3] = {G.nx, G.ny, G.nz};
    for (int a = 0; a < 3; ++a) {
        if (fabs(P.x[a] - xold[a]) > 0.5 || !(fabs(P.u[a]) < 0.5)) atomicOr(status, STATUS_PARTICLE_JUMP);
        if (G.periodic[a]) {   // keep the centre inside the periodic box
            const double L = (double)n3[a];
            if (P.x[a] >= L) P.x[a] -= L;
            else if (P.x[a] < 0.0) P.x[a] += L;
        }
    }
    if (hist_cap > 0) {
        double* h = history + (size_t)(P.steps % hist_cap) * 15;
        for (int a = 0; a < 3; ++a) {
            h[a] = Fh[a];
            h[3 + a] = Th[a];
            h[6 + a] = P.x[a];
            h[9 + a] = P.u[a];
            h[12 + a] = P.w[a];
        }
    }
    P.steps += 1;
}

// Box of cells around the sphere: cell (o + t) for t in [0, E), o from the
// current centre.  Returns false for cells outside a walled domain.
__device__ __forceinline__ bool box_cell(int t, const GridDesc& G, const BoxDesc& B, const ParticleState& P,
                                         int* ci, int* cj, int* ck) {
    const int e0 = B.E[0], e1 = B.E[1];
    const int tk = t / (e0 * e1);
    const int r = t - tk * e0 * e1;
    const int tj = r / e0;
    const int ti = r - tj * e0;
    const int n3[3] = {G.nx, G.ny, G.nz};
    const int tt[3] = {ti, tj, tk};
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int o = (B.E[a] >= n3[a]) ? 0 : (int)floor(P.x[a] - 0.5) - B.R;
        int v = o + tt[a];
        if (v < 0 || v >= n3[a]) {
            if (!G.periodic[a]) return false;
            v = v < 0 ? v + n3[a] : v - n3[a];   // |v| stays within one period: the box is narrower than the domain
        }
        c[a] = v;
    }
    *ci = c[0];
    *cj = c[1];
    *ck = c[2];
    return true;
}

}  // namespace lbmp
