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
