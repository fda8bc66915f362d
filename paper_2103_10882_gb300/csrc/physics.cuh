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
// SCALED: g holds the deviations times 2^s (FP16 storage kept in its scaled
// form); the collision is linear in g except for the equilibrium's two
// quadratic terms, which then take one factor 2^-s (P.inv_scale).
// MRT_MODE: -1 decides TRT or MRT from P.db at run time, 0 is TRT only, 1
// MRT only (kernels that know which one runs carry no code of the other).
template <typename A, bool FORCED, bool SCALED = false, int MRT_MODE = -1, bool PAIRS = false>
__device__ __forceinline__ void trt_collide(A (&g)[19], const CollideParams<A>& P, int* status) {
    static_assert(!(FORCED && SCALED), "the scaled form is for the unforced collision");
    const A q2 = SCALED ? P.inv_scale : A(1);
    // PAIRS: the moments from the sums and differences of the opposite pairs (q, q + 1), q odd,
    // which the relaxation below uses again (c_{q+1} = -c_q: a pair adds its sum to the density and
    // its difference times c_q to the momentum).  Fewer instructions, for the issue-bound FP16 bulk
    // update; 18 more live values, which the register-capped level update pays for in spills.
    A ps[9], pd[9];
    A drho = g[0], jx = A(0), jy = A(0), jz = A(0);
    if (PAIRS) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            ps[k] = g[2 * k + 1] + g[2 * k + 2];
            pd[k] = g[2 * k + 1] - g[2 * k + 2];
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int q = 2 * k + 1;
            drho += ps[k];
            if (cx(q) == 1) jx += pd[k];
            if (cx(q) == -1) jx -= pd[k];
            if (cy(q) == 1) jy += pd[k];
            if (cy(q) == -1) jy -= pd[k];
            if (cz(q) == 1) jz += pd[k];
            if (cz(q) == -1) jz -= pd[k];
        }
    } else {
        drho = A(0);
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
    }
    A ux = jx, uy = jy, uz = jz;
    if (FORCED) {
        ux += A(0.5) * P.F[0];
        uy += A(0.5) * P.F[1];
        uz += A(0.5) * P.F[2];
    }
    const A uu = (ux * ux + uy * uy + uz * uz) * q2;
    if (!(uu * q2 <= A(0.09))) atomicOr(status, STATUS_UNSTABLE_FLUID);
    const A sp = P.sp, sm = P.sm;
    const bool mrt = MRT_MODE < 0 ? P.db != A(0) : MRT_MODE == 1;
    // MRT bulk correction: sums of (f - f_eq + source/2) over the rest,
    // face and edge populations (the even modes' inputs)
    A nR = A(0), nF = A(0), nE = A(0);
    {
        const A e0 = wgt<A>(0) * (drho - A(1.5) * uu);
        if (mrt) nR = g[0] - e0;
        A o = g[0] - sp * (g[0] - e0);
        if (FORCED) {
            const A uF = ux * P.F[0] + uy * P.F[1] + uz * P.F[2];
            o += (A(1) - A(0.5) * sp) * wgt<A>(0) * (A(-3) * uF);
            if (mrt) nR += A(0.5) * wgt<A>(0) * (A(-3) * uF);
        }
        g[0] = o;
    }
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        const A cu = A(cx(q)) * ux + A(cy(q)) * uy + A(cz(q)) * uz;
        const A w = wgt<A>(q);
        const A ep = w * (drho + A(4.5) * q2 * cu * cu - A(1.5) * uu);
        const A em = w * (A(3) * cu);
        const A gp = A(0.5) * (PAIRS ? ps[q >> 1] : g[q] + g[q + 1]);
        const A gm = A(0.5) * (PAIRS ? pd[q >> 1] : g[q] - g[q + 1]);
        const A dp = sp * (gp - ep);
        const A dm = sm * (gm - em);
        if (mrt) {
            if (q < 7) nF += A(2) * (gp - ep);
            else nE += A(2) * (gp - ep);
        }
        A a = g[q] - dp - dm;
        A b = g[q + 1] - dp + dm;
        if (FORCED) {
            const A cF = A(cx(q)) * P.F[0] + A(cy(q)) * P.F[1] + A(cz(q)) * P.F[2];
            const A uF = ux * P.F[0] + uy * P.F[1] + uz * P.F[2];
            const A Sp = (A(1) - A(0.5) * sp) * w * (A(9) * cu * cF - A(3) * uF);
            const A Sm = (A(1) - A(0.5) * sm) * w * (A(3) * cF);
            a += Sp + Sm;
            b += Sp - Sm;
            if (mrt) {   // half the symmetric source of the pair
                const A hs = w * (A(9) * cu * cF - A(3) * uF);
                if (q < 7) nF += hs;
                else nE += hs;
            }
        }
        g[q] = a;
        g[q + 1] = b;
    }
    if (mrt) {
        // MRT of Sec. 2.1 = TRT with the bulk mode e4 = |c|^2 - 1 and the
        // isotropic fourth-order mode e16 = 3|c|^4 - 6|c|^2 + 1 relaxed at s_b
        // instead of s+: subtract (s_b - s+) w_q sum_k e_k(q) c_k with
        // c_k = sum_p e_k(p) (f - f_eq + source/2)_p / sum_p w_p e_k(p)^2
        // (e4: rest -1, faces 0, edges 1, norm 2/3; e16: rest 1, faces -2,
        // edges 1, norm 2).
        const A c4 = A(1.5) * (nE - nR);
        const A c16 = A(0.5) * (nR - A(2) * nF + nE);
        g[0] -= P.db * wgt<A>(0) * (c16 - c4);
        const A df = P.db * wgt<A>(1) * (A(-2) * c16);
        const A de = P.db * wgt<A>(7) * (c4 + c16);
#pragma unroll
        for (int q = 1; q < 7; ++q) g[q] -= df;
#pragma unroll
        for (int q = 7; q < 19; ++q) g[q] -= de;
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
    const int q = lane < 19 ? lane : 0;   // c_q component (0 for idle lanes)
    return axis == 0 ? cx(q) : (axis == 1 ? cy(q) : cz(q));
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
    A v = gq - ep - em;   // f - f_eq of the lane (the odd part drops out of the even sums below)
    if (FORCED) {
        const A cF = A(c0) * P.F[0] + A(c1) * P.F[1] + A(c2) * P.F[2];
        const A uF = ux * P.F[0] + uy * P.F[1] + uz * P.F[2];
        out += (A(1) - A(0.5) * P.sp) * w * (A(9) * cu * cF - A(3) * uF) + (A(1) - A(0.5) * P.sm) * w * (A(3) * cF);
        v += A(0.5) * w * (A(9) * cu * cF - A(3) * uF);
    }
    if (P.db != A(0)) {   // MRT bulk correction, as in trt_collide (uniform across the warp)
        const A e4 = lane == 0 ? A(-1) : (lane <= 6 ? A(0) : (lane < 19 ? A(1) : A(0)));
        const A e16 = lane == 0 ? A(1) : (lane <= 6 ? A(-2) : (lane < 19 ? A(1) : A(0)));
        const A c4 = A(1.5) * warp_sum<A>(e4 * v);
        const A c16 = A(0.5) * warp_sum<A>(e16 * v);
        out -= P.db * w * (e4 * c4 + e16 * c16);
    }
    return lane < 19 ? out : A(0);
}

// Particle quantities the link kernels need, converted once per block
// (thread 0 fills a shared copy): Xi = floor(X) and Xh = 1/2 - (X - Xi), so
// the offset of a cell centre p + 1/2 from the centre X is (p - Xi) + Xh
// without cancellation in A; radius and velocities u(t + 1/2), omega(t + 1/2) in A.
template <typename A>
struct LinkFrame {
    int Xi[3];
    A Xh[3], r, u[3], w[3];
    __device__ __forceinline__ void init(const ParticleState& P) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double f = floor(P.x[a]);
            Xi[a] = (int)f;
            Xh[a] = A(0.5 - (P.x[a] - f));
            u[a] = A(P.u[a]);
            w[a] = A(P.w[a]);
        }
        r = A(P.r);
    }
    // d = p + 1/2 - X for cell p (minimum image on periodic axes) and the
    // matching unwrapped coordinate pu, with d = pu + 1/2 - X.
    __device__ __forceinline__ void offset(const int p[3], const int n[3], const int periodic[3], A d[3],
                                           int pu[3]) const {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int v = p[a];
            if (periodic[a]) {
                const A t = A(v - Xi[a]) + Xh[a];
                const A half = A(0.5) * A(n[a]);
                v += t > half ? -n[a] : (t < -half ? n[a] : 0);
            }
            pu[a] = v;
            d[a] = A(v - Xi[a]) + Xh[a];
        }
    }
};

// CLI link of Sec. 2.3 for the fluid cell at offset d from the sphere
// centre, incoming direction q (k = opp(q) points into the solid): returns
// the new deviation g_q and the link's momentum-exchange force and torque
// without their lattice-weight part.  On full populations f = w + g the
// link force is (c_k - v) f~_k + (c_k + v) f_q = 2 w_k c_k + fl with
// fl = (c_k - v) g~_k + (c_k + v) g_q; the 2 w_k c_k part (and its torque
// d x 2 w_k c_k) is summed exactly by LinkSums.  Geometry and fl are
// evaluated in the arithmetic type A of the populations (FP64 on the FP64
// path); use_delta = false takes the wall half-way (delta = 1/2).
// Wall distance delta along c_k (k = opp(q)) from the cell at offset d and
// the CLI coefficients kappa0 = (1 - 2 delta) / (1 + 2 delta) and
// alpha = 4 / (1 + 2 delta) of Sec. 2.3; use_delta = false takes delta = 1/2.
template <typename A>
__device__ __forceinline__ void cli_coeffs(int q, const A d[3], bool use_delta, A r, A* delta_out, A* kappa0,
                                           A* alpha) {
    const int k = opp(q);
    A delta = A(0.5);
    if (use_delta) {   // smallest root in (0,1] of |d + s c_k|^2 = r^2 (|c_k|^2 is 1 or 2)
        const A dc = d[0] * A(cx(k)) + d[1] * A(cy(k)) + d[2] * A(cz(k));
        const A e = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - r * r;
        const bool face = k <= 6;
        A disc = dc * dc - (face ? e : A(2) * e);
        disc = disc < A(0) ? A(0) : disc;
        const A s = (-dc - sqrt(disc)) * (face ? A(1) : A(0.5));
        delta = s < A(0) ? A(0) : (s > A(1) ? A(1) : s);
    }
    const A inv = A(1) / (A(1) + A(2) * delta);
    *delta_out = delta;
    *kappa0 = (A(1) - A(2) * delta) * inv;
    *alpha = A(4) * inv;
}

template <typename A>
__device__ __forceinline__ A cli_link(int q, const A d[3], bool use_delta, A gt_k, A gt_q, A gt_far,
                                      const LinkFrame<A>& Fr, A fl[3], A tl[3]) {
    const int k = opp(q);
    const A c[3] = {A(cx(k)), A(cy(k)), A(cz(k))};
    A delta, kappa0, alpha;
    cli_coeffs<A>(q, d, use_delta, Fr.r, &delta, &kappa0, &alpha);
    const A arm[3] = {d[0] + delta * c[0], d[1] + delta * c[1], d[2] + delta * c[2]};
    const A vb[3] = {Fr.u[0] + (Fr.w[1] * arm[2] - Fr.w[2] * arm[1]), Fr.u[1] + (Fr.w[2] * arm[0] - Fr.w[0] * arm[2]),
                     Fr.u[2] + (Fr.w[0] * arm[1] - Fr.w[1] * arm[0])};
    const A vc = vb[0] * c[0] + vb[1] * c[1] + vb[2] * c[2];
    const A wk3 = k <= 6 ? A(1) / A(6) : A(1) / A(12);   // 3 w_k
    const A gnew = gt_k + kappa0 * gt_far - kappa0 * gt_q - alpha * wk3 * vc;
#pragma unroll
    for (int a = 0; a < 3; ++a) fl[a] = (c[a] - vb[a]) * gt_k + (c[a] + vb[a]) * gnew;
    tl[0] = arm[1] * fl[2] - arm[2] * fl[1];
    tl[1] = arm[2] * fl[0] - arm[0] * fl[2];
    tl[2] = arm[0] * fl[1] - arm[1] * fl[0];
    return gnew;
}

// Per-lane sums of the link forces and torques of one particle.  fl and tl
// of every link are added in the arithmetic type A; in FP32 each running
// sum carries its rounding error (Knuth's TwoSum, exact for every
// addition), so a lane's sum is exact to far below FP32 resolution without
// the slow FP64 pipe.  The block sum is formed in FP64.  The lattice-weight part
// 2 w_k c_k is summed in integers: 36 * 2 w_k is 4 on faces and 2 on edges,
// and its torque (pu + 1/2 - X) x 2 w_k c_k is carried as
// (2 pu + 1) x (36 * 2 w_k c_k) over 72 minus X x (the force part), so it
// cancels exactly wherever the links close around the body.
template <typename A>
struct LinkSums {
    A F[3] = {A(0), A(0), A(0)}, T[3] = {A(0), A(0), A(0)};
    A eF[3] = {A(0), A(0), A(0)}, eT[3] = {A(0), A(0), A(0)};   // FP32: rounding errors of F and T
    int iF[3] = {0, 0, 0};
    long long iT[3] = {0, 0, 0};

    __device__ static __forceinline__ void sum2(A& s, A& e, A x) {
        if constexpr (sizeof(A) == 8) {
            s += x;
        } else {
            const A t = s + x, xv = t - s;
            e += (s - (t - xv)) + (x - xv);
            s = t;
        }
    }
    __device__ __forceinline__ void add(int k, const int pu[3], const A fl[3], const A tl[3]) {
        const int m = k <= 6 ? 4 : 2;
        const int mc[3] = {m * cx(k), m * cy(k), m * cz(k)};
        const long long p2[3] = {2LL * pu[0] + 1, 2LL * pu[1] + 1, 2LL * pu[2] + 1};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            sum2(F[a], eF[a], fl[a]);
            sum2(T[a], eT[a], tl[a]);
            iF[a] += mc[a];
        }
        iT[0] += p2[1] * mc[2] - p2[2] * mc[1];
        iT[1] += p2[2] * mc[0] - p2[0] * mc[2];
        iT[2] += p2[0] * mc[1] - p2[1] * mc[0];
    }
};

__device__ __forceinline__ double pick3(const double v[3], int i) { return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]); }

// Double-float addition (h, l) += (bh, bl): Knuth's TwoSum of the leading
// parts, the trailing parts added to its error, renormalised (Fast2Sum).
// About 44 significant bits, in FP32 arithmetic.
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
    const float s = h + bh, v = s - h;
    const float e = ((h - (s - v)) + (bh - v)) + (l + bl);
    h = s + e;
    l = e - (h - s);
}

// Deterministic block sum of the threads' link sums into out[0..5]: force,
// and torque about X.  Every thread of the block must call it.  FP64
// additions, and conversions to FP64, are slow and narrow on this GPU, so
// in FP32 the lanes' sums (each with its TwoSum error) are reduced as
// double-float pairs, a butterfly within each warp and, after one barrier,
// one across the warps' results by warps 0..5 (one component each); only
// lane 0 of those warps converts to FP64.  In FP64 the six components are
// staged in shared memory and warp c adds column l of the warp rows
// pairwise in lane l, then across the lanes.  The integer parts are summed
// exactly by shuffles, and the constant divisions are multiplications by
// the reciprocals.  A last-block hand-off after this call is ordered by its
// barrier and release (the writers need no fence of their own).
template <int NT, typename A>
__device__ __forceinline__ void block_link_sums(const LinkSums<A>& acc, const double X[3], double* __restrict__ out) {
    static_assert(NT % 32 == 0 && NT >= 192 && NT <= 1024, "six warps take the six components");
    constexpr int NW = NT / 32;
    constexpr int SPAN = NW <= 8 ? 8 : (NW <= 16 ? 16 : 32);   // lanes of the cross-warp butterfly
    __shared__ long long si[6][NW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    long long iv[6] = {acc.iF[0], acc.iF[1], acc.iF[2], acc.iT[0], acc.iT[1], acc.iT[2]};
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) iv[c] += __shfl_down_sync(0xffffffffu, iv[c], off);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) si[c][wid] = iv[c];
    double t;
    int c;
    if constexpr (sizeof(A) == 4) {
        __shared__ float sh[6][NW], sl[6][NW];
        float h[6], l[6];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            h[a] = acc.F[a] + acc.eF[a];
            l[a] = acc.eF[a] - (h[a] - acc.F[a]);
            h[3 + a] = acc.T[a] + acc.eT[a];
            l[3 + a] = acc.eT[a] - (h[3 + a] - acc.T[a]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float oh = __shfl_xor_sync(0xffffffffu, h[k], off), ol = __shfl_xor_sync(0xffffffffu, l[k], off);
                df_add(h[k], l[k], oh, ol);
            }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                sh[k][wid] = h[k];
                sl[k][wid] = l[k];
            }
        __syncthreads();
        if (wid >= 6) return;
        c = wid;
        float th = lane < NW ? sh[c][lane] : 0.0f, tl = lane < NW ? sl[c][lane] : 0.0f;
#pragma unroll
        for (int off = SPAN / 2; off > 0; off >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, th, off), ol = __shfl_xor_sync(0xffffffffu, tl, off);
            df_add(th, tl, oh, ol);
        }
        if (lane != 0) return;
        t = (double)th + (double)tl;
    } else {
        __shared__ double sd[6][NT];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            sd[a][tid] = acc.F[a];
            sd[3 + a][tid] = acc.T[a];
        }
        __syncthreads();
        if (wid >= 6) return;
        c = wid;
        double v[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) v[w] = sd[c][lane + 32 * w];
#pragma unroll
        for (int st = 1; st < NW; st <<= 1)
#pragma unroll
            for (int w = 0; w + st < NW; w += 2 * st) v[w] += v[w + st];
        t = v[0];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane != 0) return;
    }
    long long iF[3] = {0, 0, 0}, iT = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        iF[0] += si[0][w];
        iF[1] += si[1][w];
        iF[2] += si[2][w];
        iT += si[c][w];
    }
    const double r36 = 1.0 / 36.0, r72 = 1.0 / 72.0;
    const double fr[3] = {(double)iF[0] * r36, (double)iF[1] * r36, (double)iF[2] * r36};
    if (c < 3) {
        out[c] = t + pick3(fr, c);
    } else {
        const int a1 = c == 3 ? 1 : (c == 4 ? 2 : 0), a2 = c == 3 ? 2 : (c == 4 ? 0 : 1);
        out[c] = t + ((double)iT * r72 - (X[a1] * pick3(fr, a2) - X[a2] * pick3(fr, a1)));
    }
}

__device__ __forceinline__ int src_coord(int x, int c, int n, int periodic) {
    int s = x - c;
    if (s < 0) return periodic ? s + n : -1;
    if (s >= n) return periodic ? s - n : -1;
    return s;
}

// Cell centre p + 1/2 inside the closed ball |p + 1/2 - X| <= r: the flag
// definition, evaluated in FP64 with explicit round-to-nearest products and
// sums (no contraction), minimum image on periodic axes.
__device__ __forceinline__ bool inside_ball_exact(const int p[3], const int n[3], const int periodic[3],
                                                  const ParticleState& P) {
    const double dx = wrap_diff(__dsub_rn((double)p[0] + 0.5, P.x[0]), n[0], periodic[0]);
    const double dy = wrap_diff(__dsub_rn((double)p[1] + 0.5, P.x[1]), n[1], periodic[1]);
    const double dz = wrap_diff(__dsub_rn((double)p[2] + 0.5, P.x[2]), n[2], periodic[2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 <= __dmul_rn(P.r, P.r);
}

__device__ __forceinline__ bool inside_ball(int i, int j, int k, const GridDesc& G, const ParticleState& P) {
    const int p[3] = {i, j, k}, n[3] = {G.nx, G.ny, G.nz};
    return inside_ball_exact(p, n, G.periodic, P);
}

// Per-block constants of the kernels that walk the box of cells around the
// sphere (cell o + t for t in [0, E) per axis, o from the current centre),
// filled once by thread 0 (all of their FP64 set-up work): the box
// origin and an FP32 pre-test of the ball predicate.  The FP32 squared
// distance (p - Xi + Xh)^2 differs from the FP64 one by less than
// 1e-6 (|d|^2 + 1); cells whose estimate lies below lo = r^2 - 1e-5 (r^2 + 1)
// are inside, above hi = r^2 + 1e-5 (r^2 + 1) outside, and only the thin shell
// in between evaluates inside_ball_exact, so every flag equals the FP64
// definition.
struct BoxFrame {
    int o[3];      // first box cell per axis (0 where the box spans a periodic axis)
    int Xi[3];     // floor(X)
    float Xh[3];   // 1/2 - (X - Xi)
    float lo, hi;
};

__device__ __forceinline__ void box_frame_init(BoxFrame& F, const int n[3], const int periodic[3], const BoxDesc& B,
                                               const ParticleState& P) {
    bool wide = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // a centre that is not finite or absurdly far (only after an unstable step, which the
        // status word reports) is replaced so that the integer box arithmetic stays in range
        const double x = fabs(P.x[a]) < 1e9 ? P.x[a] : 0.0;
        F.o[a] = (B.E[a] >= n[a]) ? 0 : (int)floor(x - 0.5) - B.R;
        const double f = floor(x);
        F.Xi[a] = (int)f;
        F.Xh[a] = (float)(0.5 - (x - f));
        // a sphere reaching within two cells of half a period: the FP32 tests skip minimum images
        wide |= periodic[a] && (P.r > 0.4 * n[a] || P.r + 2.0 >= 0.5 * n[a]);
    }
    const double rr = P.r * P.r, m = 1e-5 * (rr + 1.0);
    F.lo = wide ? -1.0f : (float)(rr - m);   // a sphere this wide takes the FP64 path everywhere
    F.hi = wide ? 3.0e38f : (float)(rr + m);
}

// Both frames of the sphere's current state (the link frame in FP32 and in
// FP64, and the box frame), formed once per step by the particle update, or
// after the host changed the record, and read by the box kernels of the
// refined step instead of each of their blocks forming them from the FP64
// record (FP64 is slow on this part, and every block waited for it).
__device__ __forceinline__ double particle_mass(const ParticleState& P);
__device__ __forceinline__ double particle_inertia(const ParticleState& P);

struct PFrames {
    LinkFrame<float> lf;
    LinkFrame<double> ld;
    BoxFrame bf;
    double inv[2];   // 1/m and 1/I (particle_mass, particle_inertia): fixed between changes by the host
};

template <typename A>
__device__ __forceinline__ const LinkFrame<A>& pframe_link(const PFrames& F) {
    if constexpr (sizeof(A) == 8) return F.ld;
    else return F.lf;
}

// Forms F from the record P: the three frames by lane 0 of warps 0, 1 and 2
// of the calling block (each is one FP64 sequence), the inverses by lanes 0
// and 1 of warp 3; every thread of a block of at least 128 calls it.
__device__ __forceinline__ void pframes_form(PFrames* __restrict__ F, const ParticleState& P, const int n[3],
                                             const int periodic[3], const BoxDesc& B) {
    if (threadIdx.x == 0) F->lf.init(P);
    else if (threadIdx.x == 32) F->ld.init(P);
    else if (threadIdx.x == 64) box_frame_init(F->bf, n, periodic, B, P);
    else if (threadIdx.x == 96) F->inv[0] = 1.0 / particle_mass(P);
    else if (threadIdx.x == 97) F->inv[1] = 1.0 / particle_inertia(P);
}

// The parts of F that follow the sphere along axis a (a = 0, 1, 2 by lanes
// 0, 1, 2 of one warp) after the particle update: the same values as
// pframes_form, from a shorter FP64 sequence (floor by one conversion, the
// box origin from the fraction); the radius and the FP32 pre-test bounds do
// not change during a run and keep the values pframes_form gave them.
__device__ __forceinline__ void pframes_axis(PFrames* __restrict__ F, const ParticleState& P, const int n[3],
                                             const BoxDesc& B, int a) {
    const double xr = P.x[a];
    const double x = fabs(xr) < 1e9 ? xr : 0.0;   // as box_frame_init: keep the box arithmetic in range
    const int xi = __double2int_rd(xr), bi = __double2int_rd(x);
    const double frac = xr - (double)xi, bfrac = x - (double)bi;
    F->lf.Xi[a] = xi;
    F->ld.Xi[a] = xi;
    F->ld.Xh[a] = 0.5 - frac;
    F->lf.Xh[a] = (float)(0.5 - frac);
    F->lf.u[a] = (float)P.u[a];
    F->lf.w[a] = (float)P.w[a];
    F->ld.u[a] = P.u[a];
    F->ld.w[a] = P.w[a];
    F->bf.Xi[a] = bi;
    F->bf.Xh[a] = (float)(0.5 - bfrac);
    // floor(x - 1/2): x - 1/2 and x - floor(x) are exact
    F->bf.o[a] = (B.E[a] >= n[a]) ? 0 : (bfrac < 0.5 ? bi - 1 : bi) - B.R;
}

// Box cell t (x fastest) -> cell p; false where the box leaves a wall-bounded axis.
__device__ __forceinline__ bool box_cell(int t, const int n[3], const int periodic[3], const BoxDesc& B,
                                         const BoxFrame& F, int p[3]) {
    const int e0 = B.E[0], e1 = B.E[1];
    const int tk = t / (e0 * e1);
    const int r = t - tk * e0 * e1;
    const int tj = r / e0;
    const int tt[3] = {r - tj * e0, tj, tk};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = F.o[a] + tt[a];
        if (v < 0 || v >= n[a]) {
            if (!periodic[a]) return false;
            v = v < 0 ? v + n[a] : v - n[a];   // the box is never wider than the domain
            if (v < 0 || v >= n[a]) return false;   // a centre outside the domain: touch nothing
        }
        p[a] = v;
    }
    return true;
}

__device__ __forceinline__ bool ball_flag(const int p[3], const int n[3], const int periodic[3], const BoxFrame& F,
                                          const ParticleState& P) {
    float e = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = p[a] - F.Xi[a];
        if (periodic[a]) {
            const float t = (float)v + F.Xh[a], half = 0.5f * (float)n[a];
            v += t > half ? -n[a] : (t < -half ? n[a] : 0);
        }
        const float t = (float)v + F.Xh[a];
        e = fmaf(t, t, e);
    }
    if (e < F.lo) return true;
    if (e > F.hi) return false;
    return inside_ball_exact(p, n, periodic, P);
}

// Solid flag of cell p and whether any of its 18 D3Q19 neighbours is solid,
// both as defined by the exact ball predicate.  The neighbours' FP32
// squared distances follow from the cell's own FP32 offset t as
// (t + c_q)^2, one more rounding per component than ball_flag, well inside
// the same margin; undecided cells take the FP64 expression at the wrapped
// neighbour position.  A box wider than half a period takes the FP64 path
// everywhere (lo < 0, see box_frame_init), so no minimum image is needed for
// the neighbours here.
__device__ __forceinline__ bool ball_flag_and_neighbours(const int p[3], const int n[3], const int periodic[3],
                                                         const BoxFrame& F, const ParticleState& P, bool* any_nb) {
    float t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = p[a] - F.Xi[a];
        if (periodic[a]) {
            const float u = (float)v + F.Xh[a], half = 0.5f * (float)n[a];
            v += u > half ? -n[a] : (u < -half ? n[a] : 0);
        }
        t[a] = (float)v + F.Xh[a];
    }
    const float e0 = fmaf(t[2], t[2], fmaf(t[1], t[1], t[0] * t[0]));
    const bool own = e0 < F.lo ? true : (e0 > F.hi ? false : inside_ball_exact(p, n, periodic, P));
    bool any = false;
#pragma unroll
    for (int q = 1; q < 19; ++q) {
        const float a0 = t[0] + (float)cx(q), a1 = t[1] + (float)cy(q), a2 = t[2] + (float)cz(q);
        const float e = fmaf(a2, a2, fmaf(a1, a1, a0 * a0));
        if (e < F.lo) any = true;
        else if (e <= F.hi && !any) {
            int v[3] = {p[0] + cx(q), p[1] + cy(q), p[2] + cz(q)};
            bool ok = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (v[a] < 0 || v[a] >= n[a]) {
                    if (!periodic[a]) ok = false;
                    v[a] = v[a] < 0 ? v[a] + n[a] : v[a] - n[a];
                }
            }
            if (ok && inside_ball_exact(v, n, periodic, P)) any = true;
        }
    }
    *any_nb = any;
    return own;
}

// m = (rho_p + C_v) V and I = 2/5 (rho_p + C_vw) V r^2 (Sec. 2.2: virtual mass and moment of inertia).
__device__ __forceinline__ double particle_mass(const ParticleState& P) { return (P.rho_p + P.cv) * P.V; }
__device__ __forceinline__ double particle_inertia(const ParticleState& P) {
    return 0.4 * (P.rho_p + P.cvw) * P.V * P.r * P.r;
}

// One axis a of Algorithm 1's particle update: average of the hydrodynamic
// force and torque over two steps, gravity/buoyancy, the virtual force and
// torque from the previous accelerations, and the kick-drift-kick update
// with the virtually increased mass and moment of inertia, whose inverses
// the caller passes (particle_mass, particle_inertia).  The axes are
// independent; P.steps is advanced once afterwards.
__device__ __forceinline__ void particle_advance_axis(ParticleState& P, int a, double Fh, double Th, double inv_m,
                                                      double inv_I, const GridDesc& G, double* __restrict__ history,
                                                      int hist_cap, int* __restrict__ status) {
    const double V = P.V, r = P.r;
    const bool avg = P.force_average && P.steps > 0;
    const double Fbar = avg ? 0.5 * (Fh + P.Fh_old[a]) : Fh;
    const double Tbar = avg ? 0.5 * (Th + P.Th_old[a]) : Th;
    P.Fh[a] = Fh;
    P.Th[a] = Th;
    P.Fh_old[a] = Fh;
    P.Th_old[a] = Th;
    const double Fg = (P.rho_p - 1.0) * P.g[a] * V;
    const double Fv = P.cv * V * P.a[a];
    const double Tv = 0.4 * P.cvw * V * r * r * P.b[a];
    const double Fp = Fbar + Fg + Fv;
    const double Tp = Tbar + Tv;
    P.Fp[a] = Fp;
    const double xold = P.x[a];
    const double acc = Fp * inv_m, bet = Tp * inv_I;
    // A held group (translation; rotation) keeps its velocity and records zero acceleration, so the
    // virtual force or torque after it is zero; a group released in this step starts afresh, with
    // no half kick completing a previous step.
    const bool tfree = P.fixed == 0, rfree = P.fixed != 1;
    const bool tprev = P.steps > 0 && P.prev_fixed == 0, rprev = P.steps > 0 && P.prev_fixed != 1;
    if (tfree) {
        if (tprev) P.u[a] += 0.5 * acc;   // second half kick of the previous step completes u(t)
        P.a[a] = acc;
        P.u[a] += 0.5 * acc;   // first half kick, then drift with u(t + 1/2)
        P.x[a] += P.u[a];
    } else {
        P.a[a] = 0.0;
    }
    if (rfree) {
        if (rprev) P.w[a] += 0.5 * bet;
        P.b[a] = bet;
        P.w[a] += 0.5 * bet;
    } else {
        P.b[a] = 0.0;
    }
    if (!(fabs(P.x[a] - xold) <= 0.5) || !(fabs(P.u[a]) < 0.5) || !(fabs(P.w[a]) < 1e30)) {
        // a jump or a non-finite state: flag it, and keep the sphere where it was and at rest, so that
        // the box kernels that follow until the host reads the status stay inside the domain
        atomicOr(status, STATUS_PARTICLE_JUMP);
        P.x[a] = xold;
        P.u[a] = P.w[a] = P.a[a] = P.b[a] = 0.0;
    }
    const int n = a == 0 ? G.nx : (a == 1 ? G.ny : G.nz);
    if (G.periodic[a]) {   // keep the centre inside the periodic box
        const double L = (double)n;
        if (P.x[a] >= L) P.x[a] -= L;
        else if (P.x[a] < 0.0) P.x[a] += L;
    }
    if (hist_cap > 0) {
        double* h = history + (size_t)(P.steps % hist_cap) * 15;
        h[a] = Fh;
        h[3 + a] = Th;
        h[6 + a] = P.x[a];
        h[9 + a] = P.u[a];
        h[12 + a] = P.w[a];
    }
}

// Particle update by one block of NT >= 256 threads once the nblocks force
// partials are complete: warps 0..5 sum one component each in a fixed
// order (lane l takes partials l, l + 32, ... in two alternating sums, then
// a butterfly runs across the lanes), warp 6 forms 1/m and 1/I, warp 7
// stages the record in shared memory; threads 0..2 then advance the three
// axes and the block writes the record back.  The partials may come from
// other blocks of the same launch: they are read through L2.  Every thread
// of the block must call it.
template <int NT>
__device__ __forceinline__ void particle_block_update(ParticleState* __restrict__ ps, const double* partials,
                                                      int nblocks, const GridDesc& G, double* __restrict__ history,
                                                      int hist_cap, int* __restrict__ status,
                                                      const double* __restrict__ inv = nullptr) {
    static_assert(NT % 32 == 0 && NT >= 256, "eight warps share the work");
    constexpr int words = (int)(sizeof(ParticleState) / sizeof(int));
    __shared__ double sFT[6], sinv[2];
    __shared__ ParticleState sP;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < 6) {
        // lane l sums partials l, l + 64, ... into s0 and l + 32, l + 96, ... into s1, in that
        // order; eight loads at a time are issued before their sums
        double s0 = 0.0, s1 = 0.0;
        for (int base = 0; base < nblocks; base += 256) {
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int b = base + lane + 32 * k;
                v[k] = b < nblocks ? __ldcg(partials + (size_t)b * 6 + wid) : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                if (base + lane + 32 * k < nblocks) s0 += v[k];
                if (base + lane + 32 * (k + 1) < nblocks) s1 += v[k + 1];
            }
        }
        double t = s0 + s1;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) sFT[wid] = t;
    } else if (wid == 6) {
        if (lane < 2) sinv[lane] = inv ? inv[lane] : 1.0 / (lane == 0 ? particle_mass(*ps) : particle_inertia(*ps));
    } else if (wid == 7) {
        const int* srcw = reinterpret_cast<const int*>(ps);
        int* dstw = reinterpret_cast<int*>(&sP);
#pragma unroll 4
        for (int i = lane; i < words; i += 32) dstw[i] = __ldcg(srcw + i);
    }
    __syncthreads();
    if (threadIdx.x < 3)   // the three axes in parallel
        particle_advance_axis(sP, threadIdx.x, sFT[threadIdx.x], sFT[3 + threadIdx.x], sinv[0], sinv[1], G, history,
                              hist_cap, status);
    __syncthreads();
    if (threadIdx.x == 0) {
        sP.steps += 1;
        sP.prev_fixed = sP.fixed;
    }
    __syncthreads();
    {
        const int* srcw = reinterpret_cast<const int*>(&sP);
        int* dstw = reinterpret_cast<int*>(ps);
        for (int i = threadIdx.x; i < words; i += NT) dstw[i] = srcw[i];
    }
}


// Grad refill of an uncovered cell (Sec. 2.3: the paper uses Dorschner et
// al.'s approach, read as Grad's approximation from the local strain rate).
// Strain rate S (xx, yy, zz, xy, yz, xz) from the six face neighbours'
// velocities: central differences where both are fluid, one-sided against
// the wall velocity uw where one is, zero where neither is.  nb(a, sgn, u)
// returns whether the face neighbour x + sgn e_a is fluid (before and after
// the move) and, if so, its velocity in u.
template <typename A, typename NB>
__device__ __forceinline__ void refill_strain(NB&& nb, const A uw[3], A S[6]) {
    A G[3][3];   // G[a][b] = d u_b / d x_a
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        A up[3], um[3];
        const bool okp = nb(a, 1, up), okm = nb(a, -1, um);
#pragma unroll
        for (int b = 0; b < 3; ++b)
            G[a][b] = (okp && okm) ? A(0.5) * (up[b] - um[b]) : (okp ? up[b] - uw[b] : (okm ? uw[b] - um[b] : A(0)));
    }
    S[0] = G[0][0];
    S[1] = G[1][1];
    S[2] = G[2][2];
    S[3] = A(0.5) * (G[0][1] + G[1][0]);
    S[4] = A(0.5) * (G[1][2] + G[2][1]);
    S[5] = A(0.5) * (G[0][2] + G[2][0]);
}

// Grad's non-equilibrium part of population q of a refilled post-collision
// state: gcoef w_q Q_q:S with Q_q = c_q c_q - I/3 and gcoef = -3 (1 - s+)/s+
// (the first-order Chapman-Enskog stress after one collision).
template <typename A>
__device__ __forceinline__ A grad_term(int q, const A S[6], A gcoef) {
    const A x = A(cx(q)), y = A(cy(q)), z = A(cz(q));
    const A qs = x * x * S[0] + y * y * S[1] + z * z * S[2] + A(2) * (x * y * S[3] + y * z * S[4] + x * z * S[5]) -
                 (S[0] + S[1] + S[2]) / A(3);
    return gcoef * wgt<A>(q) * qs;
}

// Last-block-done hand-off: each of nblocks blocks calls it after writing
// its partials; the block that finishes last (a device counter, reset by
// that block) gets true.  No block waits for another.  The block barrier
// followed by thread 0's acquire-release atomic at GPU scope publishes the
// partials of all the block's threads and, in the last block, makes the
// other blocks' partials visible (read them through L2).
__device__ __forceinline__ bool last_block_done(int* counter, int nblocks) {
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        int old;
        asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(counter) : "memory");
        last = old == nblocks - 1;
        if (last) *counter = 0;
    }
    __syncthreads();
    return last != 0;
}

// Box cells of [t0, t0 + chunk) whose mask byte is set, in box order, into
// the shared list sl (offsets from t0); returns their number.  blockDim.x
// is a multiple of 32; chunk may be smaller or larger.  Every thread of the
// block must call it.
__device__ __forceinline__ int block_compact_mask(const uint8_t* __restrict__ mask, long long t0, long long cells,
                                                  int chunk, int* sl) {
    __shared__ int wcount[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    int total = 0;
    for (int off = 0; off < chunk; off += (int)blockDim.x) {
        const long long t = t0 + off + threadIdx.x;
        const bool m = off + (int)threadIdx.x < chunk && t < cells && mask[t] != 0;
        const unsigned bits = __ballot_sync(0xffffffffu, m);
        if (lane == 0) wcount[wid] = __popc(bits);
        __syncthreads();
        int base = total, add = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < wid) base += wcount[w];
            add += wcount[w];
        }
        if (m) sl[base + __popc(bits & ((1u << lane) - 1u))] = off + threadIdx.x;
        total += add;
        __syncthreads();
    }
    return total;
}

}  // namespace lbmp
