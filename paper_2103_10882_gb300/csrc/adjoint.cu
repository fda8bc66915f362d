// Reverse-mode derivative of the mean drag on a fixed sphere.
//
// Objective: J = (1/N) sum_{n=1..N} F_a^n, the mean over N steps of one
// component of the momentum-exchange force (Sec. 2.3) on a sphere held at
// rest in a periodic box, with respect to the relaxation time tau (through
// s+ = 1/tau and s- of the magic parameter, Sec. 2.1), the fluid body force
// F and the initial velocity field u0 (the fluid starts at the equilibrium
// of u0).
//
// With h^n = S(g^{n-1}) the streamed (pre-collision) field, g^n = C(h^n) the
// post-collision field and F^n = sum over links (x, q) of
// c_k (2 w_k + g^{n-1}_k(x) + h^n_q(x)), k = opp(q), the adjoint fields
// nu^n = dJ/dh^n and lambda^n = dJ/dg^n obey
//     lambda^n = S^T nu^{n+1} + (1/N) sum_links c_k,a e_(x,k)      (n < N)
//     nu^n     = (dC/dh (h^n))^T lambda^n + (1/N) sum_links c_k,a e_(x,q)
// with lambda^N = 0, and
//     dJ/dtau = sum_n lambda^n . dC/dtau (h^n),  dJ/dF = sum_n lambda^n . dC/dF (h^n),
//     dJ/du0  = (dE/du0)^T lambda^0.
// S^T is streaming run backwards: a pull along -c_q, with the CLI terms of
// every link moved to the cells they read.  One kernel per reverse step
// forms lambda and nu cell by cell: it gathers nu^{n+1} from x + c_q and
// recomputes h^n from the stored g^{n-1}, so only the post-collision
// fields are kept: every interval-th one from the forward pass, the rest
// recomputed segment by segment (checkpoint and recompute).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "adjoint.h"
#include "internal.h"
#include "physics.cuh"

namespace lbmp {
namespace {

constexpr int AT = 256;   // threads per block of the cell kernels
constexpr int ADJ_MIN_CTAS = 4;   // resident reverse-step CTAs per SM asked of the compiler (FP32): 64 registers

enum : uint8_t { KIND_PLAIN = 0, KIND_SOLID = 1, KIND_NEAR = 2 };

template <typename A>
struct AdjParams {
    A sp, sm, F[3];
    A seed;      // 1/N
    int axis;    // force component of the objective
};

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ long long cell_at(const GridDesc& G, int i, int j, int k) {
    return (long long)wrapc(i, G.nx) + (long long)G.nx * ((long long)wrapc(j, G.ny) + (long long)G.ny * wrapc(k, G.nz));
}

// Transpose of the TRT collision with the Guo-type source (the derivative
// of trt_collide at h, applied to lambda), and the parameter parts
// part = (lambda . dC/ds+, lambda . dC/ds-, lambda . dC/dF).  The source is
// always differentiated, also where F = 0.
//   C_q(h) = h_q - s+ (h+_q - e+_q) - s- (h-_q - e-_q) + (1 - s+/2) S+_q + (1 - s-/2) S-_q
//   (dC/dh)^T lambda = lambda - s+ lambda+ - s- lambda- + a + b.c_p with
//   a = s+ L0, b = s+ (9 L2 u - 3 L0 u) + 3 s- L1 + (1 - s+/2)(9 L2 F - 3 L0 F),
//   L0 = sum w lambda, L1 = sum w lambda c, L2 = sum w lambda c c^T.
template <typename A>
__device__ __forceinline__ void trt_adjoint(const A (&h)[19], A (&lam)[19], const AdjParams<A>& P, A part[5]) {
    A drho = A(0), u[3] = {A(0), A(0), A(0)};
    A L0 = A(0), L1[3] = {A(0), A(0), A(0)}, L2[6] = {A(0), A(0), A(0), A(0), A(0), A(0)};   // xx yy zz xy xz yz
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        drho += h[q];
        if (cx(q) != 0) u[0] += A(cx(q)) * h[q];
        if (cy(q) != 0) u[1] += A(cy(q)) * h[q];
        if (cz(q) != 0) u[2] += A(cz(q)) * h[q];
        const A wl = wgt<A>(q) * lam[q];
        L0 += wl;
        if (cx(q) != 0) {
            L1[0] += A(cx(q)) * wl;
            L2[0] += wl;
        }
        if (cy(q) != 0) {
            L1[1] += A(cy(q)) * wl;
            L2[1] += wl;
        }
        if (cz(q) != 0) {
            L1[2] += A(cz(q)) * wl;
            L2[2] += wl;
        }
        if (cx(q) * cy(q) != 0) L2[3] += A(cx(q) * cy(q)) * wl;
        if (cx(q) * cz(q) != 0) L2[4] += A(cx(q) * cz(q)) * wl;
        if (cy(q) * cz(q) != 0) L2[5] += A(cy(q) * cz(q)) * wl;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a] += A(0.5) * P.F[a];
    const A uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const A uF = u[0] * P.F[0] + u[1] * P.F[1] + u[2] * P.F[2];
    const A sp = P.sp, sm = P.sm;
    // parameter parts: dC_q/ds+ = -(h+_q - e+_q) - S+_q / 2, dC_q/ds- = -(h-_q - e-_q) - S-_q / 2
    A tsp, tsm = A(0);
    {
        const A e0 = wgt<A>(0) * (drho - A(1.5) * uu);
        const A S0 = wgt<A>(0) * (A(-3) * uF);
        tsp = lam[0] * (-(h[0] - e0) - A(0.5) * S0);
    }
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        const A cu = A(cx(q)) * u[0] + A(cy(q)) * u[1] + A(cz(q)) * u[2];
        const A cF = A(cx(q)) * P.F[0] + A(cy(q)) * P.F[1] + A(cz(q)) * P.F[2];
        const A w = wgt<A>(q);
        const A ep = w * (drho + A(4.5) * cu * cu - A(1.5) * uu), em = w * (A(3) * cu);
        const A Sp = w * (A(9) * cu * cF - A(3) * uF), Sm = w * (A(3) * cF);
        const A hp = A(0.5) * (h[q] + h[q + 1]), hm = A(0.5) * (h[q] - h[q + 1]);
        tsp += (lam[q] + lam[q + 1]) * (-(hp - ep) - A(0.5) * Sp);
        tsm += (lam[q] - lam[q + 1]) * (-(hm - em) - A(0.5) * Sm);
    }
    const A L2u[3] = {L2[0] * u[0] + L2[3] * u[1] + L2[4] * u[2], L2[3] * u[0] + L2[1] * u[1] + L2[5] * u[2],
                      L2[4] * u[0] + L2[5] * u[1] + L2[2] * u[2]};
    const A L2F[3] = {L2[0] * P.F[0] + L2[3] * P.F[1] + L2[4] * P.F[2],
                      L2[3] * P.F[0] + L2[1] * P.F[1] + L2[5] * P.F[2],
                      L2[4] * P.F[0] + L2[5] * P.F[1] + L2[2] * P.F[2]};
    const A a0 = sp * L0;
    A b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const A du = A(9) * L2u[a] - A(3) * L0 * u[a];
        b[a] = sp * du + A(3) * sm * L1[a] + (A(1) - A(0.5) * sp) * (A(9) * L2F[a] - A(3) * L0 * P.F[a]);
        part[2 + a] = A(0.5) * b[a] + (A(1) - A(0.5) * sp) * du + A(3) * (A(1) - A(0.5) * sm) * L1[a];
    }
    part[0] = tsp;
    part[1] = tsm;
    lam[0] = lam[0] - sp * lam[0] + a0;
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        const A lp = A(0.5) * (lam[q] + lam[q + 1]), lm = A(0.5) * (lam[q] - lam[q + 1]);
        const A bc = A(cx(q)) * b[0] + A(cy(q)) * b[1] + A(cz(q)) * b[2];
        const A x = lam[q] - sp * lp - sm * lm + a0 + bc;
        const A y = lam[q + 1] - sp * lp + sm * lm + a0 - bc;
        lam[q] = x;
        lam[q + 1] = y;
    }
}

// Block sum of the per-thread parameter parts, added to this block's FP64
// accumulator (one slot per block, so the order of additions is fixed).  In
// FP32 the warps' sums are added as a double-float pair (TwoSum, exact to
// far below FP32 resolution) and converted once: FP64 arithmetic is slow on
// this part and every block ends with it.
template <typename A>
__device__ __forceinline__ void accumulate_parts(const A part[5], double* __restrict__ acc) {
    __shared__ A red[5][AT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        A v = part[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[c][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s;
        if constexpr (sizeof(A) == 4) {
            float h = 0.0f, l = 0.0f;
            for (int w = 0; w < AT / 32; ++w) df_add(h, l, red[threadIdx.x][w], 0.0f);
            s = (double)h + (double)l;
        } else {
            s = 0.0;
            for (int w = 0; w < AT / 32; ++w) s += red[threadIdx.x][w];
        }
        acc[(size_t)blockIdx.x * 5 + threadIdx.x] += s;
    }
}

// Cells whose reverse step involves a solid cell: some x + c_q, x - c_q or
// x + 2 c_q is solid.  Counts per block for the ordered compaction.
__global__ void __launch_bounds__(AT)
    k_adj_kind(const uint8_t* __restrict__ flags, GridDesc G, uint8_t* __restrict__ kind, int* __restrict__ block_count) {
    const long long x = (long long)blockIdx.x * AT + threadIdx.x;
    int near = 0;
    if (x < G.n) {
        const int i = (int)(x % G.nx), j = (int)((x / G.nx) % G.ny), k = (int)(x / ((long long)G.nx * G.ny));
        uint8_t v = KIND_SOLID;
        if (flags[x] == 0) {
            v = KIND_PLAIN;
            for (int q = 1; q < 19; ++q) {
                const bool s = flags[cell_at(G, i + cx(q), j + cy(q), k + cz(q))] != 0 ||
                               flags[cell_at(G, i - cx(q), j - cy(q), k - cz(q))] != 0 ||
                               flags[cell_at(G, i + 2 * cx(q), j + 2 * cy(q), k + 2 * cz(q))] != 0;
                if (s) v = KIND_NEAR;
            }
        }
        kind[x] = v;
        near = v == KIND_NEAR;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, near);
    __shared__ int wsum[AT / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(ballot);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < AT / 32; ++w) s += wsum[w];
        block_count[blockIdx.x] = s;
    }
}

// Ordered list of the near cells.  The block offsets are an exclusive scan
// of the per-block counts, done by every block over the blocks before it.
__global__ void __launch_bounds__(AT)
    k_adj_near_list(const uint8_t* __restrict__ kind, const int* __restrict__ block_count, GridDesc G,
                    int* __restrict__ list, int* __restrict__ count) {
    __shared__ int red[AT];
    __shared__ int wsum[AT / 32];
    int s = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += AT) s += block_count[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = AT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    const int base = red[0];
    const long long x = (long long)blockIdx.x * AT + threadIdx.x;
    const int near = x < G.n && kind[x] == KIND_NEAR;
    const unsigned ballot = __ballot_sync(0xffffffffu, near);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = __popc(ballot);
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += wsum[w];
    if (near) list[base + wbase + __popc(ballot & ((1u << lane) - 1u))] = (int)x;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        int tot = base;
        for (int w = 0; w < AT / 32; ++w) tot += wsum[w];
        *count = tot;
    }
}

// Reverse step on the cells that see no solid: h_q = g_q(x - c_q),
// lambda_q = nu_q(x + c_q).  Solid cells get nu = 0; near cells are left to
// k_adj_near.
template <typename S>
__global__ void __launch_bounds__(AT, sizeof(S) == 8 ? 1 : ADJ_MIN_CTAS)
    k_adj_plain(const S* __restrict__ gprev, const typename Store<S>::A* __restrict__ nu_next,
                typename Store<S>::A* __restrict__ nu_out, const uint8_t* __restrict__ kind, GridDesc G,
                AdjParams<typename Store<S>::A> P, double* __restrict__ acc) {
    using A = typename Store<S>::A;
    const long long x = (long long)blockIdx.x * AT + threadIdx.x;
    const size_t n = (size_t)G.n;
    A part[5] = {A(0), A(0), A(0), A(0), A(0)};
    if (x < G.n) {
        // the cell's kind is loaded beside the 38 loads of the plain case (a branch on it would
        // hold them back by one memory round trip); a cell of another kind drops them
        const uint8_t kd = kind[x];
        const int i = (int)(x % G.nx), j = (int)((x / G.nx) % G.ny), k = (int)(x / ((long long)G.nx * G.ny));
        // xs[1 + d] = i - d: the pull source x - c_q at index 1 + c, x + c_q at 1 - c
        const int xs[3] = {wrapc(i + 1, G.nx), i, wrapc(i - 1, G.nx)};
        const int ys[3] = {wrapc(j + 1, G.ny), j, wrapc(j - 1, G.ny)};
        const int zs[3] = {wrapc(k + 1, G.nz), k, wrapc(k - 1, G.nz)};
        A h[19], lam[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            const size_t src = (size_t)xs[1 + cx(q)] + (size_t)G.nx * ((size_t)ys[1 + cy(q)] + (size_t)G.ny * zs[1 + cz(q)]);
            const size_t dn = (size_t)xs[1 - cx(q)] + (size_t)G.nx * ((size_t)ys[1 - cy(q)] + (size_t)G.ny * zs[1 - cz(q)]);
            h[q] = Store<S>::load(gprev + (size_t)q * n + src, A(1));
            lam[q] = nu_next[(size_t)q * n + dn];
        }
        if (kd == KIND_SOLID) {
#pragma unroll
            for (int q = 0; q < 19; ++q) nu_out[(size_t)q * n + x] = A(0);
        } else if (kd == KIND_PLAIN) {
            trt_adjoint<A>(h, lam, P, part);
#pragma unroll
            for (int q = 0; q < 19; ++q) nu_out[(size_t)q * n + x] = lam[q];
        }
    }
    accumulate_parts<A>(part, acc);
}

// h^n at a near cell: the pull of the forward step with the CLI rule on
// links (wall at rest).
template <typename S>
__device__ __forceinline__ void near_pull(const S* __restrict__ g, const uint8_t* __restrict__ flags, const GridDesc& G,
                                          int i, int j, int k, const LinkFrame<typename Store<S>::A>& Fr, int cli,
                                          typename Store<S>::A (&h)[19]) {
    using A = typename Store<S>::A;
    const size_t n = (size_t)G.n;
    const long long x = cell_at(G, i, j, k);
    const int p[3] = {i, j, k}, n3[3] = {G.nx, G.ny, G.nz}, per[3] = {1, 1, 1};
    A d[3];
    int pu[3];
    Fr.offset(p, n3, per, d, pu);
    for (int q = 0; q < 19; ++q) {
        const long long s = cell_at(G, i - cx(q), j - cy(q), k - cz(q));
        if (q == 0 || flags[s] == 0) {
            h[q] = Store<S>::load(g + (size_t)q * n + s, A(1));
        } else {
            const int kk = opp(q);
            const long long far = cell_at(G, i + cx(q), j + cy(q), k + cz(q));
            const bool far_ok = flags[far] == 0;
            A delta, kappa0, alpha;
            cli_coeffs<A>(q, d, cli && far_ok, Fr.r, &delta, &kappa0, &alpha);
            const A gt_k = Store<S>::load(g + (size_t)kk * n + x, A(1));
            const A gt_q = Store<S>::load(g + (size_t)q * n + x, A(1));
            const A gt_far = far_ok ? Store<S>::load(g + (size_t)kk * n + far, A(1)) : A(0);
            h[q] = gt_k + kappa0 * gt_far - kappa0 * gt_q;
        }
    }
}

// lambda at a fluid cell next to the sphere: S^T nu with the link terms,
// plus (with_seed) the force's own dependence on g at the links.
template <typename A>
__device__ __forceinline__ void near_lambda(const A* __restrict__ nu, const uint8_t* __restrict__ flags,
                                            const GridDesc& G, int i, int j, int k, const LinkFrame<A>& Fr, int cli,
                                            bool with_seed, A seed, int axis, A (&lam)[19]) {
    const size_t n = (size_t)G.n;
    const long long x = cell_at(G, i, j, k);
    const int n3[3] = {G.nx, G.ny, G.nz}, per[3] = {1, 1, 1};
    const int px[3] = {i, j, k};
    A dx[3];
    int pu[3];
    Fr.offset(px, n3, per, dx, pu);
    lam[0] = nu[x];
    for (int q = 1; q < 19; ++q) {
        const int c[3] = {cx(q), cy(q), cz(q)};
        const long long y = cell_at(G, i + c[0], j + c[1], k + c[2]);
        A l;
        if (flags[y] == 0) {
            l = nu[(size_t)q * n + y];   // plain pull at y reads g_q(x)
            if (flags[cell_at(G, i + 2 * c[0], j + 2 * c[1], k + 2 * c[2])] != 0) {
                // link at y, incoming opp(q): its far cell is x
                const int py[3] = {wrapc(i + c[0], G.nx), wrapc(j + c[1], G.ny), wrapc(k + c[2], G.nz)};
                A dy[3], delta, kappa0, alpha;
                int pv[3];
                Fr.offset(py, n3, per, dy, pv);
                cli_coeffs<A>(opp(q), dy, cli != 0, Fr.r, &delta, &kappa0, &alpha);
                l += kappa0 * nu[(size_t)opp(q) * n + y];
            }
        } else {
            // link at x, incoming opp(q): g_q(x) is its g~_k, also in the force
            l = nu[(size_t)opp(q) * n + x];
            if (with_seed) l += seed * A(c[axis]);
        }
        if (flags[cell_at(G, i - c[0], j - c[1], k - c[2])] != 0) {
            // link at x, incoming q: -kappa0 g_q(x)
            const bool far_ok = flags[y] == 0;
            A delta, kappa0, alpha;
            cli_coeffs<A>(q, dx, cli && far_ok, Fr.r, &delta, &kappa0, &alpha);
            l -= kappa0 * nu[(size_t)q * n + x];
        }
        lam[q] = l;
    }
}

template <typename S>
__global__ void __launch_bounds__(AT)
    k_adj_near(const S* __restrict__ gprev, const typename Store<S>::A* __restrict__ nu_next,
               typename Store<S>::A* __restrict__ nu_out, const uint8_t* __restrict__ flags,
               const int* __restrict__ list, const int* __restrict__ count, GridDesc G,
               AdjParams<typename Store<S>::A> P, const ParticleState* __restrict__ ps, int cli, int with_seed,
               double* __restrict__ acc) {
    using A = typename Store<S>::A;
    __shared__ LinkFrame<A> Fr;
    if (threadIdx.x == 0) Fr.init(*ps);
    __syncthreads();
    const int t = blockIdx.x * AT + threadIdx.x;
    A part[5] = {A(0), A(0), A(0), A(0), A(0)};
    if (t < *count) {
        const long long x = list[t];
        const int i = (int)(x % G.nx), j = (int)((x / G.nx) % G.ny), k = (int)(x / ((long long)G.nx * G.ny));
        A h[19], lam[19];
        near_pull<S>(gprev, flags, G, i, j, k, Fr, cli, h);
        near_lambda<A>(nu_next, flags, G, i, j, k, Fr, cli, with_seed != 0, P.seed, P.axis, lam);
        trt_adjoint<A>(h, lam, P, part);
        const size_t n = (size_t)G.n;
        // the force's own dependence on h^n at the links (x, q): c_k = -c_q
        for (int q = 1; q < 19; ++q)
            if (flags[cell_at(G, i - cx(q), j - cy(q), k - cz(q))] != 0) {
                const int ca = P.axis == 0 ? cx(q) : (P.axis == 1 ? cy(q) : cz(q));
                lam[q] -= P.seed * A(ca);
            }
        for (int q = 0; q < 19; ++q) nu_out[(size_t)q * n + x] = lam[q];
    }
    accumulate_parts<A>(part, acc);
}

// lambda^0 and dJ/du0 = (dE/du0)^T lambda^0 with
// dE_q/du = w_q (3 c_q + 9 (c_q.u0) c_q - 3 u0), times the incoming dJ.
template <typename A>
__global__ void __launch_bounds__(AT)
    k_adj_init_grad(const A* __restrict__ nu, const uint8_t* __restrict__ flags, const uint8_t* __restrict__ kind,
                    GridDesc G, const double* __restrict__ u0, const ParticleState* __restrict__ ps, int cli, A seed,
                    int axis, const double* __restrict__ dJ, double* __restrict__ grad_u0) {
    __shared__ LinkFrame<A> Fr;
    if (threadIdx.x == 0) Fr.init(*ps);
    __syncthreads();
    const long long x = (long long)blockIdx.x * AT + threadIdx.x;
    if (x >= G.n) return;
    const size_t n = (size_t)G.n;
    if (kind[x] == KIND_SOLID) {
        for (int a = 0; a < 3; ++a) grad_u0[(size_t)a * n + x] = 0.0;
        return;
    }
    const int i = (int)(x % G.nx), j = (int)((x / G.nx) % G.ny), k = (int)(x / ((long long)G.nx * G.ny));
    A lam[19];
    if (kind[x] == KIND_PLAIN) {
        for (int q = 0; q < 19; ++q) lam[q] = nu[(size_t)q * n + cell_at(G, i + cx(q), j + cy(q), k + cz(q))];
    } else {
        near_lambda<A>(nu, flags, G, i, j, k, Fr, cli, true, seed, axis, lam);
    }
    const double u[3] = {u0[x], u0[n + x], u0[2 * n + x]};
    double L0 = 0.0, L1[3] = {0.0, 0.0, 0.0}, L2u[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < 19; ++q) {
        const double wl = wgt<double>(q) * (double)lam[q];
        const double c[3] = {(double)cx(q), (double)cy(q), (double)cz(q)};
        const double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        L0 += wl;
        for (int a = 0; a < 3; ++a) {
            L1[a] += wl * c[a];
            L2u[a] += wl * cu * c[a];
        }
    }
    const double s = *dJ;
    for (int a = 0; a < 3; ++a) grad_u0[(size_t)a * n + x] = s * (3.0 * L1[a] + 9.0 * L2u[a] - 3.0 * L0 * u[a]);
}

// Force of the step from the boundary kernel's partials (fixed block order).
__global__ void k_adj_force(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * 6 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

__global__ void k_adj_mean(const double* __restrict__ forces, int nsteps, int axis, double* __restrict__ J) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int n = 0; n < nsteps; ++n) s += forces[(size_t)n * 3 + axis];
        *J = s / (double)nsteps;
    }
}

// Parameter gradients from the per-block accumulators:
// dJ/dtau = ds+/dtau sum part0 + ds-/dtau sum part1 with ds+/dtau = -s+^2 and
// ds-/dtau = s-^2 Lambda / (tau - 1/2)^2; dJ/dF_a = sum part_{2+a}.
__global__ void k_adj_params(const double* __restrict__ acc, int nblocks, double tau, double magic,
                             const double* __restrict__ dJ, double* __restrict__ grad_tau,
                             double* __restrict__ grad_force) {
    __shared__ double red[5][AT];
    double v[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += AT)
        for (int c = 0; c < 5; ++c) v[c] += acc[(size_t)b * 5 + c];
    for (int c = 0; c < 5; ++c) red[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int h = AT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 5; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sp = 1.0 / tau, sm = 1.0 / (0.5 + magic / (tau - 0.5));
        const double dsp = -sp * sp, dsm = sm * sm * magic / ((tau - 0.5) * (tau - 0.5));
        const double s = *dJ;
        if (grad_tau) *grad_tau = s * (dsp * red[0][0] + dsm * red[1][0]);
        if (grad_force)
            for (int a = 0; a < 3; ++a) grad_force[a] = s * red[2 + a][0];
    }
}

template <typename F>
void with_adj_storage(int prec, F&& f) {
    if (prec == LBMP_FP64) f((double*)nullptr);
    else f((float*)nullptr);
}

}  // namespace

struct AdjointEngine {
    int nsteps = 0, interval = 0, nckpt = 0, axis = 0;
    size_t state_bytes = 0, nu_bytes = 0;
    void* ckpt = nullptr;     // nckpt states
    void* seg = nullptr;      // interval states (slot 0 unused: it is the checkpoint)
    void* nu[2] = {nullptr, nullptr};
    double* u0 = nullptr;     // copy of the initial velocity field [3][n]
    double* forces = nullptr; // [nsteps][3]
    double* acc = nullptr;    // [acc_blocks][5]
    int acc_blocks = 0, plain_blocks = 0, near_blocks = 0, near_cells = 0;
    uint8_t* kind = nullptr;
    int* blk = nullptr;
    int* near_list = nullptr;
    int* near_count = nullptr;
    int near_cap = 0;
    bool forward_done = false;
    bool geometry_done = false;   // kind bytes and near list of the (fixed) sphere
    double tau = 0, F[3] = {0, 0, 0};
    // the forward pass (one per parity of the handle's buffers) and the reverse
    // sweep replayed from CUDA graphs; dropped when tau, the body force or the
    // objective's axis change
    cudaGraphExec_t gfwd[2] = {nullptr, nullptr};
    cudaGraphExec_t gbwd = nullptr;
    double graph_tau = -1.0, graph_F[3] = {0, 0, 0};
    int graph_axis = -1;
    cudaStream_t capture_stream = nullptr;
};

namespace {

template <typename S>
void forward_step(lbmp_handle* h, const S* src, S* dst, double* force_out) {
    using A = typename Store<S>::A;
    const CollideParams<A> p = collide_params<A>(h);
    launch_bulk<S>(src, dst, h->G, p, h->status, h->stream);
    int nb = 0;
    launch_boundary<S>(src, dst, h->flags[h->fcur], h->list, h->count, h->list_cap, h->G, p, h->d_ps,
                       h->cfg.boundary == LBMP_CLI ? 1 : 0, h->partials, &nb, h->status, h->stream);
    launch_refill<S>(dst, h->flags[h->fcur], h->flags[h->fcur], h->G, h->box, h->d_ps, A(1), A(1), A(0), h->stream);
    if (force_out) k_adj_force<<<1, 32, 0, h->stream>>>(h->partials, nb, force_out);
}

template <typename S>
S* state(AdjointEngine* E, int m, int j, size_t n) {
    if (j == 0) return (S*)E->ckpt + (size_t)m * 19 * n;
    return (S*)E->seg + (size_t)j * 19 * n;
}

void drop_graphs(AdjointEngine* E) {
    for (auto& g : E->gfwd)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (E->gbwd) {
        cudaGraphExecDestroy(E->gbwd);
        E->gbwd = nullptr;
    }
}

// Enqueues `body` on the handle's stream: replayed from *graph, captured on a
// private stream the first time (the caller's stream may be the legacy
// default stream, which cannot be captured).  Profiling runs plain launches.
template <typename F>
lbmp_status captured(lbmp_handle* h, AdjointEngine* E, cudaGraphExec_t* graph, F&& body) {
    if (h->profiling) {
        body();
        return LBMP_OK;
    }
    if (!*graph) {
        if (!E->capture_stream && cudaStreamCreateWithFlags(&E->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
            return LBMP_ERR_CUDA;
        // the capture stream starts after the work already queued on the caller's stream
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return LBMP_ERR_CUDA;
        cudaEventRecord(ev, h->stream);
        cudaStreamWaitEvent(E->capture_stream, ev, 0);
        cudaEventDestroy(ev);
        cudaStream_t user = h->stream;
        h->stream = E->capture_stream;
        if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            h->stream = user;
            return LBMP_ERR_CUDA;
        }
        body();
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
        h->stream = user;
        if (e != cudaSuccess) return LBMP_ERR_CUDA;
        const cudaError_t e2 = cudaGraphInstantiate(graph, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) return LBMP_ERR_CUDA;
    }
    return cudaGraphLaunch(*graph, h->stream) == cudaSuccess ? LBMP_OK : LBMP_ERR_CUDA;
}

void release(lbmp_handle* h, AdjointEngine* E) {
    drop_graphs(E);
    if (E->capture_stream) cudaStreamDestroy(E->capture_stream);
    void* ptrs[] = {E->ckpt, E->seg, E->nu[0], E->nu[1], E->u0, E->forces, E->acc, E->kind, E->blk, E->near_list,
                    E->near_count};
    for (void* p : ptrs)
        if (p) handle_free(h, p);
    *E = AdjointEngine();
}

}  // namespace

void adjoint_destroy(lbmp_handle* h) {
    if (!h->adj) return;
    drop_graphs(h->adj);
    if (h->adj->capture_stream) cudaStreamDestroy(h->adj->capture_stream);
    delete h->adj;   // device memory is released with the handle's allocations
    h->adj = nullptr;
}

lbmp_status adjoint_check(const lbmp_handle* h, std::string* why) {
    if (h->amr || h->batch) return *why = "the drag adjoint runs on a single uniform grid", LBMP_ERR_UNSUPPORTED;
    if (!h->has_particle) return *why = "the drag adjoint needs a sphere", LBMP_ERR_INVALID_ARG;
    if (h->h_ps.fixed != 1) return *why = "the drag adjoint needs the sphere held fixed", LBMP_ERR_UNSUPPORTED;
    for (int a = 0; a < 3; ++a) {
        if (!h->G.periodic[a]) return *why = "the drag adjoint needs a periodic box", LBMP_ERR_UNSUPPORTED;
        if (h->h_ps.u[a] != 0.0 || h->h_ps.w[a] != 0.0)
            return *why = "the drag adjoint needs the sphere at rest", LBMP_ERR_UNSUPPORTED;
    }
    if (h->cfg.precision == LBMP_FP16) return *why = "the drag adjoint runs in FP32 or FP64", LBMP_ERR_UNSUPPORTED;
    if (h->cfg.bulk_factor != 1.0) return *why = "the drag adjoint is the reverse of the TRT step (bulk factor 1)", LBMP_ERR_UNSUPPORTED;
    return LBMP_OK;
}

lbmp_status adjoint_forward(lbmp_handle* h, const double* u0, int nsteps, int interval, int axis, double* J,
                            double* forces) {
    if (!h->adj) h->adj = new AdjointEngine();
    AdjointEngine* E = h->adj;
    const size_t n = (size_t)h->G.n;
    const size_t es = h->cfg.precision == LBMP_FP64 ? 8 : 4;
    const int nckpt = (nsteps + interval - 1) / interval;
    if (E->nsteps != nsteps || E->interval != interval) {
        release(h, E);
        E->nsteps = nsteps;
        E->interval = interval;
        E->nckpt = nckpt;
        E->state_bytes = es * 19 * n;
        E->nu_bytes = es * 19 * n;
        E->plain_blocks = (int)((n + AT - 1) / AT);
        E->near_cap = (int)n;
        E->near_blocks = 0;
        E->acc_blocks = E->plain_blocks * 2;   // plain blocks, then at most as many near blocks
        E->ckpt = handle_alloc(h, E->state_bytes * (size_t)nckpt);
        E->seg = handle_alloc(h, E->state_bytes * (size_t)interval);
        E->nu[0] = handle_alloc(h, E->nu_bytes);
        E->nu[1] = handle_alloc(h, E->nu_bytes);
        E->u0 = (double*)handle_alloc(h, sizeof(double) * 3 * n);
        E->forces = (double*)handle_alloc(h, sizeof(double) * 3 * (size_t)nsteps);
        E->acc = (double*)handle_alloc(h, sizeof(double) * 5 * (size_t)E->acc_blocks);
        E->kind = (uint8_t*)handle_alloc(h, n);
        E->blk = (int*)handle_alloc(h, sizeof(int) * (size_t)E->plain_blocks);
        E->near_list = (int*)handle_alloc(h, sizeof(int) * n);
        E->near_count = (int*)handle_alloc(h, sizeof(int));
        if (!E->ckpt || !E->seg || !E->nu[0] || !E->nu[1] || !E->u0 || !E->forces || !E->acc || !E->kind || !E->blk ||
            !E->near_list || !E->near_count) {
            release(h, E);
            return LBMP_ERR_OOM;
        }
    }
    E->axis = axis;
    E->tau = h->tau;
    for (int a = 0; a < 3; ++a) E->F[a] = h->body_force[a];
    if (E->graph_tau != h->tau || E->graph_F[0] != h->body_force[0] || E->graph_F[1] != h->body_force[1] ||
        E->graph_F[2] != h->body_force[2] || E->graph_axis != axis) {
        drop_graphs(E);
        E->graph_tau = h->tau;
        E->graph_axis = axis;
        for (int a = 0; a < 3; ++a) E->graph_F[a] = h->body_force[a];
    }
    if (!E->geometry_done) {   // cells of the reverse step next to the (fixed) sphere
        const unsigned gb = (unsigned)E->plain_blocks;
        k_adj_kind<<<gb, AT, 0, h->stream>>>(h->flags[h->fcur], h->G, E->kind, E->blk);
        k_adj_near_list<<<gb, AT, 0, h->stream>>>(E->kind, E->blk, h->G, E->near_list, E->near_count);
        h->launches += 2;
        if (cudaMemcpyAsync(&E->near_cells, E->near_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return LBMP_ERR_CUDA;
        h->d2h += sizeof(int);
        E->near_blocks = std::max(1, (E->near_cells + AT - 1) / AT);
        E->geometry_done = true;
    }
    cudaMemcpyAsync(E->u0, u0, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, h->stream);
    const int par = h->cur;
    const lbmp_status st = captured(h, E, &E->gfwd[par], [&]() {
        with_adj_storage(h->cfg.precision, [&](auto tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            const double zero[3] = {0.0, 0.0, 0.0};
            S* a = (S*)h->pops[par];
            S* b = (S*)h->pops[1 - par];
            launch_init_equilibrium<S>(a, h->flags[h->fcur], h->G, 1.0, zero, E->u0, (typename Store<S>::A)1,
                                       h->stream);
            cudaMemcpyAsync(E->ckpt, a, E->state_bytes, cudaMemcpyDeviceToDevice, h->stream);
            for (int s = 1; s <= nsteps; ++s) {
                forward_step<S>(h, a, b, E->forces + (size_t)(s - 1) * 3);
                std::swap(a, b);
                if (s % interval == 0 && s / interval < nckpt)
                    cudaMemcpyAsync((char*)E->ckpt + E->state_bytes * (size_t)(s / interval), a, E->state_bytes,
                                    cudaMemcpyDeviceToDevice, h->stream);
            }
        });
    });
    if (st != LBMP_OK) return st;
    h->cur = (par + nsteps) & 1;
    h->steps += nsteps;
    h->launches += 1 + 4LL * nsteps;
    h->updates += (long long)nsteps * h->G.n;
    k_adj_mean<<<1, 32, 0, h->stream>>>(E->forces, nsteps, axis, J);
    h->launches += 1;
    if (forces)
        cudaMemcpyAsync(forces, E->forces, sizeof(double) * 3 * (size_t)nsteps, cudaMemcpyDeviceToDevice, h->stream);
    E->forward_done = true;
    if (cudaGetLastError() != cudaSuccess) return LBMP_ERR_CUDA;
    return LBMP_OK;
}

lbmp_status adjoint_backward(lbmp_handle* h, const double* dJ, double* grad_tau, double* grad_force, double* grad_u0,
                             std::string* why) {
    AdjointEngine* E = h->adj;
    if (!E || !E->forward_done) return *why = "lbmp_drag_backward needs a preceding lbmp_drag_forward", LBMP_ERR_INVALID_ARG;
    if (E->tau != h->tau || E->F[0] != h->body_force[0] || E->F[1] != h->body_force[1] || E->F[2] != h->body_force[2])
        return *why = "tau or the body force changed since lbmp_drag_forward", LBMP_ERR_INVALID_ARG;
    const size_t n = (size_t)h->G.n;
    const int N = E->nsteps, K = E->interval;
    const int cli = h->cfg.boundary == LBMP_CLI ? 1 : 0;
    const unsigned gb = (unsigned)E->plain_blocks, gn = (unsigned)E->near_blocks;
    lbmp_status st = LBMP_OK;
    with_adj_storage(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using A = typename Store<S>::A;
        AdjParams<A> P;
        double sp, sm;
        relaxation_rates(h->tau, h->magic, &sp, &sm);
        P.sp = (A)sp;
        P.sm = (A)sm;
        for (int a = 0; a < 3; ++a) P.F[a] = (A)h->body_force[a];
        P.seed = (A)(1.0 / (double)N);
        P.axis = E->axis;
        st = captured(h, E, &E->gbwd, [&]() {
            cudaMemsetAsync(E->acc, 0, sizeof(double) * 5 * (size_t)E->acc_blocks, h->stream);
            cudaMemsetAsync(E->nu[0], 0, E->nu_bytes, h->stream);
            int cur = 0;   // nu[cur] holds nu^{n+1}
            for (int m = E->nckpt - 1; m >= 0; --m) {
                const int s0 = m * K, len = std::min(K, N - s0);
                for (int j = 1; j < len; ++j)
                    forward_step<S>(h, state<S>(E, m, j - 1, n), state<S>(E, m, j, n), nullptr);
                for (int s = s0 + len; s > s0; --s) {
                    const S* gprev = state<S>(E, m, s - 1 - s0, n);
                    const A* nu_next = (const A*)E->nu[cur];
                    A* nu_out = (A*)E->nu[1 - cur];
                    const long long ev = profile_mark(h);
                    k_adj_plain<S><<<gb, AT, 0, h->stream>>>(gprev, nu_next, nu_out, E->kind, h->G, P, E->acc);
                    // algorithmic bytes: 19 populations of g^{n-1} read, 19 adjoint values read and written per cell
                    const double cells = (double)n - (double)E->near_cells;
                    profile_kernel(h, ev, profile_mark(h), cells * (19.0 * sizeof(S) + 38.0 * sizeof(A)), cells);
                    k_adj_near<S><<<gn, AT, 0, h->stream>>>(gprev, nu_next, nu_out, h->flags[h->fcur], E->near_list,
                                                           E->near_count, h->G, P, h->d_ps, cli, s < N ? 1 : 0,
                                                           E->acc + (size_t)5 * E->plain_blocks);
                    cur = 1 - cur;
                }
            }
        });
        h->launches += 3LL * (N - E->nckpt) + 2LL * N;
        if (st == LBMP_OK && grad_u0) {   // nu^1 sits in nu[N % 2] after N reverse steps
            k_adj_init_grad<A><<<gb, AT, 0, h->stream>>>((const A*)E->nu[N & 1], h->flags[h->fcur], E->kind, h->G,
                                                         E->u0, h->d_ps, cli, P.seed, E->axis, dJ, grad_u0);
            h->launches += 1;
        }
    });
    if (st != LBMP_OK) return st;
    k_adj_params<<<1, AT, 0, h->stream>>>(E->acc, E->plain_blocks + E->near_blocks, h->tau, h->magic, dJ, grad_tau,
                                          grad_force);
    h->launches += 1;
    if (cudaGetLastError() != cudaSuccess) return LBMP_ERR_CUDA;
    return LBMP_OK;
}

}  // namespace lbmp
