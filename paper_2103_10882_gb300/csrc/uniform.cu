// Uniform-grid kernels of the coupled step (Algorithm 1):
//   k_bulk       stream (pull) + TRT collide of every cell         Sec. 2.1, Eq. LBE
//   k_boundary   re-does the cells next to the sphere with CLI links and
//                sums the momentum-exchange force/torque in FP64     Sec. 2.3
//   k_particle   force averaging, gravity, virtual mass, Velocity Verlet   Sec. 2.2, 3.3
//   k_flags_box, k_refill, k_build_links   remap after the sphere moved    Sec. 2.3
// Populations are stored as deviations g = f - w in SoA layout [q][z][y][x].
#include <cuda_fp16.h>

#include <type_traits>

#include "internal.h"
#include "physics.cuh"

namespace lbmp {
namespace {

constexpr int BULK_THREADS = 256;

// ------------------------------------------------------------------ bulk
// One thread per cell, pull form: g_q(x, t+1) = g~_q(x - c_q, t), then TRT.
// WALLS: some axis has no-slip walls (bounce-back at the domain edge);
// FORCED: fluid body force present.  Both are compile-time so the common
// periodic, unforced case carries no per-population branches.  Spatial
// offsets are 32-bit (cells < 2^31); each population array is addressed
// from its own base pointer.
template <typename S, bool WALLS, bool FORCED>
__global__ void __launch_bounds__(BULK_THREADS)
    k_bulk(const S* __restrict__ src, S* __restrict__ dst, GridDesc G, CollideParams<typename Store<S>::A> P,
           int* __restrict__ status) {
    using A = typename Store<S>::A;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    if (x >= nx || y >= ny) return;
    const size_t n = (size_t)G.n;
    const int cell = x + nx * (y + ny * z);
    // source coordinate x - c for c = -1, 0, +1 (-1 marks a wall)
    int xs[3], ys[3], zs[3];
    xs[1] = x;
    ys[1] = y;
    zs[1] = z;
    xs[0] = x + 1 < nx ? x + 1 : (WALLS && !G.periodic[0] ? -1 : 0);
    xs[2] = x > 0 ? x - 1 : (WALLS && !G.periodic[0] ? -1 : nx - 1);
    ys[0] = y + 1 < ny ? y + 1 : (WALLS && !G.periodic[1] ? -1 : 0);
    ys[2] = y > 0 ? y - 1 : (WALLS && !G.periodic[1] ? -1 : ny - 1);
    zs[0] = z + 1 < nz ? z + 1 : (WALLS && !G.periodic[2] ? -1 : 0);
    zs[2] = z > 0 ? z - 1 : (WALLS && !G.periodic[2] ? -1 : nz - 1);
    A g[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int sx = xs[cx(q) + 1], sy = ys[cy(q) + 1], sz = zs[cz(q) + 1];
        if (WALLS && (sx < 0 || sy < 0 || sz < 0)) {   // no-slip wall: bounce-back (moving: Ladd's term)
            const int xyz[3] = {x, y, z};
            g[q] = Store<S>::load(src + (size_t)opp(q) * n + cell, P.inv_scale) + wall_term<A>(G, q, xyz);
        } else {
            const int off = sx + nx * (sy + ny * sz);
            g[q] = Store<S>::load(src + (size_t)q * n + off, P.inv_scale);
        }
    }
    trt_collide<A, FORCED>(g, P, status);
#pragma unroll
    for (int q = 0; q < 19; ++q) Store<S>::store(dst + (size_t)q * n + cell, g[q], P.scale);
}

// FP16 storage, unforced: the same update as k_bulk, two cells (x, x + 1,
// x even) per thread.  Every population is read as the aligned pair of
// halves of its source row; the populations shifted along x take their
// outer half from the neighbouring lane (a shuffle); the first lane of a
// warp (rows start there) and the last pair of a warp or of a row load that
// one half themselves.  The collision runs on the stored, scaled values
// (trt_collide's SCALED form), so neither the loads nor the stores multiply
// by the scale, and TRT or MRT is chosen at compile time.  nx is even; rows
// hold whole pairs.
constexpr int BULK2_THREADS = 256;
template <bool WALLS, bool MRT>
__global__ void __launch_bounds__(BULK2_THREADS)
    k_bulk_h2(const __half* __restrict__ src, __half* __restrict__ dst, GridDesc G, CollideParams<float> P,
              int* __restrict__ status) {
    const int xp = blockIdx.x * blockDim.x + threadIdx.x;   // pair index
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int lane = threadIdx.x & 31;   // blockDim.x is a multiple of 32: a warp is one run of a row
    const bool valid = 2 * xp < nx && y < ny;
    const int x = valid ? 2 * xp : 0;
    const int yy = valid ? y : 0;
    const size_t n = (size_t)G.n;
    const int cell = x + nx * (yy + ny * z);
    int ys[3], zs[3];
    ys[1] = yy;
    zs[1] = z;
    ys[0] = yy + 1 < ny ? yy + 1 : (WALLS && !G.periodic[1] ? -1 : 0);
    ys[2] = yy > 0 ? yy - 1 : (WALLS && !G.periodic[1] ? -1 : ny - 1);
    zs[0] = z + 1 < nz ? z + 1 : (WALLS && !G.periodic[2] ? -1 : 0);
    zs[2] = z > 0 ? z - 1 : (WALLS && !G.periodic[2] ? -1 : nz - 1);
    // x - 1 of the pair's first cell and x + 2 of its second (-1: beyond a wall)
    const int xm = x > 0 ? x - 1 : (WALLS && !G.periodic[0] ? -1 : nx - 1);
    const int xq = x + 2 < nx ? x + 2 : (WALLS && !G.periodic[0] ? -1 : 0);
    // all loads first (the pairs, then the outer halves of the shifted populations, every lane
    // loading one: the lanes that need none read their own pair's first half), then the shuffles
    __half2 pr[19];
    __half ex[19];
    bool yw[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int sy = ys[cy(q) + 1], sz = zs[cz(q) + 1];
        yw[q] = WALLS && (sy < 0 || sz < 0);
        const int row = nx * ((yw[q] ? yy : sy) + ny * (yw[q] ? z : sz));
        const __half* pq = src + (size_t)q * n;
        pr[q] = __ldg(reinterpret_cast<const __half2*>(pq + row + x));
        if (cx(q) != 0) {
            const int xe = cx(q) == 1 ? xm : xq;
            const bool need = cx(q) == 1 ? lane == 0 : (lane == 31 || x + 2 >= nx);   // warp or row end
            ex[q] = __ldg(pq + row + ((need && xe >= 0) ? xe : x));
        }
    }
    float g0[19], g1[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const __half2 p = pr[q];
        float a, b;
        if (cx(q) == 0) {
            a = __low2float(p);
            b = __high2float(p);
        } else if (cx(q) == 1) {   // sources x - 1 and x
            const float prev = __shfl_up_sync(0xffffffffu, __high2float(p), 1);
            a = lane == 0 ? __half2float(ex[q]) : prev;
            b = __low2float(p);
        } else {                   // sources x + 1 and x + 2
            const float next = __shfl_down_sync(0xffffffffu, __low2float(p), 1);
            a = __high2float(p);
            b = (lane == 31 || x + 2 >= nx) ? __half2float(ex[q]) : next;
        }
        if (WALLS) {   // bounce-back (moving walls: Ladd's term, scaled like the stored values)
            const bool wa = yw[q] || (cx(q) == 1 && xm < 0);
            const bool wb = yw[q] || (cx(q) == -1 && xq < 0);
            if (wa || wb) {
                const __half2 o = *reinterpret_cast<const __half2*>(src + (size_t)opp(q) * n + cell);
                const int xyz0[3] = {x, yy, z}, xyz1[3] = {x + 1, yy, z};
                if (wa) a = __low2float(o) + wall_term<float>(G, q, xyz0) * P.scale;
                if (wb) b = __high2float(o) + wall_term<float>(G, q, xyz1) * P.scale;
            }
        }
        g0[q] = a;
        g1[q] = b;
    }
    if (!valid) return;
    trt_collide<float, false, true, MRT ? 1 : 0, true>(g0, P, status);
    trt_collide<float, false, true, MRT ? 1 : 0, true>(g1, P, status);
#pragma unroll
    for (int q = 0; q < 19; ++q)
        __stcs(reinterpret_cast<__half2*>(dst + (size_t)q * n + cell), __floats2half2_rn(g0[q], g1[q]));
}

// -------------------------------------------------------------- boundary
// One warp per fluid cell that has a solid neighbour, lane q handling
// population q: pulls from solid cells are replaced by the CLI rule of
// Sec. 2.3 (link geometry in the population arithmetic, force and torque
// summed in FP64), then the warp collides the cell cooperatively and writes
// it.  Each block covers 8 list entries per pass; blocks past the end of the
// list write zero partials.
constexpr int BNDW_THREADS = 256;
template <typename S, bool FORCED>
__global__ void __launch_bounds__(BNDW_THREADS)
    k_boundary(const S* __restrict__ src, S* __restrict__ dst, const uint8_t* __restrict__ flags,
               const int* __restrict__ list, const int* __restrict__ count, GridDesc G,
               CollideParams<typename Store<S>::A> P, const ParticleState* __restrict__ ps, int cli,
               double* __restrict__ partials, int* __restrict__ status) {
    using A = typename Store<S>::A;
    __shared__ LinkFrame<A> Fr;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (BNDW_THREADS / 32);
    const int cnt = *count;
    if ((int)blockIdx.x * (BNDW_THREADS / 32) >= cnt) {   // uniform across the block
        if (threadIdx.x < 6) partials[(size_t)blockIdx.x * 6 + threadIdx.x] = 0.0;
        return;
    }
    if (threadIdx.x == 0) Fr.init(*ps);
    __syncthreads();
    const size_t n = (size_t)G.n;
    const int n3[3] = {G.nx, G.ny, G.nz};
    LinkSums<A> acc;
    for (int w = blockIdx.x * (BNDW_THREADS / 32) + wib; w < cnt; w += nwarps) {
        const int cell = list[w];
        const int x = cell % G.nx, y = (cell / G.nx) % G.ny, z = cell / (G.nx * G.ny);
        A gq = A(0);
        if (lane < 19) {
            const int q = lane;
            const int c[3] = {cx(q), cy(q), cz(q)};
            const int xyz[3] = {x, y, z};
            int s3[3], f3[3];
            bool wall = false, far_ok = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                s3[a] = src_coord(xyz[a], c[a], n3[a], G.periodic[a]);    // x - c_q
                f3[a] = src_coord(xyz[a], -c[a], n3[a], G.periodic[a]);   // x + c_q
                wall |= s3[a] < 0;
                far_ok &= f3[a] >= 0;
            }
            if (wall) {
                gq = Store<S>::load(src + (size_t)opp(q) * n + cell, P.inv_scale) + wall_term<A>(G, q, xyz);
            } else {
                const size_t sidx = (size_t)s3[0] + (size_t)G.nx * ((size_t)s3[1] + (size_t)G.ny * (size_t)s3[2]);
                if (q == 0 || flags[sidx] == 0) {
                    gq = Store<S>::load(src + (size_t)q * n + sidx, P.inv_scale);
                } else {
                    const int k = opp(q);
                    size_t far = 0;
                    if (far_ok) {
                        far = (size_t)f3[0] + (size_t)G.nx * ((size_t)f3[1] + (size_t)G.ny * (size_t)f3[2]);
                        far_ok = flags[far] == 0;
                    }
                    A d[3], fl[3], tl[3];
                    int pu[3];
                    Fr.offset(xyz, n3, G.periodic, d, pu);
                    const A gt_k = Store<S>::load(src + (size_t)k * n + cell, P.inv_scale);
                    const A gt_q = Store<S>::load(src + (size_t)q * n + cell, P.inv_scale);
                    const A gt_far = far_ok ? Store<S>::load(src + (size_t)k * n + far, P.inv_scale) : A(0);
                    gq = cli_link<A>(q, d, cli && far_ok, gt_k, gt_q, gt_far, Fr, fl, tl);
                    acc.add(k, pu, fl, tl);
                }
            }
        }
        gq = warp_trt_collide<A, FORCED>(gq, lane, P, status);
        if (lane < 19) Store<S>::store(dst + (size_t)lane * n + cell, gq, P.scale);
    }
    block_link_sums<BNDW_THREADS>(acc, ps->x, partials + (size_t)blockIdx.x * 6);
}

// -------------------------------------------------------------- particle
// Sums the per-block partial forces in a fixed order, then Algorithm 1:
// average over two steps, gravity/buoyancy F_g = (rho_p - rho_f) g V,
// virtual force/torque from the previous accelerations, and Velocity
// Verlet (kick-drift-kick) with m = (rho_p + C_v) V, I = 2/5 (rho_p + C_vw) V r^2.
constexpr int PART_THREADS = 256;

__global__ void __launch_bounds__(PART_THREADS)
    k_particle(ParticleState* __restrict__ ps, const double* __restrict__ partials, int nblocks, GridDesc G,
               double* __restrict__ history, int hist_cap, int* __restrict__ status) {
    particle_block_update<PART_THREADS>(ps, partials, nblocks, G, history, hist_cap, status);
}

// ------------------------------------------------------------------ remap
__global__ void k_flags_full(uint8_t* __restrict__ flags, GridDesc G, const ParticleState* __restrict__ ps) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G.n) return;
    const int ij = c % (G.nx * G.ny);
    const int i = ij % G.nx, j = ij / G.nx, k = c / (G.nx * G.ny);
    flags[c] = (ps->present && inside_ball(i, j, k, G, *ps)) ? 1 : 0;
}

__global__ void k_flags_box(uint8_t* __restrict__ flags_next, GridDesc G, BoxDesc B,
                            const ParticleState* __restrict__ ps) {
    __shared__ BoxFrame F;
    const int n3[3] = {G.nx, G.ny, G.nz};
    if (threadIdx.x == 0) box_frame_init(F, n3, G.periodic, B, *ps);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.cells) return;
    int p[3];
    if (!box_cell(t, n3, G.periodic, B, F, p)) return;
    const size_t c = (size_t)p[0] + (size_t)G.nx * ((size_t)p[1] + (size_t)G.ny * (size_t)p[2]);
    flags_next[c] = ball_flag(p, n3, G.periodic, F, *ps) ? 1 : 0;
}

// Refill of the uncovered cell (i, j, k) = index c by the whole warp
// (Sec. 2.3): lane q = 1..18 takes the neighbour (i, j, k) + c_q (wrapped on
// periodic axes; none beyond a wall), counted when it is fluid before (fcur)
// and after (fnext) the move, with its density 1 + sum_p g_p and momentum
// sum_p c_p g_p (for Grad's strain rate from the face neighbours).  The mean
// density and the rigid-body velocity u_p + omega_p x (x - x_p) give the
// equilibrium, plus Grad's term when gcoef != 0; lane q < 19 writes
// population q.  Every lane calls it with the same cell.
template <typename S>
__device__ __forceinline__ void refill_warp(S* __restrict__ pops, const uint8_t* __restrict__ fcur,
                                            const uint8_t* __restrict__ fnext, const GridDesc& G, const int n3[3],
                                            const ParticleState& P, int i, int j, int k, size_t c,
                                            typename Store<S>::A scale, typename Store<S>::A inv_scale,
                                            typename Store<S>::A gcoef) {
    using A = typename Store<S>::A;
    const int lane = threadIdx.x & 31;
    const size_t n = (size_t)G.n;
    bool ok = false;
    A r = A(0), mo[3] = {A(0), A(0), A(0)};
    if (lane >= 1 && lane < 19) {
        int v[3] = {i + cx(lane), j + cy(lane), k + cz(lane)};
        bool in = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (v[a] < 0 || v[a] >= n3[a]) {
                if (!G.periodic[a]) in = false;
                v[a] = (v[a] + n3[a]) % n3[a];
            }
        }
        if (in) {
            const size_t y = (size_t)v[0] + (size_t)G.nx * ((size_t)v[1] + (size_t)G.ny * (size_t)v[2]);
            if (fcur[y] == 0 && fnext[y] == 0) {
                ok = true;
                A gp[19];
#pragma unroll
                for (int q = 0; q < 19; ++q) gp[q] = Store<S>::load(pops + (size_t)q * n + y, inv_scale);
                r = A(1);
#pragma unroll
                for (int q = 0; q < 19; ++q) r += gp[q];
#pragma unroll
                for (int q = 1; q < 19; ++q) {
                    mo[0] += A(cx(q)) * gp[q];
                    mo[1] += A(cy(q)) * gp[q];
                    mo[2] += A(cz(q)) * gp[q];
                }
            }
        }
    }
    const unsigned okm = __ballot_sync(0xffffffffu, ok);
    A rs = ok ? r : A(0);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, off);
    const int cnt = __popc(okm);
    const A rho = cnt > 0 ? rs / A(cnt) : A(1);
    const double d[3] = {wrap_diff((i + 0.5) - P.x[0], G.nx, G.periodic[0]),
                         wrap_diff((j + 0.5) - P.x[1], G.ny, G.periodic[1]),
                         wrap_diff((k + 0.5) - P.x[2], G.nz, G.periodic[2])};
    const A u[3] = {A(P.u[0] + (P.w[1] * d[2] - P.w[2] * d[1])), A(P.u[1] + (P.w[2] * d[0] - P.w[0] * d[2])),
                    A(P.u[2] + (P.w[0] * d[1] - P.w[1] * d[0]))};
    const A uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    A Sr[6] = {A(0), A(0), A(0), A(0), A(0), A(0)};
    if (gcoef != A(0)) {   // Grad refill: face neighbour q = 1 + 2 a (+1 for -e_a), fluid before and after the move
        auto nb = [&](int a, int sgn, A uo[3]) {
            const int q = 1 + 2 * a + (sgn > 0 ? 0 : 1);
#pragma unroll
            for (int m = 0; m < 3; ++m) uo[m] = __shfl_sync(0xffffffffu, mo[m], q);
            return ((okm >> q) & 1u) != 0;
        };
        refill_strain<A>(nb, u, Sr);
    }
    if (lane < 19) {
        const int q = lane;
        const A cu = A(cx(q)) * u[0] + A(cy(q)) * u[1] + A(cz(q)) * u[2];
        A e = wgt<A>(q) * ((rho - A(1)) + A(3) * cu + A(4.5) * cu * cu - A(1.5) * uu);
        if (gcoef != A(0)) e += grad_term<A>(q, Sr, gcoef);
        Store<S>::store(pops + (size_t)q * n + c, e, scale);
    }
}

// Cells now solid are zeroed; cells the sphere uncovered are refilled
// afterwards, one at a time by their whole warp (refill_warp).  blockDim.x
// is a multiple of 32.
template <typename S>
__global__ void k_refill(S* __restrict__ pops, const uint8_t* __restrict__ fcur, const uint8_t* __restrict__ fnext,
                         GridDesc G, BoxDesc B, const ParticleState* __restrict__ ps,
                         typename Store<S>::A scale, typename Store<S>::A inv_scale, typename Store<S>::A gcoef) {
    using A = typename Store<S>::A;
    __shared__ BoxFrame F;
    const int n3[3] = {G.nx, G.ny, G.nz};
    if (threadIdx.x == 0) box_frame_init(F, n3, G.periodic, B, *ps);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n = (size_t)G.n;
    bool uncovered = false;
    int p[3] = {0, 0, 0};
    if (t < B.cells && box_cell(t, n3, G.periodic, B, F, p)) {
        const size_t c = (size_t)p[0] + (size_t)G.nx * ((size_t)p[1] + (size_t)G.ny * (size_t)p[2]);
        if (fnext[c] != 0) {
#pragma unroll
            for (int q = 0; q < 19; ++q) Store<S>::store(pops + (size_t)q * n + c, A(0), scale);
        } else {
            uncovered = fcur[c] != 0;
        }
    }
    for (unsigned todo = __ballot_sync(0xffffffffu, uncovered); todo != 0u; todo &= todo - 1u) {
        const int src = __ffs((int)todo) - 1;
        const int i = __shfl_sync(0xffffffffu, p[0], src), j = __shfl_sync(0xffffffffu, p[1], src),
                  k = __shfl_sync(0xffffffffu, p[2], src);
        const size_t c = (size_t)i + (size_t)G.nx * ((size_t)j + (size_t)G.ny * (size_t)k);
        refill_warp<S>(pops, fcur, fnext, G, n3, *ps, i, j, k, c, scale, inv_scale, gcoef);
    }
}

// Ordered compaction of the fluid cells with a solid neighbour inside the
// box, in two passes over the box: k_links_mark flags each box cell and
// counts per block; k_links_emit gives every block its offset (sum of the
// counts of the blocks before it) and writes its cells in traversal order.
// The order is the box traversal order, identical in every run.
constexpr int LINK_THREADS = 256;

__device__ __forceinline__ int wrap_idx(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__global__ void __launch_bounds__(LINK_THREADS)
    k_links_mark(const uint8_t* __restrict__ flags, GridDesc G, BoxDesc B, const ParticleState* __restrict__ ps,
                 uint8_t* __restrict__ mask, int* __restrict__ block_count) {
    __shared__ BoxFrame F;
    const int n3[3] = {G.nx, G.ny, G.nz};
    if (threadIdx.x == 0) box_frame_init(F, n3, G.periodic, B, *ps);
    __syncthreads();
    const int t = blockIdx.x * LINK_THREADS + threadIdx.x;
    int is_b = 0;
    if (t < B.cells) {
        int p[3];
        if (box_cell(t, n3, G.periodic, B, F, p)) {
            const int i = p[0], j = p[1], k = p[2];
            const int nx = G.nx, ny = G.ny;
            const int c = i + nx * (j + ny * k);
            if (flags[c] == 0) {
#pragma unroll
                for (int q = 1; q < 19; ++q) {
                    const int a = i + cx(q), b = j + cy(q), d = k + cz(q);
                    if ((!G.periodic[0] && (a < 0 || a >= nx)) || (!G.periodic[1] && (b < 0 || b >= ny)) ||
                        (!G.periodic[2] && (d < 0 || d >= G.nz)))
                        continue;
                    const int y = wrap_idx(a, nx) + nx * (wrap_idx(b, ny) + ny * wrap_idx(d, G.nz));
                    is_b |= flags[y] != 0;
                }
            }
        }
        mask[t] = (uint8_t)is_b;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, is_b);
    __shared__ int wsum[LINK_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(ballot);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < LINK_THREADS / 32; ++w) s += wsum[w];
        block_count[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(LINK_THREADS)
    k_links_emit(const uint8_t* __restrict__ mask, const int* __restrict__ block_count, GridDesc G, BoxDesc B,
                 const ParticleState* __restrict__ ps, int* __restrict__ list, int* __restrict__ count, int capacity,
                 int* __restrict__ status) {
    __shared__ int red[LINK_THREADS];
    __shared__ int wsum[LINK_THREADS / 32];
    __shared__ BoxFrame F;
    const int n3[3] = {G.nx, G.ny, G.nz};
    if (threadIdx.x == 0) box_frame_init(F, n3, G.periodic, B, *ps);
    // offset of this block: sum of the counts of all earlier blocks
    int s = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += LINK_THREADS) s += block_count[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = LINK_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    const int base = red[0];
    const int t = blockIdx.x * LINK_THREADS + threadIdx.x;
    const int is_b = (t < B.cells) ? mask[t] : 0;
    const unsigned ballot = __ballot_sync(0xffffffffu, is_b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = __popc(ballot);
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += wsum[w];
    if (is_b) {
        int p[3];
        const bool in = box_cell(t, n3, G.periodic, B, F, p);
        const int pos = base + wbase + __popc(ballot & ((1u << lane) - 1u));
        if (pos >= capacity) atomicOr(status, STATUS_LINK_OVERFLOW);
        else if (in) list[pos] = p[0] + G.nx * (p[1] + G.ny * p[2]);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        int tot = base;
        for (int w = 0; w < LINK_THREADS / 32; ++w) tot += wsum[w];
        *count = tot < capacity ? tot : capacity;
    }
}

// Link export for inspection: slot (i*18 + q-1) of the i-th boundary cell
// holds q and delta_q when x + c_q is solid, q = -1 otherwise.
__global__ void k_export_links(const uint8_t* __restrict__ flags, const int* __restrict__ list,
                               const int* __restrict__ count, GridDesc G, const ParticleState* __restrict__ ps,
                               int32_t* __restrict__ q_out, double* __restrict__ delta_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const int cell = list[i];
    const int x = cell % G.nx, y = (cell / G.nx) % G.ny, z = cell / (G.nx * G.ny);
    const ParticleState& P = *ps;
    const double d[3] = {wrap_diff((x + 0.5) - P.x[0], G.nx, G.periodic[0]),
                         wrap_diff((y + 0.5) - P.x[1], G.ny, G.periodic[1]),
                         wrap_diff((z + 0.5) - P.x[2], G.nz, G.periodic[2])};
    const int n3[3] = {G.nx, G.ny, G.nz};
    for (int q = 1; q < 19; ++q) {
        int v[3] = {x + cx(q), y + cy(q), z + cz(q)};
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            if (v[a] < 0 || v[a] >= n3[a]) {
                if (!G.periodic[a]) ok = false;
                v[a] = (v[a] + n3[a]) % n3[a];
            }
        }
        const size_t slot = (size_t)i * 18 + (q - 1);
        const size_t yy = ok ? (size_t)v[0] + (size_t)G.nx * ((size_t)v[1] + (size_t)G.ny * (size_t)v[2]) : 0;
        if (ok && flags[yy] != 0) {
            q_out[slot] = q;
            delta_out[slot] = link_delta(d, q, P.r);
        } else {
            q_out[slot] = -1;
            delta_out[slot] = 0.0;
        }
    }
}

template <typename S>
__global__ void k_init_eq(S* __restrict__ pops, const uint8_t* __restrict__ flags, GridDesc G, double rho,
                          double u0, double u1, double u2, const double* __restrict__ ufield,
                          typename Store<S>::A scale) {
    using A = typename Store<S>::A;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G.n) return;
    const size_t n = (size_t)G.n;
    const bool fluid = flags == nullptr || flags[c] == 0;
    double u[3] = {u0, u1, u2};
    if (ufield) {
        u[0] = ufield[c];
        u[1] = ufield[n + c];
        u[2] = ufield[2 * n + c];
    }
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int q = 0; q < 19; ++q) {
        const double cu = cx(q) * u[0] + cy(q) * u[1] + cz(q) * u[2];
        const double e = wgt<double>(q) * ((rho - 1.0) + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        Store<S>::store(pops + (size_t)q * n + c, fluid ? A(e) : A(0), scale);
    }
}

template <typename S>
__global__ void k_to_f64(const S* __restrict__ pops, double* __restrict__ out, long long count,
                         typename Store<S>::A inv_scale) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (double)Store<S>::load(pops + i, inv_scale);
}

template <typename S>
__global__ void k_from_f64(const double* __restrict__ in, S* __restrict__ pops, long long count,
                           typename Store<S>::A scale) {
    using A = typename Store<S>::A;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) Store<S>::store(pops + i, (A)in[i], scale);
}

template <typename S>
__global__ void k_gather(const S* __restrict__ pops, long long ncells, const int64_t* __restrict__ cells,
                         long long n, double* __restrict__ out, typename Store<S>::A inv_scale) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 19) return;
    const long long i = t / 19;
    const int q = (int)(t % 19);
    const long long c = cells[i];
    out[t] = (c >= 0 && c < ncells) ? (double)Store<S>::load(pops + (size_t)q * ncells + c, inv_scale) : 0.0;
}

template <typename S>
__global__ void k_zero_solid(S* __restrict__ pops, const uint8_t* __restrict__ flags, GridDesc G) {
    using A = typename Store<S>::A;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= G.n || flags[c] == 0) return;
    for (int q = 0; q < 19; ++q) Store<S>::store(pops + (size_t)q * G.n + c, A(0), A(1));
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------- launchers
template <typename S>
void launch_bulk(const S* src, S* dst, const GridDesc& g, const CollideParams<typename Store<S>::A>& p,
                 int* status, cudaStream_t stream) {
    int bx = 32;
    while (bx < g.nx && bx < 128) bx *= 2;
    const int by = BULK_THREADS / bx;
    dim3 block(bx, by, 1);
    dim3 grid((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, g.nz);
    const bool walls = !(g.periodic[0] && g.periodic[1] && g.periodic[2]);
    if constexpr (std::is_same<S, __half>::value) {   // FP16, unforced, whole pairs: two cells per thread
        if (!p.forced && g.nx % 2 == 0) {
            const int pairs = g.nx / 2;
            int px = 32;
            while (px < pairs && px < 128) px *= 2;
            dim3 b2(px, BULK2_THREADS / px, 1);
            dim3 g2((pairs + px - 1) / px, (g.ny + b2.y - 1) / b2.y, g.nz);
            const bool mrt = p.db != 0.0f;
            if (walls && mrt) k_bulk_h2<true, true><<<g2, b2, 0, stream>>>(src, dst, g, p, status);
            else if (walls) k_bulk_h2<true, false><<<g2, b2, 0, stream>>>(src, dst, g, p, status);
            else if (mrt) k_bulk_h2<false, true><<<g2, b2, 0, stream>>>(src, dst, g, p, status);
            else k_bulk_h2<false, false><<<g2, b2, 0, stream>>>(src, dst, g, p, status);
            return;
        }
    }
    if (walls) {
        if (p.forced) k_bulk<S, true, true><<<grid, block, 0, stream>>>(src, dst, g, p, status);
        else k_bulk<S, true, false><<<grid, block, 0, stream>>>(src, dst, g, p, status);
    } else {
        if (p.forced) k_bulk<S, false, true><<<grid, block, 0, stream>>>(src, dst, g, p, status);
        else k_bulk<S, false, false><<<grid, block, 0, stream>>>(src, dst, g, p, status);
    }
}

template <typename S>
void launch_boundary(const S* src, S* dst, const uint8_t* flags, const int* list, const int* count, int max_cells,
                     const GridDesc& g, const CollideParams<typename Store<S>::A>& p, const ParticleState* ps,
                     int cli, double* partials, int* nblocks_out, int* status, cudaStream_t stream) {
    const int nb = boundary_grid(max_cells);
    *nblocks_out = nb;
    if (p.forced)
        k_boundary<S, true><<<nb, BNDW_THREADS, 0, stream>>>(src, dst, flags, list, count, g, p, ps, cli, partials, status);
    else
        k_boundary<S, false><<<nb, BNDW_THREADS, 0, stream>>>(src, dst, flags, list, count, g, p, ps, cli, partials, status);
}

void launch_particle_update(ParticleState* ps, const double* partials, int nblocks, const GridDesc& g,
                            double* history, int hist_cap, int* status, cudaStream_t stream) {
    k_particle<<<1, PART_THREADS, 0, stream>>>(ps, partials, nblocks, g, history, hist_cap, status);
}

void launch_flags_full(uint8_t* flags, const GridDesc& g, const ParticleState* ps, cudaStream_t stream) {
    k_flags_full<<<blocks_for(g.n, 256), 256, 0, stream>>>(flags, g, ps);
}

void launch_flags_box(uint8_t* flags_next, const GridDesc& g, const BoxDesc& b, const ParticleState* ps,
                      cudaStream_t stream) {
    k_flags_box<<<blocks_for(b.cells, 256), 256, 0, stream>>>(flags_next, g, b, ps);
}

template <typename S>
void launch_refill(S* pops, const uint8_t* flags_cur, const uint8_t* flags_next, const GridDesc& g,
                   const BoxDesc& b, const ParticleState* ps, typename Store<S>::A scale,
                   typename Store<S>::A inv_scale, typename Store<S>::A gcoef, cudaStream_t stream) {
    k_refill<S><<<blocks_for(b.cells, 128), 128, 0, stream>>>(pops, flags_cur, flags_next, g, b, ps, scale,
                                                               inv_scale, gcoef);
}

void launch_build_links(const uint8_t* flags, const GridDesc& g, const BoxDesc& b, const ParticleState* ps,
                        uint8_t* mask, int* block_count, int* list, int* count, int capacity, int* status,
                        cudaStream_t stream) {
    const unsigned nb = blocks_for(b.cells, LINK_THREADS);
    k_links_mark<<<nb, LINK_THREADS, 0, stream>>>(flags, g, b, ps, mask, block_count);
    k_links_emit<<<nb, LINK_THREADS, 0, stream>>>(mask, block_count, g, b, ps, list, count, capacity, status);
}

void launch_export_links(const uint8_t* flags, const int* list, const int* count, int max_cells, const GridDesc& g,
                         const ParticleState* ps, int cli, int32_t* q_out, double* delta_out, cudaStream_t stream) {
    (void)cli;
    if (max_cells <= 0) return;
    k_export_links<<<blocks_for(max_cells, 128), 128, 0, stream>>>(flags, list, count, g, ps, q_out, delta_out);
}

template <typename S>
void launch_init_equilibrium(S* pops, const uint8_t* flags, const GridDesc& g, double rho, const double u[3],
                             const double* u_field, typename Store<S>::A scale, cudaStream_t stream) {
    k_init_eq<S><<<blocks_for(g.n, 256), 256, 0, stream>>>(pops, flags, g, rho, u[0], u[1], u[2], u_field, scale);
}

template <typename S>
void launch_to_f64(const S* pops, double* out, long long count, typename Store<S>::A inv_scale,
                   cudaStream_t stream) {
    k_to_f64<S><<<blocks_for(count, 256), 256, 0, stream>>>(pops, out, count, inv_scale);
}

template <typename S>
void launch_from_f64(const double* in, S* pops, long long count, typename Store<S>::A scale, cudaStream_t stream) {
    k_from_f64<S><<<blocks_for(count, 256), 256, 0, stream>>>(in, pops, count, scale);
}

template <typename S>
void launch_gather(const S* pops, long long ncells, const int64_t* cells, long long n, double* out,
                   typename Store<S>::A inv_scale, cudaStream_t stream) {
    if (n <= 0) return;
    k_gather<S><<<blocks_for(n * 19, 256), 256, 0, stream>>>(pops, ncells, cells, n, out, inv_scale);
}

template <typename S>
void launch_zero_solid(S* pops, const uint8_t* flags, const GridDesc& g, cudaStream_t stream) {
    k_zero_solid<S><<<blocks_for(g.n, 256), 256, 0, stream>>>(pops, flags, g);
}

#define LBMP_INSTANTIATE(S)                                                                                        \
    template void launch_bulk<S>(const S*, S*, const GridDesc&, const CollideParams<Store<S>::A>&, int*,           \
                                 cudaStream_t);                                                                    \
    template void launch_boundary<S>(const S*, S*, const uint8_t*, const int*, const int*, int, const GridDesc&,   \
                                     const CollideParams<Store<S>::A>&, const ParticleState*, int, double*, int*,  \
                                     int*, cudaStream_t);                                                          \
    template void launch_refill<S>(S*, const uint8_t*, const uint8_t*, const GridDesc&, const BoxDesc&,            \
                                   const ParticleState*, Store<S>::A, Store<S>::A, Store<S>::A, cudaStream_t);     \
    template void launch_init_equilibrium<S>(S*, const uint8_t*, const GridDesc&, double, const double*,           \
                                             const double*, Store<S>::A, cudaStream_t);                            \
    template void launch_to_f64<S>(const S*, double*, long long, Store<S>::A, cudaStream_t);                       \
    template void launch_from_f64<S>(const double*, S*, long long, Store<S>::A, cudaStream_t);                      \
    template void launch_zero_solid<S>(S*, const uint8_t*, const GridDesc&, cudaStream_t);                       \
    template void launch_gather<S>(const S*, long long, const int64_t*, long long, double*, Store<S>::A,           \
                                   cudaStream_t);

LBMP_INSTANTIATE(double)
LBMP_INSTANTIATE(float)
LBMP_INSTANTIATE(__half)

}  // namespace lbmp
