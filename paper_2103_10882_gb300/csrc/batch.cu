// Batched sweep: many independent uniform periodic simulations of uneven size
// (the paper's (density ratio, Ga) parameter study, Sec. 5) advanced together.
// Every phase of the coupled step (Algorithm 1) is one launch covering all
// simulations: stream-collide over a flat tile list, CLI/momentum-exchange
// boundary (one grid row per simulation), particle update (one CTA per
// simulation), remap.  Two steps are captured in a CUDA graph and replayed.
// The stream-collide tile shape is chosen by timing the candidates on the
// batch itself (autotuner).
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "batch.h"
#include "physics.cuh"

namespace lbmp {
namespace {

struct SimDev {
    GridDesc G;
    long long pop_off;   // element offset of the simulation in each population pool
    long long flag_off;  // byte offset in each flag pool
    int mask_off;        // boundary mask: one byte per box cell
    int bnd_off, bnd_n;  // boundary-kernel blocks of the simulation (and their force partials)
    BoxDesc box;
    double sp, sm, db;
    long long hist_off;  // records
};

constexpr int BW = 256;   // threads of the boundary, particle and remap kernels
constexpr int BND_CHUNK = 512;   // box cells per boundary block (fewer, fuller blocks: the fixed cost per block dominates)
// Cell flags: fluid, solid (centre inside the sphere), fluid with a solid
// D3Q19 neighbour (updated by k_batch_boundary instead of the bulk kernel).
constexpr uint8_t FLAG_FLUID = 0, FLAG_SOLID = 1, FLAG_BOUNDARY = 2;

template <typename S>
__host__ __device__ __forceinline__ CollideParams<typename Store<S>::A> sim_params(const SimDev& D, typename Store<S>::A scale,
                                               typename Store<S>::A inv) {
    CollideParams<typename Store<S>::A> p;
    p.sp = (typename Store<S>::A)D.sp;
    p.sm = (typename Store<S>::A)D.sm;
    p.db = (typename Store<S>::A)D.db;
    p.F[0] = p.F[1] = p.F[2] = 0;
    p.forced = 0;
    p.scale = scale;
    p.inv_scale = inv;
    return p;
}

// ------------------------------------------------------------ stream-collide
// tile = (simulation, x0, y0, z0); block (16, TY); each thread ZC cells along z.
template <typename S, int ZC>
__global__ void __launch_bounds__(512, sizeof(S) == 8 ? 1 : 3) k_batch_bulk(const S* __restrict__ src, S* __restrict__ dst,
                                                    const uint8_t* __restrict__ flags,
                                                    const int4* __restrict__ tiles, const SimDev* __restrict__ sims,
                                                    typename Store<S>::A scale, typename Store<S>::A inv,
                                                    int* __restrict__ status) {
    using A = typename Store<S>::A;
    const int4 t = tiles[blockIdx.x];
    const SimDev& D = sims[t.x];
    const CollideParams<A> P = sim_params<S>(D, scale, inv);
    const int e = D.G.nx;
    const int x = t.y + threadIdx.x, y = t.z + threadIdx.y;
    const size_t n = (size_t)D.G.n;
    const S* s0 = src + D.pop_off;
    S* d0 = dst + D.pop_off;
    const uint8_t* fl = flags + D.flag_off;
    const int xs[3] = {x + 1 < e ? x + 1 : 0, x, x > 0 ? x - 1 : e - 1};
    const int ys[3] = {y + 1 < e ? y + 1 : 0, y, y > 0 ? y - 1 : e - 1};
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const int z = t.w + threadIdx.z * ZC + k;
        const int zs[3] = {z + 1 < e ? z + 1 : 0, z, z > 0 ? z - 1 : e - 1};
        const size_t cell = (size_t)(x + e * (y + e * z));
        if (fl[cell] != FLAG_FLUID) continue;   // solid (zeroed by the remap) or done by k_batch_boundary
        A g[19];
#pragma unroll
        for (int q = 0; q < 19; ++q)
            g[q] = Store<S>::load(s0 + (size_t)q * n + (size_t)(xs[cx(q) + 1] + e * (ys[cy(q) + 1] + e * zs[cz(q) + 1])),
                                  P.inv_scale);
        trt_collide<A, false>(g, P, status);
#pragma unroll
        for (int q = 0; q < 19; ++q) Store<S>::store(d0 + (size_t)q * n + cell, g[q], P.scale);
    }
}

// ----------------------------------------------------------------- boundary
// Boundary cells of every simulation (flag 2), found from the remap's mask
// in box order: each block compacts the marked cells of its chunk of
// BND_CHUNK box cells and its warps take them in turn, lane q handling
// population q (CLI
// links, geometry in the population arithmetic, FP64 force partials), with
// a cooperative collision.  The grid is flat: block b belongs to simulation
// bnd_sim[b], which owns bnd_n blocks (a warp per 32 box cells) and as many
// partials; the last of them to finish runs that simulation's particle
// update (Algorithm 1).  The bulk kernel skips these cells, so this kernel
// runs beside it.
// Register cap of the boundary kernel (BW threads): it runs beside the bulk kernel (three CTAs of 512 threads
// at 40 registers per SM), and at its natural 122 registers a resident boundary CTA left room for one bulk CTA.
template <typename S>
constexpr int BND_MAXREG = sizeof(S) == 8 ? 128 : 64;

template <typename S>
__global__ void __maxnreg__(BND_MAXREG<S>)
    k_batch_boundary(const S* __restrict__ src, S* __restrict__ dst, const uint8_t* __restrict__ flags,
                     const uint8_t* __restrict__ mask, const SimDev* __restrict__ sims,
                     const int* __restrict__ bnd_sim, ParticleState* ps, int cli, typename Store<S>::A scale,
                     typename Store<S>::A inv, double* partials, int* done, double* __restrict__ history,
                     int hist_cap, int* __restrict__ status) {
    using A = typename Store<S>::A;
    __shared__ LinkFrame<A> Fr;
    __shared__ BoxFrame Bf;
    const int sim = bnd_sim[blockIdx.x];
    const SimDev& D = sims[sim];
    const GridDesc& G = D.G;
    const int n3[3] = {G.nx, G.ny, G.nz};
    const int per3[3] = {1, 1, 1};
    if (threadIdx.x == 0) Fr.init(ps[sim]);   // the two FP64 set-ups on two warps
    if (threadIdx.x == 32) box_frame_init(Bf, n3, per3, D.box, ps[sim]);
    __syncthreads();
    const CollideParams<A> P = sim_params<S>(D, scale, inv);
    const S* s0 = src + D.pop_off;
    S* d0 = dst + D.pop_off;
    const uint8_t* fl = flags + D.flag_off;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const size_t n = (size_t)G.n;
    __shared__ int sl[BND_CHUNK];
    const long long t0 = (long long)(blockIdx.x - D.bnd_off) * BND_CHUNK;
    const int nm = block_compact_mask(mask + D.mask_off, t0, D.box.cells, BND_CHUNK, sl);
    LinkSums<A> acc;
    for (int i = wib; i < nm; i += BW / 32) {
        int xyz[3];
        if (!box_cell((int)(t0 + sl[i]), n3, per3, D.box, Bf, xyz)) continue;   // marked cells are inside
        const int x = xyz[0], y = xyz[1], z = xyz[2];
        const size_t cell = (size_t)x + (size_t)G.nx * ((size_t)y + (size_t)G.ny * (size_t)z);
        A gq = A(0);
        if (lane < 19) {
            const int q = lane;
            const int c[3] = {cx(q), cy(q), cz(q)};
            int s3[3], f3[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                s3[a] = src_coord(xyz[a], c[a], n3[a], 1);
                f3[a] = src_coord(xyz[a], -c[a], n3[a], 1);
            }
            const size_t sidx = (size_t)s3[0] + (size_t)G.nx * ((size_t)s3[1] + (size_t)G.ny * (size_t)s3[2]);
            if (q == 0 || fl[sidx] != FLAG_SOLID) {
                gq = Store<S>::load(s0 + (size_t)q * n + sidx, P.inv_scale);
            } else {
                const int k = opp(q);
                const size_t far = (size_t)f3[0] + (size_t)G.nx * ((size_t)f3[1] + (size_t)G.ny * (size_t)f3[2]);
                const bool far_ok = fl[far] != FLAG_SOLID;
                A d[3], flk[3], tl3[3];
                int pu[3];
                Fr.offset(xyz, n3, per3, d, pu);
                const A gt_k = Store<S>::load(s0 + (size_t)k * n + cell, P.inv_scale);
                const A gt_q = Store<S>::load(s0 + (size_t)q * n + cell, P.inv_scale);
                const A gt_far = far_ok ? Store<S>::load(s0 + (size_t)k * n + far, P.inv_scale) : A(0);
                gq = cli_link<A>(q, d, cli && far_ok, gt_k, gt_q, gt_far, Fr, flk, tl3);
                acc.add(k, pu, flk, tl3);
            }
        }
        gq = warp_trt_collide<A, false>(gq, lane, P, status);
        if (lane < 19) Store<S>::store(d0 + (size_t)lane * n + cell, gq, P.scale);
    }
    block_link_sums<BW>(acc, ps[sim].x, partials + (size_t)blockIdx.x * 6);
    if (last_block_done(done + sim, D.bnd_n))
        particle_block_update<BW>(ps + sim, partials + (size_t)D.bnd_off * 6, D.bnd_n, G,
                                  history + (size_t)D.hist_off * 15, hist_cap, status);
}

// -------------------------------------------------------------------- remap
// Refill of the uncovered cell (i, j, k) = flat index c of one simulation by
// the whole warp (Sec. 2.3): lane q = 1..18 takes the periodic neighbour
// (i, j, k) + c_q, counted when it is fluid before (fc) and after (the ball
// predicate) the move, with its density 1 + sum_p g_p and momentum
// sum_p c_p g_p (for Grad's strain rate from the face neighbours).  The mean
// density and the rigid-body velocity give the equilibrium, plus Grad's
// term when grad is set; lane q < 19 writes population q.  Every lane calls
// it with the same cell.
template <typename S>
__device__ __forceinline__ void batch_refill_warp(S* __restrict__ p0, const uint8_t* __restrict__ fc, const GridDesc& G,
                                                  const int n3[3], const BoxFrame& F, const ParticleState& P, int i,
                                                  int j, int k, size_t c, typename Store<S>::A scale,
                                                  typename Store<S>::A inv, int grad, double sp) {
    using A = typename Store<S>::A;
    const int lane = threadIdx.x & 31;
    const size_t n = (size_t)G.n;
    bool ok = false;
    A r = A(0), mo[3] = {A(0), A(0), A(0)};
    if (lane >= 1 && lane < 19) {
        int v[3] = {i + cx(lane), j + cy(lane), k + cz(lane)};
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = v[a] < 0 ? v[a] + n3[a] : (v[a] >= n3[a] ? v[a] - n3[a] : v[a]);
        if (!ball_flag(v, n3, G.periodic, F, P)) {
            const size_t y = (size_t)v[0] + (size_t)G.nx * ((size_t)v[1] + (size_t)G.ny * (size_t)v[2]);
            if (fc[y] != FLAG_SOLID) {
                ok = true;
                A gp[19];
#pragma unroll
                for (int q2 = 0; q2 < 19; ++q2) gp[q2] = Store<S>::load(p0 + (size_t)q2 * n + y, inv);
                r = A(1);
#pragma unroll
                for (int q2 = 0; q2 < 19; ++q2) r += gp[q2];
#pragma unroll
                for (int q2 = 1; q2 < 19; ++q2) {
                    mo[0] += A(cx(q2)) * gp[q2];
                    mo[1] += A(cy(q2)) * gp[q2];
                    mo[2] += A(cz(q2)) * gp[q2];
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
    const double d[3] = {wrap_diff((i + 0.5) - P.x[0], G.nx, 1), wrap_diff((j + 0.5) - P.x[1], G.ny, 1),
                         wrap_diff((k + 0.5) - P.x[2], G.nz, 1)};
    const A u[3] = {A(P.u[0] + (P.w[1] * d[2] - P.w[2] * d[1])), A(P.u[1] + (P.w[2] * d[0] - P.w[0] * d[2])),
                    A(P.u[2] + (P.w[0] * d[1] - P.w[1] * d[0]))};
    const A uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    A Sr[6] = {A(0), A(0), A(0), A(0), A(0), A(0)};
    A gcoef = A(0);
    if (grad) {   // face neighbour q = 1 + 2 a (+1 for -e_a), fluid before and after the move
        gcoef = A(-3.0 * (1.0 - sp) / sp);
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
        if (grad) e += grad_term<A>(q, Sr, gcoef);
        Store<S>::store(p0 + (size_t)q * n + c, e, scale);
    }
}

// Remap of Sec. 2.3 in one pass over each simulation's box: the new flag of
// every cell (the exact ball predicate; 2 for fluid cells with a solid
// neighbour, evaluated from the same predicate), covered cells zeroed,
// uncovered cells refilled afterwards, one at a time by their whole warp
// (batch_refill_warp), and the mask of boundary cells in box order for the
// next step's k_batch_boundary.
template <typename S>
__global__ void __launch_bounds__(BW)
    k_batch_remap(S* __restrict__ pops, const uint8_t* __restrict__ fcur, uint8_t* __restrict__ fnext,
                  const SimDev* __restrict__ sims, const ParticleState* __restrict__ ps,
                  typename Store<S>::A scale, typename Store<S>::A inv, uint8_t* __restrict__ mask, int grad) {
    using A = typename Store<S>::A;
    __shared__ BoxFrame F;
    const int sim = blockIdx.y;
    const SimDev& D = sims[sim];
    const GridDesc& G = D.G;
    if ((long long)blockIdx.x * BW >= D.box.cells) return;   // uniform across the block
    const int n3[3] = {G.nx, G.ny, G.nz};
    if (threadIdx.x == 0) box_frame_init(F, n3, G.periodic, D.box, ps[sim]);
    __syncthreads();
    const int t = blockIdx.x * BW + threadIdx.x;
    const ParticleState& P = ps[sim];
    const uint8_t* fc = fcur + D.flag_off;
    uint8_t* fn = fnext + D.flag_off;
    S* p0 = pops + D.pop_off;
    const size_t n = (size_t)G.n;
    bool uncovered = false;   // fluid after the move, solid before: refilled below by the warp
    int p[3] = {0, 0, 0};
    size_t c = 0;
    // periodic: box_cell fails only for a corrupt centre
    if (t < D.box.cells && box_cell(t, n3, G.periodic, D.box, F, p)) {
        c = (size_t)p[0] + (size_t)G.nx * ((size_t)p[1] + (size_t)G.ny * (size_t)p[2]);
        int is_b = 0;
        bool any_nb = false;
        if (ball_flag_and_neighbours(p, n3, G.periodic, F, P, &any_nb)) {
            fn[c] = FLAG_SOLID;
            for (int q = 0; q < 19; ++q) Store<S>::store(p0 + (size_t)q * n + c, A(0), scale);
        } else {
            uncovered = fc[c] == FLAG_SOLID;
            is_b = any_nb ? 1 : 0;
            fn[c] = is_b ? FLAG_BOUNDARY : FLAG_FLUID;
        }
        mask[D.mask_off + t] = (uint8_t)is_b;
    }
    for (unsigned todo = __ballot_sync(0xffffffffu, uncovered); todo != 0u; todo &= todo - 1u) {
        const int src = __ffs((int)todo) - 1;
        const int i = __shfl_sync(0xffffffffu, p[0], src), j = __shfl_sync(0xffffffffu, p[1], src),
                  k = __shfl_sync(0xffffffffu, p[2], src);
        const size_t cc = (size_t)i + (size_t)G.nx * ((size_t)j + (size_t)G.ny * (size_t)k);
        batch_refill_warp<S>(p0, fc, G, n3, F, P, i, j, k, cc, scale, inv, grad, D.sp);
    }
}

template <typename S>
__global__ void k_batch_init(S* __restrict__ pops, const uint8_t* __restrict__ flags, const SimDev* __restrict__ sims,
                             const long long* __restrict__ cell_off, int nsims, long long total,
                             typename Store<S>::A scale) {
    using A = typename Store<S>::A;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int sim = 0;
    while (sim + 1 < nsims && cell_off[sim + 1] <= g) ++sim;
    const SimDev& D = sims[sim];
    const long long c = g - cell_off[sim];
    for (int q = 0; q < 19; ++q) Store<S>::store(pops + D.pop_off + (size_t)q * D.G.n + c, A(0), scale);
    (void)flags;
}

__global__ void k_batch_flags_full(uint8_t* __restrict__ f0, uint8_t* __restrict__ f1, const SimDev* __restrict__ sims,
                                   const ParticleState* __restrict__ ps, const long long* __restrict__ cell_off,
                                   int nsims, long long total) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int sim = 0;
    while (sim + 1 < nsims && cell_off[sim + 1] <= g) ++sim;
    const SimDev& D = sims[sim];
    const int c = (int)(g - cell_off[sim]);
    const int e = D.G.nx;
    const uint8_t v = inside_ball(c % e, (c / e) % e, c / (e * e), D.G, ps[sim]) ? 1 : 0;
    f0[D.flag_off + c] = v;
    f1[D.flag_off + c] = v;
}

// Initial boundary-cell lists (uses the refill/mark kernel on unchanged flags).
template <typename S>
__global__ void k_batch_to_f64(const S* __restrict__ pops, double* __restrict__ out, long long count,
                               typename Store<S>::A inv) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (double)Store<S>::load(pops + i, inv);
}

struct Tile {
    int threads_y, zc;
};

}  // namespace

// =================================================================== engine
struct BatchEngine {
    int nsims = 0;
    std::vector<SimDev> sims;
    SimDev* d_sims = nullptr;
    long long total_cells = 0;
    std::vector<long long> cell_off;
    long long* d_cell_off = nullptr;
    void* pops[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t* flags[2] = {nullptr, nullptr};
    int fcur = 0;
    ParticleState* d_ps = nullptr;
    std::vector<ParticleState> h_ps;
    uint8_t* mask = nullptr;
    int* done = nullptr;        // last-block-done counter per simulation
    double* partials = nullptr;
    int bnd_blocks = 1;     // boundary-kernel blocks of all simulations
    int* d_bnd_sim = nullptr;   // simulation of each boundary-kernel block
    int max_box_blocks = 1;
    double* history = nullptr;
    // stream-collide tiles for every candidate shape
    int4* d_tiles[4] = {nullptr, nullptr, nullptr, nullptr};
    int ntiles[4] = {0, 0, 0, 0};
    int tile_choice = 1;
    float tile_ms[4] = {0, 0, 0, 0};
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture_stream = nullptr;
    long long graph_launches = 0;
    cudaStream_t side = nullptr;               // k_batch_boundary runs here, beside the bulk kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

const Tile TILES[4] = {{8, 1}, {16, 1}, {8, 2}, {16, 2}};   // block (16, threads_y, 1), zc cells per thread

template <typename F>
void with_storage_batch(int prec, F&& f) {
    if (prec == LBMP_FP64) f((double*)nullptr);
    else if (prec == LBMP_FP32) f((float*)nullptr);
    else f((__half*)nullptr);
}

template <typename S>
void batch_scales(const lbmp_handle* h, typename Store<S>::A* scale, typename Store<S>::A* inv) {
    const bool f16 = h->cfg.precision == LBMP_FP16;
    *scale = (typename Store<S>::A)(f16 ? std::ldexp(1.0, h->cfg.fp16_scale_log2) : 1.0);
    *inv = (typename Store<S>::A)(f16 ? std::ldexp(1.0, -h->cfg.fp16_scale_log2) : 1.0);
}

template <typename S>
void launch_bulk_choice(lbmp_handle* h, BatchEngine* B, int choice, const S* src, S* dst) {
    using A = typename Store<S>::A;
    A scale, inv;
    batch_scales<S>(h, &scale, &inv);
    const Tile t = TILES[choice];
    const dim3 block(16, t.threads_y, 1);
    if (t.zc == 1)
        k_batch_bulk<S, 1><<<B->ntiles[choice], block, 0, h->stream>>>(src, dst, B->flags[B->fcur], B->d_tiles[choice], B->d_sims, scale,
                                                                       inv, h->status);
    else
        k_batch_bulk<S, 2><<<B->ntiles[choice], block, 0, h->stream>>>(src, dst, B->flags[B->fcur], B->d_tiles[choice], B->d_sims, scale,
                                                                       inv, h->status);
}

template <typename S>
void enqueue_batch_step(lbmp_handle* h) {
    using A = typename Store<S>::A;
    BatchEngine* B = h->batch;
    A scale, inv;
    batch_scales<S>(h, &scale, &inv);
    const S* src = (const S*)B->pops[B->cur];
    S* dst = (S*)B->pops[1 - B->cur];
    // boundary cells (flag 2) and the particle updates beside the bulk kernel, which skips them
    cudaEventRecord(B->ev_fork, h->stream);
    cudaStreamWaitEvent(B->side, B->ev_fork, 0);
    k_batch_boundary<S><<<B->bnd_blocks, BW, 0, B->side>>>(src, dst, B->flags[B->fcur], B->mask, B->d_sims,
                                                           B->d_bnd_sim, B->d_ps, h->cfg.boundary == LBMP_CLI ? 1 : 0,
                                                           scale, inv, B->partials, B->done, B->history,
                                                           h->cfg.history_capacity, h->status);
    cudaEventRecord(B->ev_join, B->side);
    const long long ev = profile_mark(h);
    launch_bulk_choice<S>(h, B, B->tile_choice, src, dst);
    profile_kernel(h, ev, profile_mark(h), 38.0 * sizeof(S) * (double)B->total_cells, (double)B->total_cells);
    cudaStreamWaitEvent(h->stream, B->ev_join, 0);
    uint8_t* fnext = B->flags[1 - B->fcur];
    const dim3 gr(B->max_box_blocks, B->nsims);
    k_batch_remap<S><<<gr, BW, 0, h->stream>>>(dst, B->flags[B->fcur], fnext, B->d_sims, B->d_ps, scale, inv, B->mask,
                                               h->cfg.refill == LBMP_REFILL_GRAD ? 1 : 0);
    B->cur = 1 - B->cur;
    B->fcur = 1 - B->fcur;
    h->launches += 3;
    h->updates += B->total_cells;
}

}  // namespace

void batch_destroy(lbmp_handle* h) {
    BatchEngine* B = h->batch;
    if (!B) return;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    if (B->capture_stream) cudaStreamDestroy(B->capture_stream);
    if (B->side) cudaStreamDestroy(B->side);
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    if (B->ev_join) cudaEventDestroy(B->ev_join);
    delete B;
    h->batch = nullptr;   // device memory is released with the handle's allocations
}

lbmp_status batch_create(lbmp_handle* h, const lbmp_batch_sim* sims, int n) {
    BatchEngine* B = new (std::nothrow) BatchEngine();
    if (!B) return LBMP_ERR_OOM;
    h->batch = B;
    B->nsims = n;
    B->sims.resize(n);
    B->h_ps.resize(n);
    B->cell_off.resize(n + 1, 0);
    const size_t es = h->cfg.precision == LBMP_FP64 ? 8 : (h->cfg.precision == LBMP_FP32 ? 4 : 2);
    long long cells = 0, mask_total = 0;
    int max_box = 1;
    std::vector<int> bnd_sim;
    for (int s = 0; s < n; ++s) {
        const lbmp_batch_sim& in = sims[s];
        SimDev& D = B->sims[s];
        D.G.nx = D.G.ny = D.G.nz = in.edge;
        D.G.periodic[0] = D.G.periodic[1] = D.G.periodic[2] = 1;
        D.G.n = (long long)in.edge * in.edge * in.edge;
        D.pop_off = 19 * cells;
        D.flag_off = cells;
        B->cell_off[s] = cells;
        cells += D.G.n;
        const double sp = 1.0 / in.tau, sm = 1.0 / (0.5 + h->cfg.magic / (in.tau - 0.5));
        D.sp = sp;
        D.sm = sm;
        D.db = bulk_rate_offset(in.tau, h->cfg.bulk_factor);
        ParticleState& P = B->h_ps[s];
        std::memset(&P, 0, sizeof(P));
        for (int a = 0; a < 3; ++a) {
            P.x[a] = in.pos[a];
            P.g[a] = in.gravity[a];
        }
        P.D = in.diameter;
        P.r = 0.5 * in.diameter;
        P.rho_p = in.density_ratio;
        P.cv = in.cv;
        P.cvw = in.cv_omega;
        P.V = M_PI * in.diameter * in.diameter * in.diameter / 6.0;
        P.present = 1;
        P.force_average = h->cfg.force_average ? 1 : 0;
        BoxDesc& X = D.box;
        X.R = (int)std::ceil(P.r) + 3;
        X.cells = 1;
        for (int a = 0; a < 3; ++a) {
            X.E[a] = 2 * X.R + 2;
            if (X.E[a] >= in.edge) X.E[a] = in.edge;
            X.cells *= X.E[a];
        }
        D.mask_off = (int)mask_total;
        mask_total += X.cells;
        const int nbx = (int)((X.cells + BW - 1) / BW);
        max_box = std::max(max_box, nbx);
        D.bnd_off = (int)bnd_sim.size();
        D.bnd_n = (int)((X.cells + BND_CHUNK - 1) / BND_CHUNK);
        for (int j = 0; j < D.bnd_n; ++j) bnd_sim.push_back(s);
        D.hist_off = (long long)s * std::max(1, h->cfg.history_capacity);
    }
    B->cell_off[n] = cells;
    B->total_cells = cells;
    B->max_box_blocks = max_box;
    B->bnd_blocks = (int)bnd_sim.size();
    const size_t pop_bytes = es * 19 * (size_t)cells;
    B->pops[0] = handle_alloc(h, pop_bytes);
    B->pops[1] = handle_alloc(h, pop_bytes);
    B->flags[0] = (uint8_t*)handle_alloc(h, (size_t)cells);
    B->flags[1] = (uint8_t*)handle_alloc(h, (size_t)cells);
    B->d_sims = (SimDev*)handle_alloc(h, sizeof(SimDev) * n);
    B->d_cell_off = (long long*)handle_alloc(h, sizeof(long long) * (n + 1));
    B->d_ps = (ParticleState*)handle_alloc(h, sizeof(ParticleState) * n);
    B->mask = (uint8_t*)handle_alloc(h, (size_t)mask_total);
    B->done = (int*)handle_alloc(h, sizeof(int) * n);
    B->partials = (double*)handle_alloc(h, sizeof(double) * 6 * (size_t)B->bnd_blocks);
    B->d_bnd_sim = (int*)handle_alloc(h, sizeof(int) * (size_t)B->bnd_blocks);
    B->history = (double*)handle_alloc(h, sizeof(double) * 15 * (size_t)n * std::max(1, h->cfg.history_capacity));
    if (!B->pops[0] || !B->pops[1] || !B->flags[0] || !B->flags[1] || !B->d_sims || !B->d_cell_off || !B->d_ps ||
        !B->mask || !B->done || !B->partials || !B->d_bnd_sim || !B->history)
        return LBMP_ERR_OOM;
    if (cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return LBMP_ERR_CUDA;
    cudaMemcpyAsync(B->d_bnd_sim, bnd_sim.data(), sizeof(int) * bnd_sim.size(), cudaMemcpyHostToDevice, h->stream);
    // stream-collide tiles for every candidate shape (edges are multiples of 16)
    for (int c = 0; c < 4; ++c) {
        std::vector<int4> tiles;
        const int ty = TILES[c].threads_y, zc = TILES[c].zc;
        for (int s = 0; s < n; ++s) {
            const int e = B->sims[s].G.nx;
            for (int z = 0; z < e; z += zc)
                for (int y = 0; y < e; y += ty)
                    for (int x = 0; x < e; x += 16) tiles.push_back(make_int4(s, x, y, z));
        }
        B->ntiles[c] = (int)tiles.size();
        B->d_tiles[c] = (int4*)handle_alloc(h, sizeof(int4) * tiles.size());
        if (!B->d_tiles[c]) return LBMP_ERR_OOM;
        cudaMemcpyAsync(B->d_tiles[c], tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, h->stream);
    }
    cudaMemcpyAsync(B->d_sims, B->sims.data(), sizeof(SimDev) * n, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(B->d_cell_off, B->cell_off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(B->d_ps, B->h_ps.data(), sizeof(ParticleState) * n, cudaMemcpyHostToDevice, h->stream);
    cudaMemsetAsync(B->pops[0], 0, pop_bytes, h->stream);
    cudaMemsetAsync(B->pops[1], 0, pop_bytes, h->stream);
    cudaMemsetAsync(B->done, 0, sizeof(int) * n, h->stream);
    // flags, zero solid (fluid at rest everywhere else), initial boundary lists
    const unsigned gcells = (unsigned)((cells + 255) / 256);
    k_batch_flags_full<<<gcells, 256, 0, h->stream>>>(B->flags[0], B->flags[1], B->d_sims, B->d_ps, B->d_cell_off, n,
                                                       cells);
    with_storage_batch(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using A = typename Store<S>::A;
        A scale, inv;
        batch_scales<S>(h, &scale, &inv);
        // boundary flags and mask of the start position (both flag buffers hold its solid cells)
        const dim3 gr(B->max_box_blocks, B->nsims);
        k_batch_remap<S><<<gr, BW, 0, h->stream>>>((S*)B->pops[0], B->flags[1], B->flags[0], B->d_sims, B->d_ps,
                                                   scale, inv, B->mask, 0);   // nothing is uncovered here
    });
    h->h2d += (long long)(sizeof(SimDev) + sizeof(ParticleState) + sizeof(long long)) * n +
              (long long)(sizeof(int) * bnd_sim.size());
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) return LBMP_ERR_CUDA;
    h->has_particle = true;
    return LBMP_OK;
}

lbmp_status batch_autotune(lbmp_handle* h, int reps) {
    BatchEngine* B = h->batch;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return LBMP_ERR_CUDA;
    float best = 1e30f;
    with_storage_batch(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        // candidates read the current field and write the other buffer, which
        // the next step overwrites: the simulation state is not advanced
        const S* src = (const S*)B->pops[B->cur];
        S* dst = (S*)B->pops[1 - B->cur];
        for (int c = 0; c < 4; ++c) {
            launch_bulk_choice<S>(h, B, c, src, dst);   // warm-up
            cudaEventRecord(a, h->stream);
            for (int r = 0; r < reps; ++r) launch_bulk_choice<S>(h, B, c, src, dst);
            cudaEventRecord(b, h->stream);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            B->tile_ms[c] = ms / reps;
            if (B->tile_ms[c] < best) {
                best = B->tile_ms[c];
                B->tile_choice = c;
            }
        }
    });
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return cudaGetLastError() == cudaSuccess ? LBMP_OK : LBMP_ERR_CUDA;
}

lbmp_status batch_step(lbmp_handle* h, int n) {
    BatchEngine* B = h->batch;
    auto one = [&]() {
        with_storage_batch(h->cfg.precision, [&](auto tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            enqueue_batch_step<S>(h);
        });
        h->steps += 1;
    };
    int i = 0;
    while (i < n) {
        // the captured graph holds two steps starting from buffer 0
        if (h->profiling || n - i < 2 || B->cur != 0 || B->fcur != 0) {
            one();
            ++i;
            continue;
        }
        if (!B->graph) {
            if (!B->capture_stream && cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
                return LBMP_ERR_CUDA;
            cudaStream_t user = h->stream;
            const long long l0 = h->launches, u0 = h->updates;
            h->stream = B->capture_stream;
            if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                h->stream = user;
                return LBMP_ERR_CUDA;
            }
            with_storage_batch(h->cfg.precision, [&](auto tag) {
                using S = std::remove_pointer_t<decltype(tag)>;
                enqueue_batch_step<S>(h);
                enqueue_batch_step<S>(h);
            });
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
            h->stream = user;
            if (e != cudaSuccess) return LBMP_ERR_CUDA;
            const cudaError_t e2 = cudaGraphInstantiate(&B->graph, g, 0);
            cudaGraphDestroy(g);
            if (e2 != cudaSuccess) return LBMP_ERR_CUDA;
            B->graph_launches = h->launches - l0;
            h->launches = l0;
            h->updates = u0;
        }
        if (cudaGraphLaunch(B->graph, h->stream) != cudaSuccess) return LBMP_ERR_CUDA;
        h->launches += B->graph_launches;
        h->updates += 2 * B->total_cells;
        h->steps += 2;
        i += 2;
    }
    return cudaGetLastError() == cudaSuccess ? LBMP_OK : LBMP_ERR_CUDA;
}

lbmp_status batch_get_particle(lbmp_handle* h, int sim, ParticleState* out) {
    BatchEngine* B = h->batch;
    if (sim < 0 || sim >= B->nsims) return LBMP_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(out, B->d_ps + sim, sizeof(ParticleState), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return LBMP_ERR_CUDA;
    h->d2h += sizeof(ParticleState);
    return LBMP_OK;
}

lbmp_status batch_set_particle(lbmp_handle* h, int sim, const ParticleState* in) {
    BatchEngine* B = h->batch;
    if (sim < 0 || sim >= B->nsims) return LBMP_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(B->d_ps + sim, in, sizeof(ParticleState), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return LBMP_ERR_CUDA;
    h->h2d += sizeof(ParticleState);
    return LBMP_OK;
}

lbmp_status batch_history(lbmp_handle* h, int sim, double* ring, int cap) {
    BatchEngine* B = h->batch;
    if (sim < 0 || sim >= B->nsims) return LBMP_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(ring, B->history + (size_t)B->sims[sim].hist_off * 15, sizeof(double) * 15 * (size_t)cap,
                        cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return LBMP_ERR_CUDA;
    h->d2h += (long long)sizeof(double) * 15 * cap;
    return LBMP_OK;
}

lbmp_status batch_populations(lbmp_handle* h, int sim, double* out, size_t cap) {
    BatchEngine* B = h->batch;
    if (sim < 0 || sim >= B->nsims) return LBMP_ERR_INVALID_ARG;
    const SimDev& D = B->sims[sim];
    const long long count = 19 * D.G.n;
    if ((long long)cap < count) return LBMP_ERR_INVALID_ARG;
    double* tmp = (double*)handle_alloc(h, sizeof(double) * (size_t)count);
    if (!tmp) return LBMP_ERR_OOM;
    with_storage_batch(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using A = typename Store<S>::A;
        A scale, inv;
        batch_scales<S>(h, &scale, &inv);
        k_batch_to_f64<S><<<(unsigned)((count + 255) / 256), 256, 0, h->stream>>>((const S*)B->pops[B->cur] + D.pop_off,
                                                                                  tmp, count, inv);
    });
    cudaError_t e = cudaMemcpyAsync(out, tmp, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->d2h += (long long)sizeof(double) * count;
    handle_free(h, tmp);
    return e == cudaSuccess ? LBMP_OK : LBMP_ERR_CUDA;
}

void batch_info(const lbmp_handle* h, int64_t out[8]) {
    const BatchEngine* B = h->batch;
    out[0] = B->nsims;
    out[1] = B->total_cells;
    out[2] = 16 * TILES[B->tile_choice].threads_y;
    out[3] = TILES[B->tile_choice].zc;
    for (int c = 0; c < 4; ++c) out[4 + c] = (int64_t)(B->tile_ms[c] * 1e6);   // ns per launch
}

}  // namespace lbmp
