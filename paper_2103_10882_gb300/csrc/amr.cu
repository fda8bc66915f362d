// Refined-grid engine: block-structured levels (Sec. 4.1) with the particle
// refinement criterion (Sec. 4.2.1) and the coupling of Algorithm 1 on the
// finest level.
//
// Levels l = 0..L-1 (L-1 finest) are sets of 16^3-cell blocks; a level-(l+1)
// cell is half a level-l cell.  Each level keeps its real blocks and its
// ghost blocks (cells of the next coarser level seen at this level's
// resolution) in one pool, real blocks first, both in block-position order.
// One level-l step (recursive, finer levels sub-cycled twice, Rohde's scheme
// named in Sec. 4.1):
//   explosion   active ghost cells of level l+1 <- post-collision level-l
//               cell containing them (into the buffer of the first sub-step):
//               written by level l+1's previous last sub-step, which forms
//               those values; k_explode only after a change outside a step
//   (two level-(l+1) steps)
//   k_update    real level-l cells but the hosts: pull from real/ghost
//               neighbours, then TRT collide.  Active ghost cells stream
//               without colliding; at level l+1's last sub-step they form
//               the hosts' populations (the mean of their eight sub-cells,
//               coalescence) and collide them.  The static ghost cells beyond
//               them stand for coarse content translating rigidly and are read
//               from the coarse level, not stored.  Level l's update runs on
//               its own stream beside level l+1's sub-steps.
//   finest level: k_amr_boundary (CLI links + momentum-exchange partials),
//               particle update, remap (flags, refill, boundary cells).
// The layout (which blocks exist at which level) is integer work done on the
// host from the particle position; per-cell classifications and all
// population work run in the kernels below.
#include <cuda_fp16.h>

#include <algorithm>
#include <new>
#include <type_traits>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "amr.h"
#include "physics.cuh"

namespace lbmp {
namespace {

constexpr int BS = 16;
constexpr int B3 = BS * BS * BS;
constexpr int MAXL = 6;
// Level update CTAs: half a z-slice of a block each (128 cells); the short launches of the finer
// levels end in smaller waves than with whole slices.  10 resident CTAs per SM asked of the
// compiler (48 registers): 3% shorter launches than 12 (40 registers, spills in the ghost lanes),
// the same step time; 16 was 10% slower.
constexpr int UPD_THREADS = 128;
constexpr int UPD_MIN_CTAS = 10;     // FP32/FP16 arithmetic
constexpr int STATUS_AMR_MISSING = 8;    // a pull found no source cell
// Finest-level cell flags: fluid, solid (centre inside the sphere), and
// fluid with a solid D3Q19 neighbour (updated by k_amr_boundary).
constexpr uint8_t FLAG_FLUID = 0, FLAG_SOLID = 1, FLAG_BOUNDARY = 2;
constexpr int STATUS_NOT_FINEST = 16;    // the sphere's box left the finest level

// Device view of one level.
struct LevelView {
    int n[3];          // cells across the domain
    int nb[3];         // block positions
    int nreal, npool;
    int periodic[3];
    const int* map;        // block position -> real id, -2 - ghost id, -1 none
    const int* bpos;       // [npool][3]
    const int* nbr;        // [npool][27] pool ids of neighbour blocks, -1 none, -2 wall
    const uint8_t* host;   // [nreal][B3] 1 host, 2 second ring (levels below the finest)
    const uint8_t* refined;  // block positions covered by the next finer level
};

__device__ __forceinline__ bool wrap3(int c[3], const LevelView& V) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= V.n[a]) {
            if (!V.periodic[a]) return false;
            c[a] = c[a] < 0 ? c[a] + V.n[a] : c[a] - V.n[a];
        }
    }
    return true;
}

// Pool block (or -1) and local index of wrapped global level coordinates.
__device__ __forceinline__ int locate(const LevelView& V, const int c[3], int* cell) {
    const int m = V.map[(c[0] >> 4) + V.nb[0] * ((c[1] >> 4) + V.nb[1] * (c[2] >> 4))];
    *cell = (c[0] & 15) + BS * ((c[1] & 15) + BS * (c[2] & 15));
    if (m >= 0) return m;
    if (m <= -2) return V.nreal + (-2 - m);
    return -1;
}

__device__ __forceinline__ size_t paddr(int b, int q, int c) { return ((size_t)b * 19 + q) * B3 + c; }

template <typename A>
__device__ __forceinline__ A geq_dev(int q, A drho, const A u[3], A uu) {
    const A cu = A(cx(q)) * u[0] + A(cy(q)) * u[1] + A(cz(q)) * u[2];
    return wgt<A>(q) * (drho + A(3) * cu + A(4.5) * cu * cu - A(1.5) * uu);
}

// f = f_eq + kappa+ (f+ - f_eq+) + kappa- (f- - f_eq-), equilibrium from f's own moments.
template <typename A>
__device__ __forceinline__ void rescale19(A f[19], A kp, A km) {
    A drho = A(0), u[3] = {A(0), A(0), A(0)};
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        drho += f[q];
        u[0] += A(cx(q)) * f[q];
        u[1] += A(cy(q)) * f[q];
        u[2] += A(cz(q)) * f[q];
    }
    const A uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const A e0 = geq_dev<A>(0, drho, u, uu);
    f[0] = e0 + kp * (f[0] - e0);
#pragma unroll
    for (int q = 1; q < 19; q += 2) {
        const A eq = geq_dev<A>(q, drho, u, uu), eb = geq_dev<A>(q + 1, drho, u, uu);
        const A ep = A(0.5) * (eq + eb), em = A(0.5) * (eq - eb);
        const A fp = A(0.5) * (f[q] + f[q + 1]), fm = A(0.5) * (f[q] - f[q + 1]);
        f[q] = ep + kp * (fp - ep) + em + km * (fm - em);
        f[q + 1] = ep + kp * (fp - ep) - em - km * (fm - em);
    }
}

// Pool block of the neighbour of (b, local l) displaced by d (|d| <= 1 per
// axis), with the local index; -2 wall, -1 none.
__device__ __forceinline__ int nbr_cell(const LevelView& D, int b, int lx, int ly, int lz, int dx, int dy, int dz,
                                        int* cell) {
    const int sx = lx + dx, sy = ly + dy, sz = lz + dz;
    const int ox = sx < 0 ? -1 : (sx > 15 ? 1 : 0);
    const int oy = sy < 0 ? -1 : (sy > 15 ? 1 : 0);
    const int oz = sz < 0 ? -1 : (sz > 15 ? 1 : 0);
    *cell = (sx & 15) + BS * ((sy & 15) + BS * (sz & 15));
    return (ox | oy | oz) == 0 ? b : D.nbr[b * 27 + (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
}

// --------------------------------------------------------------- explosion
// Explosion for one coarse step of level l: every active ghost cell of level
// l+1 (list: pool block << 12 | cell, eight consecutive entries per host)
// takes the post-collision populations of its host, the level-l cell that
// contains it (hosts: real block << 12 | cell, one per eight entries), into
// f0, the source of the first sub-step.  No rescaling: the 1.5-fine-cell
// offset between the coarse centre and the first fine cell supplies the
// level change of the non-equilibrium part (Chapman-Enskog; only cells that
// change level in a regrid are rescaled, in k_migrate).
template <typename S>
__global__ void __launch_bounds__(UPD_THREADS)
    k_explode(const S* __restrict__ csrc, S* __restrict__ f0, const int* __restrict__ list,
              const int* __restrict__ hosts, int n) {
    const int i = blockIdx.x * UPD_THREADS + threadIdx.x;
    if (i >= n) return;
    const int e = list[i];
    const int b = e >> 12;
    const int c = e & 4095;
    const int hp = hosts[i >> 3];
    const int pb = hp >> 12, pc = hp & 4095;
    S f[19];   // a copy of the stored values
#pragma unroll
    for (int q = 0; q < 19; ++q) f[q] = csrc[paddr(pb, q, pc)];
#pragma unroll
    for (int q = 0; q < 19; ++q) f0[paddr(b, q, c)] = f[q];
}

// ----------------------------------------------------------------- update
template <typename S>
struct UpdateArgs {
    using A = typename Store<S>::A;
    LevelView D;
    const S* src;
    S* dst;
    CollideParams<A> P;
    // levels with a coarser level C: its post-collision populations of the
    // current coarse step (csrc, read for static ghost neighbours), per group
    // of eight active ghost cells their host (real block << 12 | cell of C),
    // per active ghost cell the mask of populations whose upwind neighbour is
    // a static ghost cell; at the last sub-step also C's destination buffer
    // and collision parameters, for the hosts (coalescence)
    LevelView C;
    const S* csrc;
    const int* ghost_host;
    const uint32_t* smask;
    S* cdst;
    CollideParams<A> Pc;
    const uint8_t* solid;     // finest level with a sphere: solid flags of real cells
    int* status;
};

// Where an active ghost cell finds a static ghost cell upwind.  Static ghost
// cells (the sub-cells of the second ring of coarse cells) hold the exploded
// coarse values at the first sub-step and stream rigidly, without
// colliding, into the second, so each of their values is that of a coarse
// cell, which the pull reads directly: with P the host of the active cell x
// and s in {0,1}^3 its sub-cell offset, the coarse cell containing x - c_q
// is P + o, o_a = s_a - 1 for c_a = 1, s_a for c_a = -1, 0 for c_a = 0
// (first sub-step); at the second sub-step the static cell has carried the
// content of the coarse cell containing x - 2 c_q, which is P - c_q, or
// kept its own (P + o) where that lies beyond a wall.
struct GhostPull {
    uint32_t smask;   // bit q: the upwind neighbour x - c_q is a static ghost cell
    int hb, hc;       // the host P: real block and cell of the coarser level
    int sub;          // sub-cell offset s = (sub & 1, (sub >> 1) & 1, sub >> 2)
    bool second;      // the level's second sub-step
};

// Pull of the 19 populations of cell (b, c) into g, as stored (FP16: the
// scaled values g * 2^s, which the collision takes in its SCALED form).  nb27 lists the pool
// ids of block b's 26 neighbours (and itself at index 13).  GHOST: (b, c) is
// an active ghost cell and gp says where static ghost cells lie upwind.
// Returns whether a source was missing (no block), which the caller reports.
template <typename S, bool GHOST = false>
__device__ __forceinline__ bool pull_cell(const UpdateArgs<S>& U, int b, int c, const int* nb27,
                                          typename Store<S>::A g[19], GhostPull gp = GhostPull{}) {
    using A = typename Store<S>::A;
    const int lx = c & 15, ly = (c >> 4) & 15, lz = c >> 8;
    // source x - c_q per axis, indexed by 1 - c: block shift and local coordinate.
    // Every population is one load: from the neighbouring cell (real or
    // ghost), or at a domain wall (-2) the cell's own opposite population
    // (bounce-back).  No block (-1) is an error: the value is 0 and the
    // status word says so.
    const int bsx[3] = {lx == 0 ? -1 : 0, 0, lx == 15 ? 1 : 0};
    const int bsy[3] = {ly == 0 ? -1 : 0, 0, ly == 15 ? 1 : 0};
    const int bsz[3] = {lz == 0 ? -1 : 0, 0, lz == 15 ? 1 : 0};
    const int lsx[3] = {(lx - 1) & 15, lx, (lx + 1) & 15};
    const int lsy[3] = {((ly - 1) & 15) * BS, ly * BS, ((ly + 1) & 15) * BS};
    const int lsz[3] = {((lz - 1) & 15) * BS * BS, lz * BS * BS, ((lz + 1) & 15) * BS * BS};
    bool missing = false;
#pragma unroll
    for (int q = 0; q < 19; ++q) {
        const int ix = 1 - cx(q), iy = 1 - cy(q), iz = 1 - cz(q);
        const int nbk = nb27[13 + bsx[ix] + 3 * bsy[iy] + 9 * bsz[iz]];   // entry 13 is b itself
        const bool own = nbk < 0;
        const int sb = own ? b : nbk, sq = own ? opp(q) : q;
        const int sc = own ? c : lsx[ix] + lsy[iy] + lsz[iz];
        const S* src = U.src + (unsigned)((sb * 19 + sq) * B3 + sc);   // pools hold < 2^31 elements
        bool lost = nbk == -1;
        if (GHOST && q > 0 && ((gp.smask >> q) & 1u)) {   // static ghost upwind: its coarse cell
            const int hx = gp.hc & 15, hy = (gp.hc >> 4) & 15, hz = gp.hc >> 8;
            const int ox = cx(q) == 1 ? (gp.sub & 1) - 1 : (cx(q) == -1 ? (gp.sub & 1) : 0);
            const int oy = cy(q) == 1 ? ((gp.sub >> 1) & 1) - 1 : (cy(q) == -1 ? ((gp.sub >> 1) & 1) : 0);
            const int oz = cz(q) == 1 ? (gp.sub >> 2) - 1 : (cz(q) == -1 ? (gp.sub >> 2) : 0);
            int cc;
            int cb = gp.second ? nbr_cell(U.C, gp.hb, hx, hy, hz, -cx(q), -cy(q), -cz(q), &cc) : -2;
            if (cb == -2) cb = nbr_cell(U.C, gp.hb, hx, hy, hz, ox, oy, oz, &cc);
            lost = cb < 0;
            src = U.csrc + (unsigned)(((lost ? 0 : cb) * 19 + q) * B3 + cc);
        }
        const A v = Store<S>::load_raw(src);
        missing |= lost;
        g[q] = lost ? A(0) : v;
    }
    return missing;
}


// One launch per level step: the first gblocks CTAs stream the active ghost
// cells of the level (glist: pool block << 12 | cell, eight consecutive
// entries per host cell of the coarser level), no collision.  At the first
// sub-step they store them into dst.  At the last sub-step they sum each
// host's eight in a fixed shuffle tree instead; all eight lanes take the
// mean as the host's populations (coalescence) and collide them with the
// coarser level's parameters; the first writes the host into the coarser
// level's destination buffer (the step of the coarser level that its own
// update, which skips hosts, is taking beside), and each writes the result
// into its own ghost cell of dst, the source of the level's next first
// sub-step: the explosion of the host's new post-collision state.  The other CTAs
// update the real blocks, B3 / UPD_THREADS CTAs per block, each a run of
// UPD_THREADS cells in block order (full warps).  All read src (and the
// ghost lanes the coarser level's csrc); the real-block CTAs write dst only.
template <typename S, bool HAS_FINE, bool HAS_COARSE, bool COUPLED>
__global__ void __launch_bounds__(UPD_THREADS, sizeof(S) == 8 ? 1 : UPD_MIN_CTAS)
    k_update(UpdateArgs<S> U, const int* __restrict__ glist, int nglist, int gblocks, int coalesce) {
    using A = typename Store<S>::A;
    if (HAS_COARSE && (int)blockIdx.x < gblocks) {   // uniform across the block
        const int i = blockIdx.x * UPD_THREADS + threadIdx.x;
        // every lane of the last sub-step takes part in the shuffles (nglist is a multiple of 8)
        const bool valid = i < nglist;
        if (!coalesce && !valid) return;
        A g[19];
        int hp = 0, b = 0, c = 0;
        if (valid) {
            const int e = glist[i];
            b = e >> 12;
            c = e & 4095;
            hp = U.ghost_host[i >> 3];
            const GhostPull gp{U.smask[i], hp >> 12, hp & 4095, i & 7, coalesce != 0};
            if (pull_cell<S, true>(U, b, c, U.D.nbr + (size_t)b * 27, g, gp)) atomicOr(U.status, STATUS_AMR_MISSING);
            if (!coalesce) {
#pragma unroll
                for (int q = 0; q < 19; ++q) Store<S>::store_raw(U.dst + paddr(b, q, c), g[q]);
                return;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 19; ++q) g[q] = A(0);
        }
#pragma unroll
        for (int q = 0; q < 19; ++q) {
            A v = g[q];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            g[q] = v;
        }
        if (valid) {
            // each of the eight lanes holds the sum and forms the host's collided populations
#pragma unroll
            for (int q = 0; q < 19; ++q) g[q] *= A(0.125);
            trt_collide<A, false, sizeof(S) == 2>(g, U.Pc, U.status);
            if ((i & 7) == 0) {   // the host, into the coarser level's new state
                const int hb = hp >> 12, hc = hp & 4095;
#pragma unroll
                for (int q = 0; q < 19; ++q) Store<S>::store_raw(U.cdst + paddr(hb, q, hc), g[q]);
            }
            // and the explosion of that new state: this ghost cell, in the buffer the level's next
            // pair of sub-steps starts from
#pragma unroll
            for (int q = 0; q < 19; ++q) Store<S>::store_raw(U.dst + paddr(b, q, c), g[q]);
        }
        return;
    }
    // Real cells: pull and collide.  The cell's mark is loaded beside the pulls rather than before
    // them (a branch on it would hold the pulls back by one memory round trip); the pulls of a
    // cell it then excludes are dropped.  The finest level's flags: 1 solid (stored as zero), 2
    // fluid next to the sphere (k_amr_boundary's cells).  Hosts (levels with a finer level, mark 1)
    // are left to the finer level's last sub-step, which forms their coalesced populations.
    __shared__ int nb27[27];
    constexpr int SPB = B3 / UPD_THREADS;   // CTAs per block
    const int b = (blockIdx.x - gblocks) / SPB;
    const int c = ((blockIdx.x - gblocks) % SPB) * UPD_THREADS + threadIdx.x;
    uint8_t mark = 0;
    if (COUPLED) mark = U.solid[(size_t)b * B3 + c];
    else if (HAS_FINE) mark = U.D.host[(size_t)b * B3 + c];
    if (threadIdx.x < 27) nb27[threadIdx.x] = U.D.nbr[b * 27 + threadIdx.x];
    __syncthreads();
    A g[19];
    const bool missing = pull_cell<S>(U, b, c, nb27, g);
    if (COUPLED) {
        if (mark == FLAG_SOLID) {
#pragma unroll
            for (int q = 0; q < 19; ++q) Store<S>::store_raw(U.dst + paddr(b, q, c), A(0));
            return;
        }
        if (mark == FLAG_BOUNDARY) return;
    }
    if (HAS_FINE && mark == 1) return;
    if (missing) atomicOr(U.status, STATUS_AMR_MISSING);
    trt_collide<A, false, sizeof(S) == 2>(g, U.P, U.status);
#pragma unroll
    for (int q = 0; q < 19; ++q) Store<S>::store_raw(U.dst + paddr(b, q, c), g[q]);
}

// ---------------------------------------------------------------- coupling
constexpr int BNDW_THREADS = 256;
constexpr int BND_CHUNK = 128;     // box cells per boundary CTA (sizes the grid)
// Register cap of the boundary kernel (BNDW_THREADS threads).  It runs beside the finest level's
// update for most of that update, so every register it holds is taken from the update's CTAs: at
// 56 in FP32 a boundary CTA (14,336 registers) leaves room for 1,280 update threads of 40 registers
// instead of 1,024.
template <typename S>
constexpr int BND_MAXREG = sizeof(S) == 8 ? 128 : (sizeof(S) == 4 ? 56 : 64);
constexpr int LINK_THREADS = 64;   // box cells per run of the boundary mask (one count per run)
constexpr int REMAP_THREADS = 256;   // remap blocks: their uncovered cells are spread over the eight warps

// Exclusive prefix of n counts into pre[0..n] (pre[n] = total), computed by
// the whole CTA (NT threads, two consecutive counts per thread and pass);
// every thread must call it.  first0, first1: counts 2 threadIdx.x and
// 2 threadIdx.x + 1 (0 beyond n), loaded by the caller ahead.
template <int NT>
__device__ __forceinline__ int block_prefix(const int* __restrict__ count, int n, int* pre, int first0, int first1) {
    __shared__ int wsum[NT / 32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 2 * NT) {
        const int i = base + 2 * (int)threadIdx.x;
        const int c0 = base == 0 ? first0 : (i < n ? count[i] : 0);
        const int c1 = base == 0 ? first1 : (i + 1 < n ? count[i + 1] : 0);
        int v = c0 + c1;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += y;
        }
        if (lane == 31) wsum[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int w = lane < NT / 32 ? wsum[lane] : 0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += y;
            }
            if (lane < NT / 32) wsum[lane] = w;
        }
        __syncthreads();
        const int incl = carry + (wid > 0 ? wsum[wid - 1] : 0) + v;   // through count i + 1
        if (i < n) pre[i + 1] = incl - c1;
        if (i + 1 < n) pre[i + 2] = incl;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[NT / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) pre[0] = 0;
    __syncthreads();
    return pre[n];
}

// Boundary cells of the finest level (flag 2: fluid with a solid
// neighbour), from the mask the remap wrote in box order and its count of
// marked cells per run of LINK_THREADS box cells.  The marked cells are
// spread evenly over all warps of the grid: every CTA turns the counts into
// a prefix, and warp w of W takes the marked cells w, w + W, ... (box
// order), one cell per warp at a time, lane q handling population q (CLI
// links of Sec. 2.3, geometry in the population arithmetic, FP64 force
// partials per CTA), with a cooperative collision.  The level update skips
// these cells, so this kernel runs beside it.  The block that finishes
// last sums the partials and runs the particle update of Algorithm 1.
// Dynamic shared memory: (runs + 1) ints.
template <typename S>
__global__ void __maxnreg__(BND_MAXREG<S>)
    k_amr_boundary(LevelView D, const S* __restrict__ src, S* __restrict__ dst, const uint8_t* __restrict__ solid,
                   const uint8_t* __restrict__ mask, const int* __restrict__ run_count, BoxDesc B,
                   CollideParams<typename Store<S>::A> P, ParticleState* ps, int cli, double* partials, int* done,
                   GridDesc G, double* __restrict__ history, int hist_cap, int* __restrict__ status,
                   PFrames* __restrict__ frames) {
    using A = typename Store<S>::A;
    extern __shared__ int pre[];   // [runs + 1]
    __shared__ LinkFrame<A> Fr;
    __shared__ BoxFrame Bf;
    const int runs = (int)((B.cells + LINK_THREADS - 1) / LINK_THREADS);
    const int i2 = 2 * (int)threadIdx.x;   // this thread's first two counts, in flight during the set-up
    const int first0 = i2 < runs ? run_count[i2] : 0, first1 = i2 + 1 < runs ? run_count[i2 + 1] : 0;
    if (threadIdx.x == 0) Fr = pframe_link<A>(*frames);   // formed by the last particle update
    if (threadIdx.x == 32) Bf = frames->bf;
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int total = block_prefix<BNDW_THREADS>(run_count, runs, pre, first0, first1);
    const int W = (int)gridDim.x * (BNDW_THREADS / 32);
    LinkSums<A> acc;
    for (int j = (int)blockIdx.x * (BNDW_THREADS / 32) + wib; j < total; j += W) {
        // run r holding marked cell j: the largest r with pre[r] <= j
        int lo = 0, hi = runs;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pre[mid] <= j) lo = mid;
            else hi = mid;
        }
        const long long r0 = (long long)lo * LINK_THREADS;
        const bool m0 = r0 + lane < B.cells && mask[r0 + lane] != 0;
        const bool m1 = r0 + 32 + lane < B.cells && mask[r0 + 32 + lane] != 0;
        const unsigned b0 = __ballot_sync(0xffffffffu, m0), b1 = __ballot_sync(0xffffffffu, m1);
        int k = j - pre[lo];
        unsigned bits = b0;
        int base = 0;
        if (k >= __popc(b0)) {
            k -= __popc(b0);
            bits = b1;
            base = 32;
        }
        for (; k > 0; --k) bits &= bits - 1u;   // drop the k lowest marked cells
        const int t = (int)(r0 + base + __ffs((int)bits) - 1);
        int g[3], c;
        if (!box_cell(t, D.n, D.periodic, B, Bf, g)) continue;   // marked cells are inside the domain
        const int b = locate(D, g, &c);
        const int lx = c & 15, ly = (c >> 4) & 15, lz = c >> 8;
        A gq = A(0);
        if (lane < 19) {
            const int q = lane;
            const int cq[3] = {cx(q), cy(q), cz(q)};
            int sc;
            const int sb = nbr_cell(D, b, lx, ly, lz, -cq[0], -cq[1], -cq[2], &sc);
            if (sb == -2) {
                gq = Store<S>::load(src + paddr(b, opp(q), c), P.inv_scale);
            } else if (sb < 0) {
                atomicOr(status, STATUS_AMR_MISSING);
            } else if (q == 0 || sb >= D.nreal || solid[(size_t)sb * B3 + sc] != FLAG_SOLID) {
                gq = Store<S>::load(src + paddr(sb, q, sc), P.inv_scale);
            } else {
                const int k = opp(q);
                int fc;
                const int fb = nbr_cell(D, b, lx, ly, lz, cq[0], cq[1], cq[2], &fc);   // x - c_k
                const bool far_ok = fb >= 0 && fb < D.nreal && solid[(size_t)fb * B3 + fc] != FLAG_SOLID;
                A d[3], fl[3], tl3[3];
                int pu[3];
                Fr.offset(g, D.n, D.periodic, d, pu);
                const A gt_k = Store<S>::load(src + paddr(b, k, c), P.inv_scale);
                const A gt_q = Store<S>::load(src + paddr(b, q, c), P.inv_scale);
                const A gt_far = far_ok ? Store<S>::load(src + paddr(fb, k, fc), P.inv_scale) : A(0);
                gq = cli_link<A>(q, d, cli && far_ok, gt_k, gt_q, gt_far, Fr, fl, tl3);
                acc.add(k, pu, fl, tl3);
            }
        }
        gq = warp_trt_collide<A, false>(gq, lane, P, status);
        if (lane < 19) Store<S>::store(dst + paddr(b, lane, c), gq, P.scale);
    }
    block_link_sums<BNDW_THREADS>(acc, ps->x, partials + (size_t)blockIdx.x * 6);
    if (last_block_done(done, (int)gridDim.x)) {   // every other block is past its use of the frames
        particle_block_update<BNDW_THREADS>(ps, partials, gridDim.x, G, history, hist_cap, status, frames->inv);
        __syncthreads();
        if (threadIdx.x < 3) pframes_axis(frames, *ps, D.n, B, threadIdx.x);   // of the moved sphere
    }
}


// Refill of the uncovered cell (b, c) at g by the whole warp (Sec. 2.3).
// Lane q = 1..18 takes the neighbour g + c_q, counted when it is fluid
// before (fcur) and after (the ball predicate) the move, with its density
// 1 + sum_p g_p and its momentum sum_p c_p g_p (used for the six face
// neighbours by Grad's strain rate).  The mean density of the counted
// neighbours and the rigid-body velocity u_p + omega_p x (x - x_p) give the
// equilibrium, plus Grad's non-equilibrium term when gcoef != 0; lane
// q < 19 writes population q.  Every lane calls it with the same cell.
// With lf (the FP32 link frame of the moved sphere) an FP32 path forms the
// offset (g + 1/2 - X = (g - Xi) + Xh, minimum image on periodic axes) and
// the rigid-body velocity in FP32 instead of FP64, which is slow here.
template <typename S>
__device__ __forceinline__ void refill_cell_warp(const LevelView& D, S* __restrict__ pops,
                                                 const uint8_t* __restrict__ fcur, const BoxFrame& F,
                                                 const ParticleState& P, int b, int c, const int g[3],
                                                 typename Store<S>::A scale, typename Store<S>::A inv_scale,
                                                 typename Store<S>::A gcoef, const LinkFrame<float>* lf) {
    using A = typename Store<S>::A;
    const int lane = threadIdx.x & 31;
    bool ok = false;
    A r = A(0), mo[3] = {A(0), A(0), A(0)};
    if (lane >= 1 && lane < 19) {
        int v[3] = {g[0] + cx(lane), g[1] + cy(lane), g[2] + cz(lane)};
        if (wrap3(v, D) && !ball_flag(v, D.n, D.periodic, F, P)) {
            int vc;
            const int vb = locate(D, v, &vc);
            if (vb >= 0 && vb < D.nreal) {
                // the populations are loaded beside the flag (not after it): a solid neighbour's are dropped
                A gp[19];
#pragma unroll
                for (int p = 0; p < 19; ++p) gp[p] = Store<S>::load(pops + paddr(vb, p, vc), inv_scale);
                ok = fcur[(size_t)vb * B3 + vc] != FLAG_SOLID;
                r = A(1);
#pragma unroll
                for (int p = 0; p < 19; ++p) r += gp[p];
#pragma unroll
                for (int p = 1; p < 19; ++p) {
                    mo[0] += A(cx(p)) * gp[p];
                    mo[1] += A(cy(p)) * gp[p];
                    mo[2] += A(cz(p)) * gp[p];
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
    A u[3];
    if (sizeof(A) == 4 && lf) {
        float d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int v = g[a] - lf->Xi[a];
            if (D.periodic[a]) {
                const float t = (float)v + lf->Xh[a], half = 0.5f * (float)D.n[a];
                v += t > half ? -D.n[a] : (t < -half ? D.n[a] : 0);
            }
            d[a] = (float)v + lf->Xh[a];
        }
        u[0] = A(lf->u[0] + (lf->w[1] * d[2] - lf->w[2] * d[1]));
        u[1] = A(lf->u[1] + (lf->w[2] * d[0] - lf->w[0] * d[2]));
        u[2] = A(lf->u[2] + (lf->w[0] * d[1] - lf->w[1] * d[0]));
    } else {
        const double d[3] = {wrap_diff((g[0] + 0.5) - P.x[0], D.n[0], D.periodic[0]),
                             wrap_diff((g[1] + 0.5) - P.x[1], D.n[1], D.periodic[1]),
                             wrap_diff((g[2] + 0.5) - P.x[2], D.n[2], D.periodic[2])};
        u[0] = A(P.u[0] + (P.w[1] * d[2] - P.w[2] * d[1]));
        u[1] = A(P.u[1] + (P.w[2] * d[0] - P.w[0] * d[2]));
        u[2] = A(P.u[2] + (P.w[0] * d[1] - P.w[1] * d[0]));
    }
    const A uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    A Sr[6] = {A(0), A(0), A(0), A(0), A(0), A(0)};
    if (gcoef != A(0)) {   // Grad refill: face neighbour q = 1 + 2 a (+1 for -e_a), fluid before and after
        auto nb = [&](int a, int sgn, A uo[3]) {
            const int q = 1 + 2 * a + (sgn > 0 ? 0 : 1);
#pragma unroll
            for (int k = 0; k < 3; ++k) uo[k] = __shfl_sync(0xffffffffu, mo[k], q);
            return ((okm >> q) & 1u) != 0;
        };
        refill_strain<A>(nb, u, Sr);
    }
    if (lane < 19) {
        A e = geq_dev<A>(lane, rho - A(1), u, uu);
        if (gcoef != A(0)) e += grad_term<A>(lane, Sr, gcoef);
        Store<S>::store(pops + paddr(b, lane, c), e, scale);
    }
}

// Frames of the current record, after the host changed it (one block of 128 threads).
__global__ void k_pframes(const ParticleState* __restrict__ ps, PFrames* __restrict__ frames, LevelView D, BoxDesc B) {
    pframes_form(frames, *ps, D.n, D.periodic, B);
}

// Remap of Sec. 2.3 after the particle moved, over the box of finest cells
// around the sphere, in one pass: the new solid flag of every cell (the
// exact ball predicate); newly covered cells drop their populations (the
// update already zeroed the cells that were solid before); uncovered cells
// are listed in shared memory and refilled afterwards, each by one warp of
// the block in turn (refill_cell_warp: it reads only cells that are fluid
// before and after the move, which nothing here writes); fluid cells with a
// solid neighbour are marked for the boundary list (counts per run of
// LINK_THREADS box cells for the ordered compaction).  Neighbour flags are
// evaluated from the same predicate instead of being read back, so no
// second pass is needed.
template <typename S>
__global__ void __launch_bounds__(REMAP_THREADS)
    k_amr_remap(LevelView D, S* __restrict__ pops, const uint8_t* __restrict__ fcur, uint8_t* __restrict__ fnext,
                BoxDesc B, const ParticleState* __restrict__ ps, typename Store<S>::A scale,
                typename Store<S>::A inv_scale, uint8_t* __restrict__ mask, int* __restrict__ block_count,
                int* __restrict__ status, typename Store<S>::A gcoef, const PFrames* __restrict__ frames) {
    using A = typename Store<S>::A;
    __shared__ BoxFrame F;
    __shared__ int s_n;
    __shared__ int s_cell[2][REMAP_THREADS], s_g[3][REMAP_THREADS];   // uncovered cells: pool block, cell, position
    if (threadIdx.x == 0) {
        if (frames) F = frames->bf;   // formed by the particle update that moved the sphere
        else box_frame_init(F, D.n, D.periodic, B, *ps);
        s_n = 0;
    }
    __syncthreads();
    const ParticleState& P = *ps;
    const int t = blockIdx.x * REMAP_THREADS + threadIdx.x;
    int is_b = 0;
    if (t < B.cells) {
        int g[3];
        if (box_cell(t, D.n, D.periodic, B, F, g)) {
            int c;
            const int b = locate(D, g, &c);
            if (b < 0 || b >= D.nreal) {
                atomicOr(status, STATUS_NOT_FINEST);
            } else {
                const size_t x = (size_t)b * B3 + c;
                bool any_nb = false;
                const bool solid = ball_flag_and_neighbours(g, D.n, D.periodic, F, P, &any_nb);
                const bool was_solid = fcur[x] == FLAG_SOLID;
                if (solid) {
                    fnext[x] = FLAG_SOLID;
                    if (!was_solid)
#pragma unroll
                        for (int q = 0; q < 19; ++q) Store<S>::store(pops + paddr(b, q, c), A(0), scale);
                } else {
                    is_b = any_nb ? 1 : 0;
                    fnext[x] = is_b ? FLAG_BOUNDARY : FLAG_FLUID;
                    if (was_solid) {   // uncovered: fluid after the move, solid before
                        const int k = atomicAdd(&s_n, 1);
                        s_cell[0][k] = b;
                        s_cell[1][k] = c;
                        s_g[0][k] = g[0];
                        s_g[1][k] = g[1];
                        s_g[2][k] = g[2];
                    }
                }
            }
        }
        mask[t] = (uint8_t)is_b;
    }
    __syncthreads();
    const int wid = threadIdx.x >> 5;
    for (int k = wid; k < s_n; k += REMAP_THREADS / 32) {
        const int g3[3] = {s_g[0][k], s_g[1][k], s_g[2][k]};
        refill_cell_warp<S>(D, pops, fcur, F, P, s_cell[0][k], s_cell[1][k], g3, scale, inv_scale, gcoef,
                            frames ? &frames->lf : nullptr);
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, is_b);
    __shared__ int wsum[REMAP_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wsum[wid] = __popc(ballot);
    __syncthreads();
    constexpr int RUNS = REMAP_THREADS / LINK_THREADS, WPR = LINK_THREADS / 32;
    if ((int)threadIdx.x < RUNS) {
        const long long run = (long long)blockIdx.x * RUNS + threadIdx.x;
        if (run * LINK_THREADS < B.cells) {
            int s = 0;
            for (int w = 0; w < WPR; ++w) s += wsum[threadIdx.x * WPR + w];
            block_count[run] = s;
        }
    }
}

__global__ void __launch_bounds__(LINK_THREADS)
    k_amr_links_emit(LevelView D, const uint8_t* __restrict__ mask, const int* __restrict__ block_count, BoxDesc B,
                     const ParticleState* __restrict__ ps, int* __restrict__ list, int* __restrict__ count,
                     int capacity, int* __restrict__ status) {
    __shared__ int red[LINK_THREADS];
    __shared__ int wsum[LINK_THREADS / 32];
    __shared__ BoxFrame F;
    if (threadIdx.x == 0) box_frame_init(F, D.n, D.periodic, B, *ps);
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
    const int is_b = t < B.cells ? mask[t] : 0;
    const unsigned ballot = __ballot_sync(0xffffffffu, is_b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = __popc(ballot);
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += wsum[w];
    if (is_b) {
        int g[3], c;
        const bool in = box_cell(t, D.n, D.periodic, B, F, g);
        const int b = in ? locate(D, g, &c) : -1;
        const int pos = base + wbase + __popc(ballot & ((1u << lane) - 1u));
        if (pos >= capacity) atomicOr(status, STATUS_LINK_OVERFLOW);
        else if (b >= 0) list[pos] = (b << 12) | c;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        int tot = base;
        for (int w = 0; w < LINK_THREADS / 32; ++w) tot += wsum[w];
        *count = tot < capacity ? tot : capacity;
    }
}

// ------------------------------------------------------ classification
// Host flag of every real cell: 1 when a cell covered by the next finer
// level lies within Chebyshev distance 1, 2 when the nearest is at 2 (the
// second ring).  Each CTA (a run of 256 cells) also counts its hosts into
// run_counts[run].
__global__ void __launch_bounds__(256) k_host_flags(LevelView D, uint8_t* __restrict__ host, int* __restrict__ run_counts) {
    const int b = blockIdx.x >> 4;
    const int bx = D.bpos[3 * b], by = D.bpos[3 * b + 1], bz = D.bpos[3 * b + 2];
    const int c = ((blockIdx.x & 15) << 8) + threadIdx.x;
    const int g[3] = {bx * BS + (c & 15), by * BS + ((c >> 4) & 15), bz * BS + (c >> 8)};
    int dist = 3;
    for (int dz = -2; dz <= 2; ++dz)
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx) {
                int v[3] = {g[0] + dx, g[1] + dy, g[2] + dz};
                if (!wrap3(v, D)) continue;
                if (D.refined[(v[0] >> 4) + D.nb[0] * ((v[1] >> 4) + D.nb[1] * (v[2] >> 4))]) {
                    const int m = max(abs(dx), max(abs(dy), abs(dz)));
                    dist = min(dist, m);
                }
            }
    const int kind = dist <= 1 ? 1 : (dist == 2 ? 2 : 0);
    host[(size_t)b * B3 + c] = (uint8_t)kind;
    __shared__ int wc[8];
    const unsigned b1 = __ballot_sync(0xffffffffu, kind == 1);
    if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(b1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 8; ++w) t += wc[w];
        run_counts[blockIdx.x] = t;
    }
}

// Active ghost-cell list of level l+1 from the host flags of level l (same
// runs as k_host_flags): the eight sub-cells of every host (flag 1) in host
// order (real block, then cell) and sub-cell order, each entry the
// sub-cell's pool block << 12 | cell, and per host its real block << 12 |
// cell in hosts.
__global__ void __launch_bounds__(256)
    k_ghost_lists(LevelView C, const uint8_t* __restrict__ host, const int* __restrict__ run_counts, LevelView F,
                  int* __restrict__ list, int* __restrict__ hosts, int* __restrict__ status) {
    __shared__ int red[256];
    __shared__ int wc[8];
    int s1 = 0;
    for (int r = threadIdx.x; r < (int)blockIdx.x; r += 256) s1 += run_counts[r];
    red[threadIdx.x] = s1;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    const int b = blockIdx.x >> 4;
    const int c = ((blockIdx.x & 15) << 8) + threadIdx.x;
    const bool is_host = host[(size_t)b * B3 + c] == 1;
    const unsigned b1 = __ballot_sync(0xffffffffu, is_host);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wc[warp] = __popc(b1);
    __syncthreads();
    if (!is_host) return;
    int pos = red[0];
    for (int w = 0; w < warp; ++w) pos += wc[w];
    pos += __popc(b1 & ((1u << lane) - 1u));
    hosts[pos] = (b << 12) | c;
    int* out = list + 8 * pos;
    const int p[3] = {C.bpos[3 * b] * BS + (c & 15), C.bpos[3 * b + 1] * BS + ((c >> 4) & 15), C.bpos[3 * b + 2] * BS + (c >> 8)};
    for (int sub = 0; sub < 8; ++sub) {
        const int g[3] = {2 * p[0] + (sub & 1), 2 * p[1] + ((sub >> 1) & 1), 2 * p[2] + (sub >> 2)};
        int gc;
        const int gb = locate(F, g, &gc);
        if (gb < F.nreal) {   // by construction every sub-cell of a host is a ghost cell
            atomicOr(status, STATUS_AMR_MISSING);
            out[sub] = 0;
            continue;
        }
        out[sub] = (gb << 12) | gc;
    }
}

// Static-neighbour masks of the active ghost cells of level F (list and
// hosts of k_ghost_lists, n entries): bit q is set when the upwind
// neighbour x - c_q lies in a ghost block and its coarse cell (P + o, see
// GhostPull) is a second-ring cell of level C (host flag 2).  A ghost
// neighbour whose coarse cell is neither a host nor in the second ring is
// an error of the layout.
__global__ void __launch_bounds__(256)
    k_ghost_smask(LevelView C, LevelView F, const int* __restrict__ list, const int* __restrict__ hosts, int n,
                  uint32_t* __restrict__ smask, int* __restrict__ status) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const int e = list[i], hp = hosts[i >> 3];
    const int b = e >> 12, c = e & 4095, hb = hp >> 12, hc = hp & 4095, sub = i & 7;
    const int s[3] = {sub & 1, (sub >> 1) & 1, sub >> 2};
    uint32_t m = 0;
    for (int q = 1; q < 19; ++q) {
        const int cq[3] = {cx(q), cy(q), cz(q)};
        int nc;
        const int nbk = nbr_cell(F, b, c & 15, (c >> 4) & 15, c >> 8, -cq[0], -cq[1], -cq[2], &nc);
        if (nbk < F.nreal) continue;   // a real cell, a wall or no block: the ordinary pull
        int o[3];
        for (int a = 0; a < 3; ++a) o[a] = cq[a] == 1 ? s[a] - 1 : (cq[a] == -1 ? s[a] : 0);
        int pc;
        const int pb = nbr_cell(C, hb, hc & 15, (hc >> 4) & 15, hc >> 8, o[0], o[1], o[2], &pc);
        const int kind = (pb >= 0 && pb < C.nreal) ? C.host[(size_t)pb * B3 + pc] : 0;
        if (kind == 2) m |= 1u << q;
        else if (kind != 1) atomicOr(status, STATUS_AMR_MISSING);
    }
    smask[i] = m;
}

__global__ void k_amr_flags_full(LevelView D, uint8_t* __restrict__ f0, uint8_t* __restrict__ f1,
                                 const ParticleState* __restrict__ ps) {
    const int b = blockIdx.x >> 4;
    const ParticleState P = *ps;
    const int bx = D.bpos[3 * b], by = D.bpos[3 * b + 1], bz = D.bpos[3 * b + 2];
    {
        const int c = ((blockIdx.x & 15) << 8) + threadIdx.x;
        const int g[3] = {bx * BS + (c & 15), by * BS + ((c >> 4) & 15), bz * BS + (c >> 8)};
        const uint8_t v = (P.present && inside_ball_exact(g, D.n, D.periodic, P)) ? 1 : 0;
        f0[(size_t)b * B3 + c] = v;
        f1[(size_t)b * B3 + c] = v;
    }
}

template <typename S>
__global__ void k_amr_zero_solid(S* __restrict__ pops, const uint8_t* __restrict__ flags) {
    using A = typename Store<S>::A;
    const int b = blockIdx.x >> 4;
    const int c = ((blockIdx.x & 15) << 8) + threadIdx.x;
    if (flags[(size_t)b * B3 + c])
        for (int q = 0; q < 19; ++q) Store<S>::store(pops + paddr(b, q, c), A(0), A(1));
}

template <typename S>
__global__ void k_amr_init(LevelView D, S* __restrict__ pops, const uint8_t* __restrict__ solid, double rho,
                           double u0, double u1, double u2, double amp, int dir, int axis, double h, double Lax,
                           typename Store<S>::A scale) {
    using A = typename Store<S>::A;
    const int b = blockIdx.x >> 4;
    const int bx = D.bpos[3 * b], by = D.bpos[3 * b + 1], bz = D.bpos[3 * b + 2];
    {
        const int c = ((blockIdx.x & 15) << 8) + threadIdx.x;
        const int g[3] = {bx * BS + (c & 15), by * BS + ((c >> 4) & 15), bz * BS + (c >> 8)};
        double u[3] = {u0, u1, u2};
        if (amp != 0.0) u[dir] += amp * sin(2.0 * M_PI * (g[axis] + 0.5) * h / Lax);
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const bool s = solid && solid[(size_t)b * B3 + c] == FLAG_SOLID;
        for (int q = 0; q < 19; ++q) {
            const double cu = cx(q) * u[0] + cy(q) * u[1] + cz(q) * u[2];
            const double e = wgt<double>(q) * ((rho - 1.0) + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
            Store<S>::store(pops + paddr(b, q, c), s ? A(0) : A(e), scale);
        }
    }
}

// Regrid: every real cell of the new layout from the old layout (copy,
// explosion of the old coarser cell, or mean of the old finer cells), with
// the post-collision rescaling chained over the levels crossed.
template <typename S>
struct MigrateArgs {
    using A = typename Store<S>::A;
    LevelView N;          // new level
    S* dst;
    int l;
    int L;
    LevelView O[MAXL];    // old levels
    const S* osrc[MAXL];
    A kp[MAXL], km[MAXL];  // c->f post-collision factors between level k and k+1
    int rescale;
    A scale, inv_scale;
};

template <typename S>
__global__ void k_migrate(MigrateArgs<S> M) {
    using A = typename Store<S>::A;
    const int b = blockIdx.x >> 4;
    const LevelView& N = M.N;
    const int bx = N.bpos[3 * b], by = N.bpos[3 * b + 1], bz = N.bpos[3 * b + 2];
    {
        const int c = ((blockIdx.x & 15) << 8) + threadIdx.x;
        const int g[3] = {bx * BS + (c & 15), by * BS + ((c >> 4) & 15), bz * BS + (c >> 8)};
        A f[19];
        for (int q = 0; q < 19; ++q) f[q] = A(0);
        for (int lo = 0; lo < M.L; ++lo) {
            const LevelView& O = M.O[lo];
            if (lo <= M.l) {
                const int sh = M.l - lo;
                const int v[3] = {g[0] >> sh, g[1] >> sh, g[2] >> sh};
                int oc;
                const int ob = locate(O, v, &oc);
                if (ob < 0 || ob >= O.nreal) continue;
                for (int q = 0; q < 19; ++q) f[q] = Store<S>::load(M.osrc[lo] + paddr(ob, q, oc), M.inv_scale);
                if (M.rescale)
                    for (int k = lo; k < M.l; ++k) rescale19<A>(f, M.kp[k], M.km[k]);
                break;
            } else {
                const int k = 1 << (lo - M.l);
                const int v0[3] = {g[0] * k, g[1] * k, g[2] * k};
                int oc;
                const int ob = locate(O, v0, &oc);
                if (ob < 0 || ob >= O.nreal) continue;
                for (int dz = 0; dz < k; ++dz)
                    for (int dy = 0; dy < k; ++dy)
                        for (int dx = 0; dx < k; ++dx) {
                            const int v[3] = {v0[0] + dx, v0[1] + dy, v0[2] + dz};
                            const int vb = locate(O, v, &oc);
                            for (int q = 0; q < 19; ++q)
                                f[q] += Store<S>::load(M.osrc[lo] + paddr(vb, q, oc), M.inv_scale);
                        }
                const A inv = A(1) / A(k * k * k);
                for (int q = 0; q < 19; ++q) f[q] *= inv;
                if (M.rescale)
                    for (int kk = lo - 1; kk >= M.l; --kk) rescale19<A>(f, A(1) / M.kp[kk], A(1) / M.km[kk]);
                break;
            }
        }
        for (int q = 0; q < 19; ++q) Store<S>::store(M.dst + paddr(b, q, c), f[q], M.scale);
    }
}

template <typename S>
__global__ void k_amr_export(LevelView D, const S* __restrict__ pops, int32_t* __restrict__ xyz,
                             double* __restrict__ out, typename Store<S>::A inv_scale) {
    const int b = blockIdx.x >> 4;
    const int bx = D.bpos[3 * b], by = D.bpos[3 * b + 1], bz = D.bpos[3 * b + 2];
    {
        const int c = ((blockIdx.x & 15) << 8) + threadIdx.x;
        const size_t m = (size_t)b * B3 + c;
        xyz[3 * m] = bx * BS + (c & 15);
        xyz[3 * m + 1] = by * BS + ((c >> 4) & 15);
        xyz[3 * m + 2] = bz * BS + (c >> 8);
        for (int q = 0; q < 19; ++q) out[m * 19 + q] = (double)Store<S>::load(pops + paddr(b, q, c), inv_scale);
    }
}

// Flow sensor (Sec. 4.2.2): the largest scaled curl phi_c = |curl u| s^1.5
// (r = 2; s and the derivatives in finest-level units) over the cells of
// each real block of one level.  u = sum_q g_q c_q summed in q order;
// derivatives are central differences inside the block and one-sided on its
// faces; products, sums, quotients and the root are rounded one by one (no
// contraction), so the FP64 form reproduces the plain definition exactly.
// One CTA per real block; the block's velocities are staged in shared
// memory ([3][4096] of the arithmetic type), the maximum is reduced across
// the CTA, and out[b] = max |curl u| * s^1.5 (weight = s^1.5 from the host).
constexpr int SENSOR_THREADS = 512;

__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rn_sqrt(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ float rn_sqrt(float a) { return __fsqrt_rn(a); }

template <typename S>
__global__ void __launch_bounds__(SENSOR_THREADS)
    k_block_sensor(const S* __restrict__ pops, typename Store<S>::A inv, typename Store<S>::A s, double weight,
                   double* __restrict__ out) {
    using A = typename Store<S>::A;
    extern __shared__ __align__(16) unsigned char sensor_smem[];
    A* u = reinterpret_cast<A*>(sensor_smem);   // [3][B3]
    __shared__ A warp_best[SENSOR_THREADS / 32];
    const S* p = pops + (size_t)blockIdx.x * 19 * B3;
    for (int c = threadIdx.x; c < B3; c += SENSOR_THREADS) {
        A m0 = A(0), m1 = A(0), m2 = A(0);
#pragma unroll
        for (int q = 1; q < 19; ++q) {   // q = 0 has c = 0
            const A g = Store<S>::load(p + q * B3 + c, inv);
            if (cx(q)) m0 = rn_add(m0, cx(q) > 0 ? g : -g);
            if (cy(q)) m1 = rn_add(m1, cy(q) > 0 ? g : -g);
            if (cz(q)) m2 = rn_add(m2, cz(q) > 0 ? g : -g);
        }
        u[c] = m0;
        u[B3 + c] = m1;
        u[2 * B3 + c] = m2;
    }
    __syncthreads();
    A best = A(0);
    for (int c = threadIdx.x; c < B3; c += SENSOR_THREADS) {
        const int pc[3] = {c & (BS - 1), (c >> 4) & (BS - 1), c >> 8};
        // d u_k / d x_a
        auto d = [&](int k, int a) -> A {
            const int st = a == 0 ? 1 : (a == 1 ? BS : BS * BS);
            const int lo = pc[a] > 0 ? c - st : c, hi = pc[a] < BS - 1 ? c + st : c;
            const A span = (pc[a] > 0 && pc[a] < BS - 1) ? A(2) : A(1);
            return rn_div(rn_add(u[k * B3 + hi], -u[k * B3 + lo]), rn_mul(span, s));
        };
        const A wx = rn_add(d(2, 1), -d(1, 2));
        const A wy = rn_add(d(0, 2), -d(2, 0));
        const A wz = rn_add(d(1, 0), -d(0, 1));
        const A c2 = rn_add(rn_add(rn_mul(wx, wx), rn_mul(wy, wy)), rn_mul(wz, wz));
        best = fmax(best, rn_sqrt(c2));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0) warp_best[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        A m = warp_best[0];
        for (int w = 1; w < SENSOR_THREADS / 32; ++w) m = fmax(m, warp_best[w]);
        out[blockIdx.x] = __dmul_rn((double)m, weight);
    }
}


__global__ void k_amr_export_links(LevelView D, const uint8_t* __restrict__ flags, const int* __restrict__ list,
                                   const int* __restrict__ count, const ParticleState* __restrict__ ps,
                                   int64_t* __restrict__ cell_out, int32_t* __restrict__ q_out,
                                   double* __restrict__ delta_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count) return;
    const int e = list[i];
    const int b = e >> 12, c = e & 4095;
    const int g[3] = {D.bpos[3 * b] * BS + (c & 15), D.bpos[3 * b + 1] * BS + ((c >> 4) & 15),
                      D.bpos[3 * b + 2] * BS + (c >> 8)};
    const ParticleState& P = *ps;
    const double d[3] = {wrap_diff((g[0] + 0.5) - P.x[0], D.n[0], D.periodic[0]),
                         wrap_diff((g[1] + 0.5) - P.x[1], D.n[1], D.periodic[1]),
                         wrap_diff((g[2] + 0.5) - P.x[2], D.n[2], D.periodic[2])};
    for (int q = 1; q < 19; ++q) {
        const size_t slot = (size_t)i * 18 + (q - 1);
        cell_out[slot] = (int64_t)g[0] + (int64_t)D.n[0] * ((int64_t)g[1] + (int64_t)D.n[1] * g[2]);
        int v[3] = {g[0] + cx(q), g[1] + cy(q), g[2] + cz(q)};
        int vc, vb = -1;
        if (wrap3(v, D)) vb = locate(D, v, &vc);
        if (vb >= 0 && vb < D.nreal && flags[(size_t)vb * B3 + vc] == FLAG_SOLID) {
            q_out[slot] = q;
            delta_out[slot] = link_delta(d, q, P.r);
        } else {
            q_out[slot] = -1;
            delta_out[slot] = 0.0;
        }
    }
}

// =================================================================== host
using Mask = std::vector<uint8_t>;

struct Level {
    int n[3] = {0, 0, 0}, nb[3] = {0, 0, 0};
    int nreal = 0, nghost = 0;
    std::vector<int> map, bpos, nbr;
    Mask refined;
    int* d_map = nullptr;
    int* d_bpos = nullptr;
    int* d_nbr = nullptr;
    uint8_t* d_refined = nullptr;
    uint8_t* d_host = nullptr;
    int nglist = 0;              // active ghost cells (host sub-cells)
    bool ghosts_valid = false;   // the active ghost cells of the current buffer hold the coarser level's hosts
    int* d_glist = nullptr;      // the active ghost cells, pool block << 12 | cell, eight per host
    int* d_ghost_host = nullptr; // per eight: the host, real block << 12 | cell of the coarser level
    uint32_t* d_smask = nullptr; // per active ghost cell: populations with a static ghost cell upwind
    void* d_pops[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t* d_flags[2] = {nullptr, nullptr};   // finest level only
    int fcur = 0;
    double taup = 0, taum = 0;
};

}  // namespace

struct AmrEngine {
    int L = 1;
    int n0[3] = {0, 0, 0};
    int periodic[3] = {1, 1, 1};
    std::vector<Level> lv;
    bool have_box = false;
    double box_lo[3] = {0, 0, 0}, box_hi[3] = {0, 0, 0};
    int boundary_blocks = 1;
    long long coarse_steps = 0;
    // captured runs of one and of two level-0 steps ([steps - 1]) per parity
    // of the level-0 buffers; dropped whenever the layout or a kernel
    // parameter changes
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    long long graph_launches[2] = {0, 0}, graph_updates[2] = {0, 0};
    double graph_tau = 0.0;
    cudaStream_t capture_stream = nullptr;   // private stream used only for capturing
    int* d_done = nullptr;   // last-block-done counter of the boundary kernel (zero between launches)
    PFrames* d_frames = nullptr;   // frames of the sphere's current state (written by the particle update)
    std::vector<std::vector<uint8_t>> cover;      // block coverage per level of the current layout
    cudaStream_t side = nullptr;                  // k_amr_boundary runs here, beside the finest update
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_remap = nullptr;   // a finest remap left on the side stream (remap_pending) ends here
    bool remap_pending = false;
    // Levels below the finest each update on a stream of their own, beside the finer levels'
    // sub-steps (the finest level runs on the caller's stream).  ev_state[l]: level l's last
    // update ended; ev_xdone[l]: the explosion into level l+1 ended, and with it every earlier
    // sub-step of level l+1 (which wrote level l's hosts and read its other buffer).
    cudaStream_t lstream[MAXL] = {};
    cudaEvent_t ev_state[MAXL] = {};
    cudaEvent_t ev_xdone[MAXL] = {};
    cudaEvent_t ev_begin = nullptr;
    int prio_high = 0, prio_low = 0;   // the greatest and the least stream priority
    double sensor_sigma = 0.0, sensor_c = 0.0;   // flow sensor (sigma_c = 0: off)
    double* d_sensor = nullptr;                   // per real block of all levels
    size_t sensor_cap = 0;
    // a layout rebuild failed part way (an allocation or a CUDA call): the levels are incomplete and
    // every call but destroy refuses
    bool broken = false;

};

// Populations changed outside a step: every level's active ghost cells are
// exploded again by the next step.
void amr_invalidate_ghosts(AmrEngine* E) {
    for (auto& V : E->lv) V.ghosts_valid = false;
}

bool amr_ghosts_valid(const AmrEngine* E) {
    for (size_t l = 1; l < E->lv.size(); ++l)
        if (E->lv[l].nglist > 0 && !E->lv[l].ghosts_valid) return false;
    return true;
}

void amr_drop_graphs(AmrEngine* E) {
    for (int k = 0; k < 2; ++k)
        for (int p = 0; p < 2; ++p)
            if (E->graph[k][p]) {
                cudaGraphExecDestroy(E->graph[k][p]);
                E->graph[k][p] = nullptr;
            }
}

namespace {

size_t esize(const lbmp_handle* h) {
    return h->cfg.precision == LBMP_FP64 ? 8 : (h->cfg.precision == LBMP_FP32 ? 4 : 2);
}

template <typename F>
void with_storage_amr(int prec, F&& f) {
    if (prec == LBMP_FP64) f((double*)nullptr);
    else if (prec == LBMP_FP32) f((float*)nullptr);
    else f((__half*)nullptr);
}

LevelView view(const AmrEngine* E, const Level& V) {
    LevelView w;
    for (int a = 0; a < 3; ++a) {
        w.n[a] = V.n[a];
        w.nb[a] = V.nb[a];
        w.periodic[a] = E->periodic[a];
    }
    w.nreal = V.nreal;
    w.npool = V.nreal + V.nghost;
    w.map = V.d_map;
    w.bpos = V.d_bpos;
    w.nbr = V.d_nbr;
    w.host = V.d_host;
    w.refined = V.d_refined;
    return w;
}

void lattice_of(const AmrEngine* E, int l, int nb[3]) {
    for (int a = 0; a < 3; ++a) nb[a] = E->n0[a] * (1 << l) / BS;
}

int bidx(const int nb[3], int x, int y, int z) { return x + nb[0] * (y + nb[1] * z); }

// wrap a block position on periodic axes; false if outside through a wall
bool wrap_pos(const AmrEngine* E, const int nb[3], int p[3]) {
    for (int a = 0; a < 3; ++a) {
        if (p[a] < 0 || p[a] >= nb[a]) {
            if (!E->periodic[a]) return false;
            p[a] = ((p[a] % nb[a]) + nb[a]) % nb[a];
        }
    }
    return true;
}

Mask parents(const AmrEngine* E, const Mask& fine, int lf) {
    int nf[3], nc[3];
    lattice_of(E, lf, nf);
    lattice_of(E, lf - 1, nc);
    Mask out((size_t)nc[0] * nc[1] * nc[2], 0);
    for (int z = 0; z < nf[2]; ++z)
        for (int y = 0; y < nf[1]; ++y)
            for (int x = 0; x < nf[0]; ++x)
                if (fine[bidx(nf, x, y, z)]) out[bidx(nc, x >> 1, y >> 1, z >> 1)] = 1;
    return out;
}

Mask children(const AmrEngine* E, const Mask& coarse, int lc) {
    int nf[3], nc[3];
    lattice_of(E, lc + 1, nf);
    lattice_of(E, lc, nc);
    Mask out((size_t)nf[0] * nf[1] * nf[2], 0);
    for (int z = 0; z < nf[2]; ++z)
        for (int y = 0; y < nf[1]; ++y)
            for (int x = 0; x < nf[0]; ++x) out[bidx(nf, x, y, z)] = coarse[bidx(nc, x >> 1, y >> 1, z >> 1)];
    return out;
}

Mask dilate(const AmrEngine* E, const Mask& m, int l) {
    int nb[3];
    lattice_of(E, l, nb);
    Mask out(m);
    for (int z = 0; z < nb[2]; ++z)
        for (int y = 0; y < nb[1]; ++y)
            for (int x = 0; x < nb[0]; ++x) {
                if (!m[bidx(nb, x, y, z)]) continue;
                for (int dz = -1; dz <= 1; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int p[3] = {x + dx, y + dy, z + dz};
                            if (wrap_pos(E, nb, p)) out[bidx(nb, p[0], p[1], p[2])] = 1;
                        }
            }
    return out;
}

// Level-l block positions covered by blocks of level >= l (Sec. 4.1, 4.2.1):
// finest = siblings of the required set; each coarser level adds the 26
// neighbours of the parents of the next finer level (2:1 balance).  wish
// (optional) holds, per level l >= 1, positions the flow sensor wants
// covered at level >= l; they join the required set of their level before
// the siblings are added.
std::vector<Mask> coverage(const AmrEngine* E, const Mask& finest, const std::vector<Mask>* wish = nullptr) {
    std::vector<Mask> R(E->L);
    int nb[3];
    lattice_of(E, 0, nb);
    R[0].assign((size_t)nb[0] * nb[1] * nb[2], 1);
    if (E->L == 1) return R;
    Mask need = finest;
    if (wish)
        for (size_t i = 0; i < need.size(); ++i) need[i] |= (*wish)[E->L - 1][i];
    R[E->L - 1] = children(E, parents(E, need, E->L - 1), E->L - 2);
    for (int l = E->L - 2; l >= 1; --l) {
        Mask grown = dilate(E, parents(E, R[l + 1], l + 1), l);
        if (wish)
            for (size_t i = 0; i < grown.size(); ++i) grown[i] |= (*wish)[l][i];
        R[l] = children(E, parents(E, grown, l), l - 1);
    }
    return R;
}

// What the flow sensor asks of each real block (Sec. 4.2.2), as positions to
// keep covered per level: above sigma_c a block asks for level l+1 (its
// eight children; the finest level asks for itself), below c sigma_c for
// level l-1 (its parent), in between for level l (itself).  A block that no
// wish, balance or sphere keeps is coarsened; since its siblings' wishes
// keep the whole octet, octets coarsen only together, one level per regrid.
std::vector<Mask> sensor_wishes(const AmrEngine* E, const std::vector<std::vector<double>>& phi) {
    std::vector<Mask> W(E->L);
    for (int l = 0; l < E->L; ++l) {
        int nb[3];
        lattice_of(E, l, nb);
        W[l].assign((size_t)nb[0] * nb[1] * nb[2], 0);
    }
    for (int l = 0; l < E->L; ++l) {
        const Level& V = E->lv[l];
        for (int b = 0; b < V.nreal; ++b) {
            const int* p = &V.bpos[3 * (size_t)b];
            const double v = phi[l][b];
            int want = l;
            if (v > E->sensor_sigma) want = std::min(l + 1, E->L - 1);
            else if (v < E->sensor_c * E->sensor_sigma) want = std::max(l - 1, 0);
            int nb[3];
            lattice_of(E, want, nb);
            if (want > l) {
                for (int k = 0; k < 8; ++k)
                    W[want][bidx(nb, 2 * p[0] + (k & 1), 2 * p[1] + ((k >> 1) & 1), 2 * p[2] + (k >> 2))] = 1;
            } else if (want == l) {
                W[l][bidx(nb, p[0], p[1], p[2])] = 1;
            } else {
                W[want][bidx(nb, p[0] >> 1, p[1] >> 1, p[2] >> 1)] = 1;
            }
        }
    }
    return W;
}

Mask required_from_particle(const AmrEngine* E, const ParticleState& P) {
    int nb[3];
    lattice_of(E, E->L - 1, nb);
    Mask m((size_t)nb[0] * nb[1] * nb[2], 0);
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int)std::floor((P.x[a] - P.r - 1.0) / BS);
        hi[a] = (int)std::floor((P.x[a] + P.r + 1.0) / BS);
    }
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                int p[3] = {x, y, z};
                if (wrap_pos(E, nb, p)) m[bidx(nb, p[0], p[1], p[2])] = 1;
            }
    return dilate(E, m, E->L - 1);
}

Mask required_from_box(const AmrEngine* E) {
    int nb[3];
    lattice_of(E, E->L - 1, nb);
    Mask m((size_t)nb[0] * nb[1] * nb[2], 0);
    for (int z = 0; z < nb[2]; ++z)
        for (int y = 0; y < nb[1]; ++y)
            for (int x = 0; x < nb[0]; ++x) {
                const int p[3] = {x, y, z};
                bool in = true;
                for (int a = 0; a < 3; ++a)
                    if (!((p[a] + 1) * BS > E->box_lo[a] && p[a] * BS < E->box_hi[a])) in = false;
                if (in) m[bidx(nb, x, y, z)] = 1;
            }
    return m;
}

// Smallest per-axis cell distance between [a0, a0+la) and [b0, b0+lb) on an
// axis of n cells (periodic images considered when periodic).
int axis_gap(int a0, int la, int b0, int lb, int n, bool periodic) {
    auto gap = [&](int bs) { return std::max(0, std::max(bs - (a0 + la - 1), a0 - (bs + lb - 1))); };
    int g = gap(b0);
    if (periodic) g = std::min(g, std::min(gap(b0 + n), gap(b0 - n)));
    return g;
}

lbmp_status upload(lbmp_handle* h, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return LBMP_OK;
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return LBMP_ERR_CUDA;
    h->h2d += (long long)bytes;
    return LBMP_OK;
}

void free_level(lbmp_handle* h, Level& V) {
    handle_free(h, V.d_map);
    handle_free(h, V.d_bpos);
    handle_free(h, V.d_nbr);
    handle_free(h, V.d_refined);
    handle_free(h, V.d_host);
    handle_free(h, V.d_glist);
    handle_free(h, V.d_ghost_host);
    handle_free(h, V.d_smask);
    handle_free(h, V.d_pops[0]);
    handle_free(h, V.d_pops[1]);
    handle_free(h, V.d_flags[0]);
    handle_free(h, V.d_flags[1]);
    V = Level();
}

void level_rates(AmrEngine* E, double tau, double magic) {
    for (int l = 0; l < E->L; ++l) {
        Level& V = E->lv[l];
        V.taup = 0.5 + (tau - 0.5) / (double)(1 << (E->L - 1 - l));
        V.taum = 0.5 + magic / (V.taup - 0.5);
    }
}

void kappa_post(const Level& C, const Level& F, double* kp, double* km) {
    *kp = std::fabs(C.taup - 1.0) < 1e-12 ? 1.0 : (F.taup - 1.0) / (2.0 * (C.taup - 1.0));
    *km = std::fabs(C.taum - 1.0) < 1e-12 ? 1.0 : (F.taum - 1.0) / (2.0 * (C.taum - 1.0));
}

// Builds the new layout from the coverage sets, moves the populations over
// and classifies cells.  The old layout is freed afterwards.
lbmp_status build_layout(lbmp_handle* h, const std::vector<Mask>& R) {
    AmrEngine* E = h->amr;
    const int L = E->L;
    amr_drop_graphs(E);
    std::vector<Level> old;
    old.swap(E->lv);
    // the old layout is freed on every way out (after the migration on success)
    struct OldLevels {
        lbmp_handle* h;
        std::vector<Level>& v;
        ~OldLevels() {
            for (auto& V : v) free_level(h, V);
        }
    } old_guard{h, old};
    E->broken = true;   // until the new layout is complete
    E->lv.assign(L, Level());
    for (int l = 0; l < L; ++l) {
        Level& V = E->lv[l];
        for (int a = 0; a < 3; ++a) {
            V.n[a] = E->n0[a] * (1 << l);
            V.nb[a] = V.n[a] / BS;
        }
        const size_t np = (size_t)V.nb[0] * V.nb[1] * V.nb[2];
        V.map.assign(np, -1);
        V.refined = (l + 1 < L) ? parents(E, R[l + 1], l + 1) : Mask(np, 0);
        for (int z = 0; z < V.nb[2]; ++z)
            for (int y = 0; y < V.nb[1]; ++y)
                for (int x = 0; x < V.nb[0]; ++x) {
                    const int i = bidx(V.nb, x, y, z);
                    if (R[l][i] && !V.refined[i]) {
                        V.map[i] = V.nreal++;
                        V.bpos.insert(V.bpos.end(), {x, y, z});
                    }
                }
    }
    // ghost blocks of level l+1: children of real level-l positions holding a
    // level-l cell within Chebyshev distance 2 of a refined position
    for (int l = 0; l + 1 < L; ++l) {
        Level& C = E->lv[l];
        Level& F = E->lv[l + 1];
        for (int z = 0; z < F.nb[2]; ++z)
            for (int y = 0; y < F.nb[1]; ++y)
                for (int x = 0; x < F.nb[0]; ++x) {
                    const int par[3] = {x >> 1, y >> 1, z >> 1};
                    if (C.map[bidx(C.nb, par[0], par[1], par[2])] < 0) continue;
                    const int child[3] = {x, y, z};
                    bool ghost = false;
                    for (int dz = -1; dz <= 1 && !ghost; ++dz)
                        for (int dy = -1; dy <= 1 && !ghost; ++dy)
                            for (int dx = -1; dx <= 1 && !ghost; ++dx) {
                                int p[3] = {par[0] + dx, par[1] + dy, par[2] + dz};
                                if (!wrap_pos(E, C.nb, p)) continue;
                                if (!C.refined[bidx(C.nb, p[0], p[1], p[2])]) continue;
                                int d = 0;
                                for (int a = 0; a < 3; ++a)
                                    d = std::max(d, axis_gap(child[a] * 8, 8, p[a] * BS, BS, C.n[a], E->periodic[a] != 0));
                                if (d <= 2) ghost = true;
                            }
                    if (ghost) {
                        F.map[bidx(F.nb, x, y, z)] = -2 - F.nghost++;
                        F.bpos.insert(F.bpos.end(), {x, y, z});   // appended after all real blocks
                    }
                }
    }
    // neighbour tables
    for (int l = 0; l < L; ++l) {
        Level& V = E->lv[l];
        const int np = V.nreal + V.nghost;
        V.nbr.assign((size_t)np * 27, -1);
        for (int b = 0; b < np; ++b)
            for (int k = 0; k < 27; ++k) {
                int p[3] = {V.bpos[3 * b] + (k % 3) - 1, V.bpos[3 * b + 1] + (k / 3) % 3 - 1, V.bpos[3 * b + 2] + k / 9 - 1};
                if (!wrap_pos(E, V.nb, p)) {
                    V.nbr[(size_t)b * 27 + k] = -2;
                    continue;
                }
                const int m = V.map[bidx(V.nb, p[0], p[1], p[2])];
                V.nbr[(size_t)b * 27 + k] = m >= 0 ? m : (m <= -2 ? V.nreal + (-2 - m) : -1);
            }
    }
    level_rates(E, h->tau, h->magic);
    for (int l = 0; l < L; ++l)   // kernels address a level pool with 32-bit element offsets
        if ((long long)(E->lv[l].nreal + E->lv[l].nghost) * 19 * B3 >= (1LL << 31)) return LBMP_ERR_UNSUPPORTED;
    // device arrays
    const size_t es = esize(h);
    for (int l = 0; l < L; ++l) {
        Level& V = E->lv[l];
        const int np = V.nreal + V.nghost;
        const size_t nmap = V.map.size();
        V.d_map = (int*)handle_alloc(h, sizeof(int) * nmap);
        V.d_refined = (uint8_t*)handle_alloc(h, nmap);
        V.d_bpos = (int*)handle_alloc(h, sizeof(int) * 3 * (size_t)std::max(np, 1));
        V.d_nbr = (int*)handle_alloc(h, sizeof(int) * 27 * (size_t)std::max(np, 1));
        V.d_pops[0] = handle_alloc(h, es * 19 * B3 * (size_t)std::max(np, 1));
        V.d_pops[1] = handle_alloc(h, es * 19 * B3 * (size_t)std::max(np, 1));
        V.d_host = (uint8_t*)handle_alloc(h, (size_t)B3 * std::max(V.nreal, 1));
        if (!V.d_map || !V.d_refined || !V.d_bpos || !V.d_nbr || !V.d_pops[0] || !V.d_pops[1] || !V.d_host)
            return LBMP_ERR_OOM;
        if (l == L - 1) {
            V.d_flags[0] = (uint8_t*)handle_alloc(h, (size_t)B3 * std::max(V.nreal, 1));
            V.d_flags[1] = (uint8_t*)handle_alloc(h, (size_t)B3 * std::max(V.nreal, 1));
            if (!V.d_flags[0] || !V.d_flags[1]) return LBMP_ERR_OOM;
        }
        if (upload(h, V.d_map, V.map.data(), sizeof(int) * nmap) || upload(h, V.d_refined, V.refined.data(), nmap) ||
            upload(h, V.d_bpos, V.bpos.data(), sizeof(int) * V.bpos.size()) ||
            upload(h, V.d_nbr, V.nbr.data(), sizeof(int) * V.nbr.size()))
            return LBMP_ERR_CUDA;
        cudaMemsetAsync(V.d_pops[0], 0, es * 19 * B3 * (size_t)std::max(np, 1), h->stream);
        cudaMemsetAsync(V.d_pops[1], 0, es * 19 * B3 * (size_t)std::max(np, 1), h->stream);
        cudaMemsetAsync(V.d_host, 0, (size_t)B3 * std::max(V.nreal, 1), h->stream);
    }
    // classification and the ghost-cell lists of every finer level, built on
    // the device from the coarser level's host flags (one copy of the per-run
    // counts back to size the lists)
    std::vector<int*> d_runs(L, nullptr);
    std::vector<std::vector<int>> runs(L);
    bool ok = true;
    for (int l = 0; l + 1 < L && ok; ++l) {
        Level& C = E->lv[l];
        if (C.nreal == 0) continue;
        const size_t nr = (size_t)C.nreal * 16;
        d_runs[l] = (int*)handle_alloc(h, sizeof(int) * nr);
        if (!d_runs[l]) {
            ok = false;
            break;
        }
        runs[l].resize(nr);
        k_host_flags<<<(unsigned)nr, 256, 0, h->stream>>>(view(E, C), C.d_host, d_runs[l]);
        if (cudaMemcpyAsync(runs[l].data(), d_runs[l], sizeof(int) * nr, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
            ok = false;
        h->d2h += (long long)(sizeof(int) * nr);
    }
    if (ok && cudaStreamSynchronize(h->stream) != cudaSuccess) ok = false;
    for (int l = 0; l + 1 < L && ok; ++l) {
        Level& C = E->lv[l];
        Level& F = E->lv[l + 1];
        long long n1 = 0;
        for (size_t r = 0; r < runs[l].size(); ++r) n1 += runs[l][r];
        F.nglist = (int)(8 * n1);
        const size_t ng = std::max<size_t>((size_t)F.nglist, 8);
        F.d_glist = (int*)handle_alloc(h, sizeof(int) * ng);
        F.d_ghost_host = (int*)handle_alloc(h, sizeof(int) * (ng / 8));
        F.d_smask = (uint32_t*)handle_alloc(h, sizeof(uint32_t) * ng);
        if (!F.d_glist || !F.d_ghost_host || !F.d_smask) {
            ok = false;
            break;
        }
        if (F.nglist > 0) {
            k_ghost_lists<<<(unsigned)C.nreal * 16, 256, 0, h->stream>>>(view(E, C), C.d_host, d_runs[l], view(E, F),
                                                                           F.d_glist, F.d_ghost_host, h->status);
            k_ghost_smask<<<(unsigned)((F.nglist + 255) / 256), 256, 0, h->stream>>>(
                view(E, C), view(E, F), F.d_glist, F.d_ghost_host, F.nglist, F.d_smask, h->status);
        }
    }
    if (ok && cudaStreamSynchronize(h->stream) != cudaSuccess) ok = false;
    for (int l = 0; l < L; ++l) handle_free(h, d_runs[l]);
    if (!ok) return LBMP_ERR_OOM;
    // populations from the old layout
    if (!old.empty()) {
        with_storage_amr(h->cfg.precision, [&](auto tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            using A = typename Store<S>::A;
            MigrateArgs<S> M;
            M.L = L;
            for (int k = 0; k < L; ++k) {
                M.O[k] = view(E, old[k]);
                M.osrc[k] = (const S*)old[k].d_pops[old[k].cur];
                double kp = 1, km = 1;
                if (k + 1 < L) kappa_post(E->lv[k], E->lv[k + 1], &kp, &km);
                M.kp[k] = (A)kp;
                M.km[k] = (A)km;
            }
            M.rescale = h->cfg.rescale_noneq ? 1 : 0;
            M.scale = (A)(h->cfg.precision == LBMP_FP16 ? std::ldexp(1.0, h->cfg.fp16_scale_log2) : 1.0);
            M.inv_scale = (A)(h->cfg.precision == LBMP_FP16 ? std::ldexp(1.0, -h->cfg.fp16_scale_log2) : 1.0);
            for (int l = 0; l < L; ++l) {
                Level& V = E->lv[l];
                if (V.nreal == 0) continue;
                M.N = view(E, V);
                M.dst = (S*)V.d_pops[V.cur];
                M.l = l;
                k_migrate<S><<<(unsigned)V.nreal * 16, 256, 0, h->stream>>>(M);
            }
        });
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBMP_ERR_CUDA;
    for (auto& V : old) free_level(h, V);   // (the migration above has finished reading them)
    // finest-level flags and boundary cells
    Level& Ff = E->lv[L - 1];
    if (h->has_particle || h->h_ps.present) {
        if (Ff.nreal > 0) {
            k_amr_flags_full<<<(unsigned)Ff.nreal * 16, 256, 0, h->stream>>>(view(E, Ff), Ff.d_flags[0], Ff.d_flags[1], h->d_ps);
            with_storage_amr(h->cfg.precision, [&](auto tag) {
                using S = std::remove_pointer_t<decltype(tag)>;
                k_amr_zero_solid<S><<<(unsigned)Ff.nreal * 16, 256, 0, h->stream>>>((S*)Ff.d_pops[Ff.cur], Ff.d_flags[0]);
            });
        }
        Ff.fcur = 0;
        // boundary cells of the current position (both flag buffers already hold its flags,
        // so the remap pass only marks: nothing is covered or uncovered)
        const unsigned nb = (unsigned)((h->box.cells + REMAP_THREADS - 1) / REMAP_THREADS);
        with_storage_amr(h->cfg.precision, [&](auto tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            using A = typename Store<S>::A;
            k_amr_remap<S><<<nb, REMAP_THREADS, 0, h->stream>>>(view(E, Ff), (S*)Ff.d_pops[Ff.cur], Ff.d_flags[1],
                                                               Ff.d_flags[0], h->box, h->d_ps, (A)1, (A)1,
                                                               h->link_mask, h->link_blocks, h->status, (A)0, nullptr);
        });
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) return LBMP_ERR_CUDA;
    E->broken = false;
    return LBMP_OK;
}

// keep_if_unchanged: a periodic regrid whose block coverage equals the
// current one changes nothing (the populations would be copied onto the
// same blocks and the flags are already those of the current position),
// so the layout, its lists and the captured graphs are kept.
lbmp_status regrid_now(lbmp_handle* h, bool keep_if_unchanged = false, const std::vector<Mask>* wish = nullptr) {
    AmrEngine* E = h->amr;
    int nb[3];
    lattice_of(E, E->L - 1, nb);
    Mask m((size_t)nb[0] * nb[1] * nb[2], 0);
    if (h->h_ps.present) m = required_from_particle(E, h->h_ps);
    if (E->have_box) {
        const Mask mb = required_from_box(E);
        for (size_t i = 0; i < m.size(); ++i) m[i] |= mb[i];
    }
    std::vector<Mask> R = coverage(E, m, wish);
    if (keep_if_unchanged && R == E->cover) return LBMP_OK;
    const lbmp_status s = build_layout(h, R);
    if (s == LBMP_OK) E->cover.swap(R);
    else E->cover.clear();
    return s;
}

template <typename S>
CollideParams<typename Store<S>::A> level_params(const lbmp_handle* h, const Level& V) {
    using A = typename Store<S>::A;
    CollideParams<A> p;
    p.sp = (A)(1.0 / V.taup);
    p.sm = (A)(1.0 / V.taum);
    p.db = (A)bulk_rate_offset(V.taup, h->cfg.bulk_factor);   // Lambda_b fixed on every level, like Lambda
    p.F[0] = p.F[1] = p.F[2] = (A)0;
    p.forced = 0;
    if (h->cfg.precision == LBMP_FP16) {
        p.scale = (A)std::ldexp(1.0, h->cfg.fp16_scale_log2);
        p.inv_scale = (A)std::ldexp(1.0, -h->cfg.fp16_scale_log2);
    } else {
        p.scale = (A)1;
        p.inv_scale = (A)1;
    }
    return p;
}

// Stream of level l's launches: the caller's for the finest level (and for
// every level while per-kernel events are taken), a stream of its own for
// each coarser level.
cudaStream_t level_stream(const lbmp_handle* h, int l) {
    const AmrEngine* E = h->amr;
    return (h->profiling || l == E->L - 1) ? h->stream : E->lstream[l];
}

// One step of level l (sub: which of its parent's two sub-steps, 0 for
// level 0).  Work order and dependencies:
//   - level l+1's stream waits for level l's last update (ev_state[l]):
//     level l+1's sub-steps read level l's current state for their static
//     ghost cells; level l's hosts of that state, and their explosion into
//     level l+1's active ghost cells, were written by level l+1's previous
//     last sub-step, earlier on the same stream (an explicit explosion
//     replaces it after a change outside a step);
//   - level l+1 takes its two sub-steps, the second writing level l's hosts
//     of the new state and their explosion;
//   - level l's update (on its own stream) waits only for the start of
//     level l+1's two sub-steps (ev_xdone[l]), after which no earlier
//     sub-step of level l+1 still reads the buffer it writes; it runs beside
//     them and writes every real cell of level l but the hosts.
// The finest level runs on the caller's stream, so the critical path is the
// chain of finest sub-steps, with the coarser updates beside it.
template <typename S>
void enqueue_advance(lbmp_handle* h, int l, int sub) {
    using A = typename Store<S>::A;
    AmrEngine* E = h->amr;
    const int L = E->L;
    Level& V = E->lv[l];
    const CollideParams<A> P = level_params<S>(h, V);
    const cudaStream_t st = level_stream(h, l);
    if (l + 1 < L) {
        Level& F = E->lv[l + 1];
        const cudaStream_t fs = level_stream(h, l + 1);
        if (fs != st) cudaStreamWaitEvent(fs, E->ev_state[l], 0);
        // the active ghost cells of level l+1 normally hold the hosts' current state already (the
        // previous last sub-step of level l+1 wrote it); after a change of layout or populations
        // outside a step they are exploded here
        if (F.nglist > 0 && !F.ghosts_valid) {
            const unsigned grid = (unsigned)((F.nglist + UPD_THREADS - 1) / UPD_THREADS);
            k_explode<S><<<grid, UPD_THREADS, 0, fs>>>((const S*)V.d_pops[V.cur], (S*)F.d_pops[F.cur], F.d_glist,
                                                       F.d_ghost_host, F.nglist);
            h->launches += 1;
        }
        if (fs != st) cudaEventRecord(E->ev_xdone[l], fs);
        enqueue_advance<S>(h, l + 1, 0);
        enqueue_advance<S>(h, l + 1, 1);
        F.ghosts_valid = true;
        if (fs != st) cudaStreamWaitEvent(st, E->ev_xdone[l], 0);
    }
    UpdateArgs<S> U;
    U.D = view(E, V);
    U.src = (const S*)V.d_pops[V.cur];
    U.dst = (S*)V.d_pops[1 - V.cur];
    U.P = P;
    U.C = U.D;
    U.csrc = nullptr;
    U.ghost_host = nullptr;
    U.smask = nullptr;
    U.cdst = nullptr;
    U.Pc = P;
    U.solid = nullptr;
    U.status = h->status;
    const bool has_fine = l + 1 < L, has_coarse = l > 0;
    const int coalesce = (has_coarse && sub == 1) ? 1 : 0;   // this sub-step ends the coarser level's step
    if (has_coarse) {
        Level& C = E->lv[l - 1];
        U.C = view(E, C);
        U.csrc = (const S*)C.d_pops[C.cur];   // the coarser level's step flips cur after both sub-steps
        U.ghost_host = V.d_ghost_host;
        U.smask = V.d_smask;
        if (coalesce) {
            U.cdst = (S*)C.d_pops[1 - C.cur];
            U.Pc = level_params<S>(h, C);
        }
    }
    const bool coupled = (l == L - 1) && h->has_particle;
    if (coupled) {
        U.solid = V.d_flags[V.fcur];
        // the boundary cells (flag 2) go to k_amr_boundary on the side stream, beside the update
        const LevelView D = view(E, V);
        GridDesc G;
        G.nx = V.n[0];
        G.ny = V.n[1];
        G.nz = V.n[2];
        for (int a = 0; a < 3; ++a) G.periodic[a] = E->periodic[a];
        G.n = (long long)V.n[0] * V.n[1] * V.n[2];
        if (E->remap_pending) {   // the previous remap (side stream) before this update
            cudaStreamWaitEvent(st, E->ev_remap, 0);
            E->remap_pending = false;
        }
        cudaEventRecord(E->ev_fork, st);
        cudaStreamWaitEvent(E->side, E->ev_fork, 0);
        const size_t pre_bytes = sizeof(int) * (size_t)((h->box.cells + LINK_THREADS - 1) / LINK_THREADS + 1);
        k_amr_boundary<S><<<E->boundary_blocks, BNDW_THREADS, pre_bytes, E->side>>>(
            D, U.src, U.dst, U.solid, h->link_mask, h->link_blocks, h->box, P, h->d_ps, h->cfg.boundary == LBMP_CLI ? 1 : 0,
            h->partials, E->d_done, G, h->history, h->cfg.history_capacity, h->status, E->d_frames);
        cudaEventRecord(E->ev_join, E->side);
        h->launches += 1;
    }
    const long long ev0 = profile_mark(h);
    // the active ghost cells streamed (static ones are read from the coarser level)
    const int ng = has_coarse ? V.nglist : 0;
    const int gblocks = (ng + UPD_THREADS - 1) / UPD_THREADS;
    if (V.nreal > 0 || gblocks > 0) {
        const unsigned grid = (unsigned)(V.nreal * (B3 / UPD_THREADS) + gblocks);
        const int* gl = V.d_glist;
        if (has_fine && has_coarse) k_update<S, true, true, false><<<grid, UPD_THREADS, 0, st>>>(U, gl, ng, gblocks, coalesce);
        else if (has_fine) k_update<S, true, false, false><<<grid, UPD_THREADS, 0, st>>>(U, gl, ng, gblocks, coalesce);
        else if (has_coarse && coupled) k_update<S, false, true, true><<<grid, UPD_THREADS, 0, st>>>(U, gl, ng, gblocks, coalesce);
        else if (has_coarse) k_update<S, false, true, false><<<grid, UPD_THREADS, 0, st>>>(U, gl, ng, gblocks, coalesce);
        else if (coupled) k_update<S, false, false, true><<<grid, UPD_THREADS, 0, st>>>(U, gl, ng, gblocks, coalesce);
        else k_update<S, false, false, false><<<grid, UPD_THREADS, 0, st>>>(U, gl, ng, gblocks, coalesce);
        h->launches += 1;
    }
    profile_kernel(h, ev0, profile_mark(h), 38.0 * sizeof(S) * (double)V.nreal * B3, (double)V.nreal * B3);
    h->updates += (long long)V.nreal * B3;
    if (coupled) {
        const LevelView D = view(E, V);
        uint8_t* fnext = V.d_flags[1 - V.fcur];
        const unsigned nl = (unsigned)((h->box.cells + REMAP_THREADS - 1) / REMAP_THREADS);
        // After the second sub-step the next work on this stream is the next explosion into this
        // level, which touches neither the finest real cells, their flags nor the particle, so the
        // remap runs beside it on the side stream (after the boundary kernel there) and the next
        // finest update, or the end of the level-0 step, waits for it.  After the first sub-step the
        // next finest update follows at once.
        const bool beside = has_coarse && sub == 1;
        cudaStream_t rs = st;
        if (beside) {
            cudaEventRecord(E->ev_fork, st);
            cudaStreamWaitEvent(E->side, E->ev_fork, 0);
            rs = E->side;
        } else {
            cudaStreamWaitEvent(st, E->ev_join, 0);
        }
        k_amr_remap<S><<<nl, REMAP_THREADS, 0, rs>>>(D, U.dst, V.d_flags[V.fcur], fnext, h->box, h->d_ps, P.scale,
                                                    P.inv_scale, h->link_mask, h->link_blocks, h->status,
                                                    (A)grad_refill_coef(h->cfg.refill, V.taup), E->d_frames);
        if (beside) {
            cudaEventRecord(E->ev_remap, E->side);
            E->remap_pending = true;
        }
        V.fcur = 1 - V.fcur;
        h->launches += 1;
    }
    if (st != h->stream) cudaEventRecord(E->ev_state[l], st);
    V.cur = 1 - V.cur;
}

}  // namespace

// ================================================================== API
lbmp_status amr_cuda_error(lbmp_handle* h, const char* where) {
    const cudaError_t e = cudaGetLastError();
    h->err = std::string("refined step: ") + where + ": " + cudaGetErrorString(e);
    return LBMP_ERR_CUDA;
}

lbmp_status amr_create(lbmp_handle* h) {
    AmrEngine* E = new (std::nothrow) AmrEngine();
    if (!E) return LBMP_ERR_OOM;
    E->L = h->cfg.levels;
    E->n0[0] = h->cfg.nx;
    E->n0[1] = h->cfg.ny;
    E->n0[2] = h->cfg.nz;
    for (int a = 0; a < 3; ++a) E->periodic[a] = h->cfg.bc[a] == LBMP_PERIODIC ? 1 : 0;
    h->amr = E;
    E->d_done = (int*)handle_alloc(h, sizeof(int));
    if (!E->d_done) return LBMP_ERR_OOM;
    // Priorities: the finest level's chain is the critical path.  Its side stream (the boundary
    // kernel and remap) has the highest: a boundary CTA needs the registers of three update CTAs,
    // and without it the finest update's CTAs take every slot that frees.  Then the captured
    // step's own stream (the finest update), then the coarser levels' streams, each below the next
    // finer one, which fill the SMs the chain leaves.  A graph keeps them with UseNodePriority.
    if (cudaDeviceGetStreamPriorityRange(&E->prio_low, &E->prio_high) != cudaSuccess) return LBMP_ERR_CUDA;
    if (cudaStreamCreateWithPriority(&E->side, cudaStreamNonBlocking, E->prio_high) != cudaSuccess ||
        cudaEventCreateWithFlags(&E->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&E->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&E->ev_remap, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&E->ev_begin, cudaEventDisableTiming) != cudaSuccess)
        return LBMP_ERR_CUDA;
    for (int l = 0; l + 1 < E->L; ++l)   // finer levels first: a level's update gates the next explosion from it
        if (cudaStreamCreateWithPriority(&E->lstream[l], cudaStreamNonBlocking,
                                         std::min(E->prio_low, E->prio_high + 1 + (E->L - 1 - l))) != cudaSuccess ||
            cudaEventCreateWithFlags(&E->ev_state[l], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&E->ev_xdone[l], cudaEventDisableTiming) != cudaSuccess)
            return LBMP_ERR_CUDA;

    if (cudaMemsetAsync(E->d_done, 0, sizeof(int), h->stream) != cudaSuccess) return LBMP_ERR_CUDA;
    return regrid_now(h);
}

void amr_destroy(lbmp_handle* h) {
    if (!h->amr) return;
    amr_drop_graphs(h->amr);
    if (h->amr->capture_stream) cudaStreamDestroy(h->amr->capture_stream);
    if (h->amr->side) cudaStreamDestroy(h->amr->side);
    if (h->amr->ev_fork) cudaEventDestroy(h->amr->ev_fork);
    if (h->amr->ev_join) cudaEventDestroy(h->amr->ev_join);
    if (h->amr->ev_remap) cudaEventDestroy(h->amr->ev_remap);
    if (h->amr->ev_begin) cudaEventDestroy(h->amr->ev_begin);
    for (int l = 0; l < MAXL; ++l) {
        if (h->amr->lstream[l]) cudaStreamDestroy(h->amr->lstream[l]);
        if (h->amr->ev_state[l]) cudaEventDestroy(h->amr->ev_state[l]);
        if (h->amr->ev_xdone[l]) cudaEventDestroy(h->amr->ev_xdone[l]);
    }

    for (auto& V : h->amr->lv) free_level(h, V);
    handle_free(h, h->amr->d_sensor);
    delete h->amr;
    h->amr = nullptr;
}

lbmp_status amr_add_sphere(lbmp_handle* h) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    const Level& F = E->lv[E->L - 1];
    // box around the sphere at the finest level (as in the uniform engine)
    BoxDesc& B = h->box;
    B.R = (int)std::ceil(h->h_ps.r) + 3;
    B.cells = 1;
    for (int a = 0; a < 3; ++a) {
        B.E[a] = 2 * B.R + 2;
        if (E->periodic[a] && B.E[a] >= F.n[a]) B.E[a] = F.n[a];
        B.cells *= B.E[a];
    }
    const double h3 = 0.5 * std::sqrt(3.0);
    const double ro = h->h_ps.r + std::sqrt(2.0) + h3, ri = std::max(0.0, h->h_ps.r - h3);
    const double shell = 4.0 / 3.0 * M_PI * (ro * ro * ro - ri * ri * ri);
    h->list_cap = (int)std::min<double>((double)B.cells, std::ceil(shell) + 64.0);
    h->list = (int*)handle_alloc(h, sizeof(int) * (size_t)h->list_cap);
    E->boundary_blocks = (int)((B.cells + BND_CHUNK - 1) / BND_CHUNK);
    h->partials = (double*)handle_alloc(h, sizeof(double) * 6 * (size_t)E->boundary_blocks);
    if (!E->d_frames) E->d_frames = (PFrames*)handle_alloc(h, sizeof(PFrames));
    if (!E->d_frames) return LBMP_ERR_OOM;
    h->link_mask = (uint8_t*)handle_alloc(h, (size_t)B.cells);
    h->link_blocks = (int*)handle_alloc(h, sizeof(int) * (size_t)((B.cells + LINK_THREADS - 1) / LINK_THREADS));
    if (!h->list || !h->partials || !h->link_mask || !h->link_blocks) return LBMP_ERR_OOM;
    // the boundary kernel keeps a prefix of the remap's run counts in dynamic shared memory
    const int pre_bytes = (int)(sizeof(int) * ((B.cells + LINK_THREADS - 1) / LINK_THREADS + 1));
    bool attr_ok = true;
    with_storage_amr(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        attr_ok = cudaFuncSetAttribute(k_amr_boundary<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       std::max(pre_bytes, 1024)) == cudaSuccess;
    });
    if (!attr_ok) return amr_cuda_error(h, "sphere too large for the boundary kernel's shared memory");
    if (cudaMemcpyAsync(h->d_ps, &h->h_ps, sizeof(ParticleState), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return LBMP_ERR_CUDA;
    h->h2d += sizeof(ParticleState);
    h->has_particle = true;
    h->frames_stale = true;
    amr_invalidate_ghosts(E);
    return regrid_now(h);
}

lbmp_status amr_refine_box(lbmp_handle* h, const double lo[3], const double hi[3]) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    E->have_box = true;
    for (int a = 0; a < 3; ++a) {
        E->box_lo[a] = lo[a];
        E->box_hi[a] = hi[a];
    }
    return regrid_now(h);
}

namespace {

// Sensor value of every real block of every level (k_block_sensor, one
// launch per level into one device array, one copy back).
lbmp_status sensor_values(lbmp_handle* h, std::vector<std::vector<double>>& phi) {
    AmrEngine* E = h->amr;
    size_t total = 0;
    for (const Level& V : E->lv) total += (size_t)V.nreal;
    phi.assign(E->L, std::vector<double>());
    if (total == 0) return LBMP_OK;
    if (total > E->sensor_cap) {
        handle_free(h, E->d_sensor);
        E->d_sensor = (double*)handle_alloc(h, sizeof(double) * total);
        E->sensor_cap = E->d_sensor ? total : 0;
        if (!E->d_sensor) return LBMP_ERR_OOM;
    }
    bool launched = true;
    with_storage_amr(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using A = typename Store<S>::A;
        const size_t smem = 3 * (size_t)B3 * sizeof(A);
        if (cudaFuncSetAttribute(k_block_sensor<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            launched = false;
            return;
        }
        const A inv = (A)(h->cfg.precision == LBMP_FP16 ? std::ldexp(1.0, -h->cfg.fp16_scale_log2) : 1.0);
        size_t off = 0;
        for (int l = 0; l < E->L; ++l) {
            const Level& V = E->lv[l];
            if (V.nreal == 0) continue;
            const double sz = (double)(1 << (E->L - 1 - l));   // cell size in finest units
            k_block_sensor<S><<<(unsigned)V.nreal, SENSOR_THREADS, smem, h->stream>>>(
                (const S*)V.d_pops[V.cur], inv, (A)sz, std::pow(sz, 1.5), E->d_sensor + off);
            h->launches += 1;
            off += (size_t)V.nreal;
        }
    });
    if (!launched || cudaGetLastError() != cudaSuccess) return amr_cuda_error(h, "k_block_sensor");
    std::vector<double> all(total);
    if (cudaMemcpyAsync(all.data(), E->d_sensor, sizeof(double) * total, cudaMemcpyDeviceToHost, h->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return amr_cuda_error(h, "sensor copy");
    h->d2h += (long long)(sizeof(double) * total);
    size_t off = 0;
    for (int l = 0; l < E->L; ++l) {
        const int n = E->lv[l].nreal;
        phi[l].assign(all.begin() + off, all.begin() + off + n);
        off += (size_t)n;
    }
    return LBMP_OK;
}

}  // namespace

lbmp_status amr_regrid(lbmp_handle* h) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    if (h->has_particle) {
        if (cudaMemcpyAsync(&h->h_ps, h->d_ps, sizeof(ParticleState), cudaMemcpyDeviceToHost, h->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return LBMP_ERR_CUDA;
        h->d2h += sizeof(ParticleState);
    }
    if (E->sensor_sigma > 0.0) {
        std::vector<std::vector<double>> phi;
        const lbmp_status s = sensor_values(h, phi);
        if (s != LBMP_OK) return s;
        const std::vector<Mask> wish = sensor_wishes(E, phi);
        return regrid_now(h, true, &wish);
    }
    return regrid_now(h, true);
}

lbmp_status amr_set_sensor(lbmp_handle* h, double sigma, double c) {
    AmrEngine* E = h->amr;
    E->sensor_sigma = sigma;
    E->sensor_c = sigma > 0.0 ? c : 0.0;
    return LBMP_OK;
}

lbmp_status amr_block_sensor(lbmp_handle* h, int level, double* out, size_t cap, size_t* n) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    if (level < 0 || level >= E->L) return LBMP_ERR_INVALID_ARG;
    *n = (size_t)E->lv[level].nreal;
    if (!out || cap == 0 || *n == 0) return LBMP_OK;
    std::vector<std::vector<double>> phi;
    const lbmp_status s = sensor_values(h, phi);
    if (s != LBMP_OK) return s;
    for (size_t b = 0; b < *n && b < cap; ++b) out[b] = phi[level][b];
    return LBMP_OK;
}

lbmp_status amr_init_fluid(lbmp_handle* h, double rho, const double u[3], double amp, int dir, int axis) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    amr_invalidate_ghosts(E);
    const double Lax = (double)E->lv[E->L - 1].n[axis];
    with_storage_amr(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using A = typename Store<S>::A;
        const A scale = (A)(h->cfg.precision == LBMP_FP16 ? std::ldexp(1.0, h->cfg.fp16_scale_log2) : 1.0);
        for (int l = 0; l < E->L; ++l) {
            Level& V = E->lv[l];
            if (V.nreal == 0) continue;
            const uint8_t* solid = (l == E->L - 1 && h->has_particle) ? V.d_flags[V.fcur] : nullptr;
            k_amr_init<S><<<(unsigned)V.nreal * 16, 256, 0, h->stream>>>(view(E, V), (S*)V.d_pops[V.cur], solid, rho, u[0], u[1], u[2],
                                                           amp, dir, axis, (double)(1 << (E->L - 1 - l)), Lax, scale);
        }
    });
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) return LBMP_ERR_CUDA;
    return LBMP_OK;
}

lbmp_status amr_step(lbmp_handle* h, int n) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    level_rates(E, h->tau, h->magic);
    if (E->graph_tau != h->tau) {
        amr_drop_graphs(E);
        E->graph_tau = h->tau;
    }
    if (h->has_particle && h->frames_stale) {   // the host changed the record: its frames first
        k_pframes<<<1, 128, 0, h->stream>>>(h->d_ps, E->d_frames, view(E, E->lv[E->L - 1]), h->box);
        h->launches += 1;
        h->frames_stale = false;
    }
    // k consecutive level-0 steps.  The coarser levels' streams join here and rejoin the caller's
    // stream at the end; between two steps of one call the stream events alone order the work, so
    // the second step's coarser updates can start beside the first step's last finest sub-steps.
    auto enqueue = [&](int k) {
        const bool fork = !h->profiling && E->L > 1;
        if (fork) {
            cudaEventRecord(E->ev_begin, h->stream);
            for (int l = 0; l + 1 < E->L; ++l) {
                cudaStreamWaitEvent(E->lstream[l], E->ev_begin, 0);
                cudaEventRecord(E->ev_state[l], E->lstream[l]);
            }
        }
        for (int j = 0; j < k; ++j)
            with_storage_amr(h->cfg.precision, [&](auto tag) {
                using S = std::remove_pointer_t<decltype(tag)>;
                enqueue_advance<S>(h, 0, 0);
            });
        if (E->remap_pending) {   // the steps end with everything on the caller's stream
            cudaStreamWaitEvent(h->stream, E->ev_remap, 0);
            E->remap_pending = false;
        }
        if (fork)
            for (int l = 0; l + 1 < E->L; ++l) cudaStreamWaitEvent(h->stream, E->ev_state[l], 0);
    };
    auto regrid_due = [&](long long steps) {
        return h->cfg.regrid_interval > 0 && (h->has_particle || E->sensor_sigma > 0.0) &&
               steps % h->cfg.regrid_interval == 0;
    };
    for (int i = 0; i < n;) {
        // two steps per graph where no regrid falls between them (one per profiled step)
        const int k = (!h->profiling && n - i >= 2 && !regrid_due(E->coarse_steps + 1)) ? 2 : 1;
        if (h->profiling) {   // per-kernel events: plain launches
            const long long ev_step = profile_mark(h);
            enqueue(k);
            profile_step(h, ev_step, profile_mark(h));
        } else if (!amr_ghosts_valid(E)) {   // a step that explodes ghost cells is not the one a graph repeats
            enqueue(k);
        } else {
            const int par = E->lv[0].cur;
            cudaGraphExec_t& gx = E->graph[k - 1][par];
            if (!gx) {
                // capture the steps on a private stream (the caller's stream
                // may be the legacy default stream, which cannot be
                // captured); enqueue() advances the host-side buffer indices
                // exactly as the replayed graph will
                if (!E->capture_stream &&
                    cudaStreamCreateWithPriority(&E->capture_stream, cudaStreamNonBlocking,
                                                 std::min(E->prio_high + 1, E->prio_low)) != cudaSuccess)
                    return amr_cuda_error(h, "cudaStreamCreate");
                const long long l0 = h->launches, u0 = h->updates;
                cudaStream_t user = h->stream;
                h->stream = E->capture_stream;
                cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed);
                if (e != cudaSuccess) {
                    h->stream = user;
                    return amr_cuda_error(h, "cudaStreamBeginCapture");
                }
                enqueue(k);
                cudaGraph_t g = nullptr;
                e = cudaStreamEndCapture(h->stream, &g);
                h->stream = user;
                if (e != cudaSuccess) return amr_cuda_error(h, "cudaStreamEndCapture");
                cudaGraphExec_t ge = nullptr;
                e = cudaGraphInstantiateWithFlags(&ge, g, cudaGraphInstantiateFlagUseNodePriority);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return amr_cuda_error(h, "cudaGraphInstantiate");
                gx = ge;
                E->graph_launches[k - 1] = h->launches - l0;
                E->graph_updates[k - 1] = h->updates - u0;
                if (cudaGraphLaunch(ge, h->stream) != cudaSuccess) return amr_cuda_error(h, "cudaGraphLaunch");
            } else {
                if (cudaGraphLaunch(gx, h->stream) != cudaSuccess) return amr_cuda_error(h, "cudaGraphLaunch");
                // the same buffer flips as the captured enqueue: level l flips k 2^l times
                if (k & 1) E->lv[0].cur = 1 - E->lv[0].cur;
                h->launches += E->graph_launches[k - 1];
                h->updates += E->graph_updates[k - 1];
            }
        }
        E->coarse_steps += k;
        h->steps += k;
        i += k;
        if (cudaGetLastError() != cudaSuccess) return amr_cuda_error(h, "kernel launch");
        if (regrid_due(E->coarse_steps)) {
            const lbmp_status s = amr_regrid(h);
            if (s != LBMP_OK) return s;
        }
    }
    return LBMP_OK;
}

// ------------------------------------------------------------ checkpoint
namespace {
bool ck_put(FILE* f, const void* p, size_t n) { return n == 0 || std::fwrite(p, 1, n, f) == n; }
bool ck_get(FILE* f, void* p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }
}  // namespace

// Refined part of a checkpoint: the block coverage of every level, every
// level's real-block populations (current buffer, storage type), then the
// level-0 step count, the sensor and the refined box.
lbmp_status amr_save(lbmp_handle* h, FILE* f) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    const int32_t L = E->L;
    bool ok = ck_put(f, &L, sizeof(L));
    for (int l = 0; l < L && ok; ++l) {
        const int64_t n = (int64_t)E->cover[l].size();
        ok = ck_put(f, &n, sizeof(n)) && ck_put(f, E->cover[l].data(), (size_t)n);
    }
    const size_t es = esize(h);
    for (int l = 0; l < L && ok; ++l) {
        const Level& V = E->lv[l];
        const int32_t nr = V.nreal;
        const size_t bytes = es * 19 * B3 * (size_t)V.nreal;
        std::vector<unsigned char> buf(bytes);
        ok = ck_put(f, &nr, sizeof(nr)) &&
             (bytes == 0 || cudaMemcpy(buf.data(), V.d_pops[V.cur], bytes, cudaMemcpyDeviceToHost) == cudaSuccess) &&
             ck_put(f, buf.data(), bytes);
    }
    const int64_t cs = E->coarse_steps;
    const int32_t hb = E->have_box ? 1 : 0;
    ok = ok && ck_put(f, &cs, sizeof(cs)) && ck_put(f, &E->sensor_sigma, sizeof(double)) &&
         ck_put(f, &E->sensor_c, sizeof(double)) && ck_put(f, &hb, sizeof(hb)) && ck_put(f, E->box_lo, sizeof(E->box_lo)) &&
         ck_put(f, E->box_hi, sizeof(E->box_hi));
    return ok ? LBMP_OK : LBMP_ERR_CUDA;
}

// Rebuilds the saved hierarchy (the finest flags follow from the restored
// sphere position) and restores every level's populations.
lbmp_status amr_load(lbmp_handle* h, FILE* f) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    int32_t L = 0;
    if (!ck_get(f, &L, sizeof(L)) || L != E->L) return LBMP_ERR_INVALID_ARG;
    std::vector<Mask> R(L);
    for (int l = 0; l < L; ++l) {
        int nb[3];
        lattice_of(E, l, nb);
        int64_t n = 0;
        if (!ck_get(f, &n, sizeof(n)) || n != (int64_t)nb[0] * nb[1] * nb[2]) return LBMP_ERR_INVALID_ARG;
        R[l].resize((size_t)n);
        if (!ck_get(f, R[l].data(), (size_t)n)) return LBMP_ERR_INVALID_ARG;
    }
    const lbmp_status s = build_layout(h, R);
    if (s != LBMP_OK) return s;
    E->cover = R;
    const size_t es = esize(h);
    for (int l = 0; l < L; ++l) {
        Level& V = E->lv[l];
        int32_t nr = 0;
        if (!ck_get(f, &nr, sizeof(nr)) || nr != V.nreal) return LBMP_ERR_INVALID_ARG;
        const size_t bytes = es * 19 * B3 * (size_t)V.nreal;
        std::vector<unsigned char> buf(bytes);
        if (!ck_get(f, buf.data(), bytes)) return LBMP_ERR_INVALID_ARG;
        if (bytes && cudaMemcpy(V.d_pops[V.cur], buf.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return LBMP_ERR_CUDA;
        h->h2d += (long long)bytes;
    }
    int64_t cs = 0;
    int32_t hb = 0;
    if (!ck_get(f, &cs, sizeof(cs)) || !ck_get(f, &E->sensor_sigma, sizeof(double)) ||
        !ck_get(f, &E->sensor_c, sizeof(double)) || !ck_get(f, &hb, sizeof(hb)) || !ck_get(f, E->box_lo, sizeof(E->box_lo)) ||
        !ck_get(f, E->box_hi, sizeof(E->box_hi)))
        return LBMP_ERR_INVALID_ARG;
    E->coarse_steps = cs;
    E->have_box = hb != 0;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? LBMP_OK : LBMP_ERR_CUDA;
}

lbmp_status amr_level_shape(lbmp_handle* h, int level, int out[3]) {
    AmrEngine* E = h->amr;
    if (level < 0 || level >= E->L) return LBMP_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) out[a] = E->lv[level].n[a];
    return LBMP_OK;
}

lbmp_status amr_block_map(lbmp_handle* h, int level, int32_t* out, size_t cap, size_t* n) {
    AmrEngine* E = h->amr;
    if (level < 0 || level >= E->L) return LBMP_ERR_INVALID_ARG;
    const Level& V = E->lv[level];
    *n = V.map.size();
    if (out)
        for (size_t i = 0; i < V.map.size() && i < cap; ++i)
            out[i] = V.map[i] >= 0 ? V.map[i] : (V.map[i] <= -2 ? -2 : -1);
    return LBMP_OK;
}

lbmp_status amr_level_cells(lbmp_handle* h, int level, int32_t* xyz, double* g, size_t cap, size_t* n) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    if (level < 0 || level >= E->L) return LBMP_ERR_INVALID_ARG;
    Level& V = E->lv[level];
    const size_t cells = (size_t)V.nreal * B3;
    *n = cells;
    if (!xyz || !g || cap < cells || cells == 0) return LBMP_OK;
    int32_t* dx = (int32_t*)handle_alloc(h, sizeof(int32_t) * 3 * cells);
    double* dg = (double*)handle_alloc(h, sizeof(double) * 19 * cells);
    if (!dx || !dg) {
        handle_free(h, dx);
        handle_free(h, dg);
        return LBMP_ERR_OOM;
    }
    with_storage_amr(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using A = typename Store<S>::A;
        const A inv = (A)(h->cfg.precision == LBMP_FP16 ? std::ldexp(1.0, -h->cfg.fp16_scale_log2) : 1.0);
        k_amr_export<S><<<(unsigned)V.nreal * 16, 256, 0, h->stream>>>(view(E, V), (const S*)V.d_pops[V.cur], dx, dg, inv);
    });
    cudaError_t e = cudaMemcpyAsync(xyz, dx, sizeof(int32_t) * 3 * cells, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g, dg, sizeof(double) * 19 * cells, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->d2h += (long long)(sizeof(int32_t) * 3 + sizeof(double) * 19) * (long long)cells;
    handle_free(h, dx);
    handle_free(h, dg);
    return e == cudaSuccess ? LBMP_OK : LBMP_ERR_CUDA;
}

lbmp_status amr_level_flags(lbmp_handle* h, int level, uint8_t* out, size_t cap, size_t* n) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    if (level < 0 || level >= E->L) return LBMP_ERR_INVALID_ARG;
    Level& V = E->lv[level];
    const size_t cells = (size_t)V.nreal * B3;
    *n = cells;
    if (!out || cap < cells || cells == 0) return LBMP_OK;
    if (level != E->L - 1 || !h->has_particle) {
        std::memset(out, 0, cells);
        return LBMP_OK;
    }
    cudaError_t e = cudaMemcpyAsync(out, V.d_flags[V.fcur], cells, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    h->d2h += (long long)cells;
    return e == cudaSuccess ? LBMP_OK : LBMP_ERR_CUDA;
}

lbmp_status amr_links(lbmp_handle* h, int64_t* cell, int32_t* q, double* delta, size_t cap, size_t* n) {
    if (h->amr->broken) return LBMP_ERR_OOM;   // an earlier rebuild of the hierarchy failed
    AmrEngine* E = h->amr;
    *n = 0;
    if (!h->has_particle) return LBMP_OK;
    // the step keeps the boundary cells as a mask in box order; compact it for the export
    {
        const Level& Vf = E->lv[E->L - 1];
        const unsigned nl = (unsigned)((h->box.cells + LINK_THREADS - 1) / LINK_THREADS);
        k_amr_links_emit<<<nl, LINK_THREADS, 0, h->stream>>>(view(E, Vf), h->link_mask, h->link_blocks, h->box,
                                                             h->d_ps, h->list, h->count, h->list_cap, h->status);
    }
    int cnt = 0;
    if (cudaMemcpyAsync(&cnt, h->count, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return LBMP_ERR_CUDA;
    if (cnt == 0) return LBMP_OK;
    Level& V = E->lv[E->L - 1];
    int64_t* dc = (int64_t*)handle_alloc(h, sizeof(int64_t) * 18 * (size_t)cnt);
    int32_t* dq = (int32_t*)handle_alloc(h, sizeof(int32_t) * 18 * (size_t)cnt);
    double* dd = (double*)handle_alloc(h, sizeof(double) * 18 * (size_t)cnt);
    if (!dc || !dq || !dd) {
        handle_free(h, dc);
        handle_free(h, dq);
        handle_free(h, dd);
        return LBMP_ERR_OOM;
    }
    k_amr_export_links<<<(cnt + 127) / 128, 128, 0, h->stream>>>(view(E, V), V.d_flags[V.fcur], h->list, h->count,
                                                                 h->d_ps, dc, dq, dd);
    std::vector<int64_t> hc((size_t)cnt * 18);
    std::vector<int32_t> hq((size_t)cnt * 18);
    std::vector<double> hd((size_t)cnt * 18);
    cudaError_t e = cudaMemcpyAsync(hc.data(), dc, sizeof(int64_t) * hc.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hq.data(), dq, sizeof(int32_t) * hq.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd.data(), dd, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    handle_free(h, dc);
    handle_free(h, dq);
    handle_free(h, dd);
    if (e != cudaSuccess) return LBMP_ERR_CUDA;
    size_t m = 0;
    for (size_t s = 0; s < hq.size(); ++s) {
        if (hq[s] < 0) continue;
        if (m < cap) {
            if (cell) cell[m] = hc[s];
            if (q) q[m] = hq[s];
            if (delta) delta[m] = hd[s];
        }
        ++m;
    }
    *n = m;
    return LBMP_OK;
}

long long amr_cell_updates_per_coarse_step(const lbmp_handle* h) {
    const AmrEngine* E = h->amr;
    long long u = 0;
    for (int l = 0; l < E->L; ++l) u += (long long)E->lv[l].nreal * B3 * (1LL << l);
    return u;
}

int amr_launches_per_coarse_step(const lbmp_handle* h) {
    const AmrEngine* E = h->amr;
    int per = 0;
    for (int l = E->L - 1; l >= 0; --l) {
        // the update (the explosions into finer levels happen only after a change outside a step)
        int own = 1 + ((l == E->L - 1 && h->has_particle) ? 2 : 0);
        per = own + 2 * per;
    }
    return per;
}

}  // namespace lbmp
