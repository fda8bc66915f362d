// Internal declarations shared by the host API and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <cmath>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/lbmp.h"
#include "lattice.cuh"

namespace lbmp {

struct GridDesc {
    int nx, ny, nz;
    int periodic[3];
    long long n;   // nx * ny * nz
    // velocities of the no-slip domain walls [axis][0 low face, 1 high face] (uniform grids);
    // moving != 0 when any is nonzero
    double uw[3][2][3] = {};
    int moving = 0;
};

// Moving-wall term of a pull from beyond a no-slip domain wall half-way
// between cells: bounce-back plus Ladd's 2 w_q rho_0 c_q.u_w / c_s^2 = 6 w_q
// c_q.u_w (the CLI rule of Sec. 2.3 at delta = 1/2), summed over the faces
// the link from the cell xyz against c_q crosses.
template <typename A>
__device__ __forceinline__ A wall_term(const GridDesc& G, int q, const int xyz[3]) {
    if (!G.moving) return A(0);
    const int n3[3] = {G.nx, G.ny, G.nz};
    const int c3[3] = {cx(q), cy(q), cz(q)};
    A t = A(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int s = xyz[a] - c3[a];
        if (G.periodic[a] || (s >= 0 && s < n3[a])) continue;
        const double* u = G.uw[a][s < 0 ? 0 : 1];
        t += A(6) * wgt<A>(q) * (A(c3[0]) * A(u[0]) + A(c3[1]) * A(u[1]) + A(c3[2]) * A(u[2]));
    }
    return t;
}

// Collision parameters in the arithmetic precision A of the storage type.
template <typename A>
struct CollideParams {
    A sp, sm;          // s+ = 1/tau, s- from the magic parameter
    A db;              // MRT: s_b - s+ (bulk factor Lambda_b != 1), 0 for TRT
    A F[3];            // fluid body force
    int forced;
    A scale, inv_scale;   // FP16 storage scaling (1 otherwise)
};

// Axis-aligned box of cells around the sphere, fixed extent, origin read
// from the particle state on the device.
struct BoxDesc {
    int R;        // half width in cells
    int E[3];     // extent per axis (clamped to the domain for periodic axes)
    long long cells;
};

// Grid of the warp-per-cell boundary kernels (8 warps per block, grid-stride
// over the boundary list); also the number of force partials.  The list
// capacity is about three times the boundary cells of the sphere, so one
// block per 32 entries of capacity gives each warp one or two cells: enough
// warps to hide the gathers' latency, few enough that the per-block set-up
// and the FP64 reduction stay small.  At most eight blocks per SM.
inline int boundary_grid(int capacity) {
    const int b = (capacity + 31) / 32;
    return b < 1 ? 1 : (b > 1216 ? 1216 : b);
}

// Launchers (uniform.cu).  All are asynchronous on `stream`.
template <typename S>
void launch_bulk(const S* src, S* dst, const GridDesc& g, const CollideParams<typename Store<S>::A>& p,
                 int* status, cudaStream_t stream);
template <typename S>
void launch_boundary(const S* src, S* dst, const uint8_t* flags, const int* list, const int* count, int max_cells,
                     const GridDesc& g, const CollideParams<typename Store<S>::A>& p, const ParticleState* ps,
                     int cli, double* partials, int* nblocks_out, int* status, cudaStream_t stream);
void launch_particle_update(ParticleState* ps, const double* partials, int nblocks, const GridDesc& g,
                            double* history, int hist_cap, int* status, cudaStream_t stream);
void launch_flags_full(uint8_t* flags, const GridDesc& g, const ParticleState* ps, cudaStream_t stream);
void launch_flags_box(uint8_t* flags_next, const GridDesc& g, const BoxDesc& b, const ParticleState* ps,
                      cudaStream_t stream);
template <typename S>
void launch_refill(S* pops, const uint8_t* flags_cur, const uint8_t* flags_next, const GridDesc& g,
                   const BoxDesc& b, const ParticleState* ps, typename Store<S>::A scale,
                   typename Store<S>::A inv_scale, typename Store<S>::A gcoef, cudaStream_t stream);
// Boundary-cell list of the box; mask (b.cells bytes) and block_count
// (ceil(b.cells / 256) ints) are scratch.
void launch_build_links(const uint8_t* flags, const GridDesc& g, const BoxDesc& b, const ParticleState* ps,
                        uint8_t* mask, int* block_count, int* list, int* count, int capacity, int* status,
                        cudaStream_t stream);
void launch_export_links(const uint8_t* flags, const int* list, const int* count, int max_cells,
                         const GridDesc& g, const ParticleState* ps, int cli, int32_t* q_out, double* delta_out,
                         cudaStream_t stream);
template <typename S>
void launch_init_equilibrium(S* pops, const uint8_t* flags, const GridDesc& g, double rho, const double u[3],
                             const double* u_field, typename Store<S>::A scale, cudaStream_t stream);
template <typename S>
void launch_to_f64(const S* pops, double* out, long long count, typename Store<S>::A inv_scale,
                   cudaStream_t stream);
template <typename S>
void launch_from_f64(const double* in, S* pops, long long count, typename Store<S>::A scale, cudaStream_t stream);
template <typename S>
void launch_gather(const S* pops, long long ncells, const int64_t* cells, long long n, double* out,
                   typename Store<S>::A inv_scale, cudaStream_t stream);
template <typename S>
void launch_zero_solid(S* pops, const uint8_t* flags, const GridDesc& g, cudaStream_t stream);

struct AmrEngine;
struct BatchEngine;
struct AdjointEngine;

// Profiling events on the handle's stream (api.cu); -1 when profiling is off.
long long profile_mark(lbmp_handle* h);
void profile_kernel(lbmp_handle* h, long long start, long long end, double bytes, double updates);
void profile_step(lbmp_handle* h, long long start, long long end);

// Device allocation through the handle's allocator (api.cu).
void* handle_alloc(lbmp_handle* h, size_t bytes);
void handle_free(lbmp_handle* h, void* p);

}  // namespace lbmp

// One simulation (opaque to callers of the C ABI).
struct lbmp_handle {
    lbmp_config cfg;
    lbmp::GridDesc G;
    cudaStream_t stream = nullptr;
    void* pops[2] = {nullptr, nullptr};
    int cur = 0;                         // pops[cur] holds the post-collision field
    uint8_t* flags[2] = {nullptr, nullptr};
    int fcur = 0;                        // flags[fcur] are the flags of pops[cur]
    int* list = nullptr;                 // boundary cells
    int* count = nullptr;
    int list_cap = 0;
    uint8_t* link_mask = nullptr;        // scratch of the link compaction (one byte per box cell)
    int* link_blocks = nullptr;          // scratch: per-block counts
    double* partials = nullptr;
    int partial_blocks = 0;
    lbmp::ParticleState* d_ps = nullptr;
    lbmp::ParticleState h_ps;                  // host copy of the parameters
    double* history = nullptr;
    int* status = nullptr;
    lbmp::BoxDesc box;
    bool has_particle = false;
    bool frames_stale = true;            // the host changed the particle record since the refined step formed its frames
    bool ps_current = false;             // h_ps equals the device record (read with the status after a step)
    double tau = 0.6, magic = 3.0 / 16.0;
    double body_force[3] = {0, 0, 0};
    long long steps = 0, updates = 0, launches = 0, h2d = 0, d2h = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;    // events of the current measurement
    size_t ev_used = 0;
    // (start, end) event indices of stream-collide launches with their algorithmic bytes and cell updates
    std::vector<std::pair<size_t, size_t>> prof_kernel;
    std::vector<double> prof_bytes, prof_updates;
    std::vector<std::pair<size_t, size_t>> prof_step;
    std::vector<std::pair<void*, size_t>> allocations;
    std::string err;
    lbmp::AmrEngine* amr = nullptr;     // refined hierarchy (levels > 1), else null
    lbmp::BatchEngine* batch = nullptr; // batched sweep, else null
    lbmp::AdjointEngine* adj = nullptr; // drag adjoint workspace, else null
};

namespace lbmp {

// s- from the magic parameter: Lambda = (1/s+ - 1/2)(1/s- - 1/2)  (Sec. 2.1)
inline void relaxation_rates(double tau, double magic, double* sp, double* sm) {
    *sp = 1.0 / tau;
    *sm = 1.0 / (0.5 + magic / (tau - 0.5));
}

// Coefficient of Grad's refill term for relaxation time tau (-3 (1 - s+)/s+,
// see refill_strain and grad_term), or 0 for the equilibrium refill.
inline double grad_refill_coef(int refill, double tau) {
    if (refill != LBMP_REFILL_GRAD) return 0.0;
    const double sp = 1.0 / tau;
    return -3.0 * (1.0 - sp) / sp;
}

// MRT bulk rate from the bulk factor: Lambda_b = (1/s_b - 1/2)/(1/s_nu - 1/2)
// (Sec. 2.1); returns s_b - s+, exactly 0 for Lambda_b = 1 (TRT).
inline double bulk_rate_offset(double tau, double bulk) {
    if (bulk == 1.0) return 0.0;
    return 1.0 / (0.5 + bulk * (tau - 0.5)) - 1.0 / tau;
}

template <typename A>
inline CollideParams<A> collide_params(const lbmp_handle* h) {
    CollideParams<A> p;
    double sp, sm;
    relaxation_rates(h->tau, h->magic, &sp, &sm);
    p.sp = (A)sp;
    p.sm = (A)sm;
    p.db = (A)bulk_rate_offset(h->tau, h->cfg.bulk_factor);
    for (int a = 0; a < 3; ++a) p.F[a] = (A)h->body_force[a];
    p.forced = (h->body_force[0] != 0.0 || h->body_force[1] != 0.0 || h->body_force[2] != 0.0) ? 1 : 0;
    if (h->cfg.precision == LBMP_FP16) {
        p.scale = (A)std::ldexp(1.0, h->cfg.fp16_scale_log2);
        p.inv_scale = (A)std::ldexp(1.0, -h->cfg.fp16_scale_log2);
    } else {
        p.scale = (A)1;
        p.inv_scale = (A)1;
    }
    return p;
}

}  // namespace lbmp

