// Host side of the C ABI declared in include/lbmp.h: handle management,
// parameter conversion and the per-step launch sequence of Algorithm 1.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "adjoint.h"
#include "amr.h"
#include "batch.h"

using namespace lbmp;

namespace {

thread_local std::string g_create_error;

size_t elem_size(int prec) { return prec == LBMP_FP64 ? 8 : (prec == LBMP_FP32 ? 4 : 2); }

lbmp_status fail(lbmp_handle* h, lbmp_status s, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return s;
}

lbmp_status cuda_fail(lbmp_handle* h, cudaError_t e, const char* where) {
    return fail(h, LBMP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBMP_CK(h, call)                                          \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);  \
    } while (0)

void* dev_alloc(lbmp_handle* h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (h->cfg.alloc) {
        p = h->cfg.alloc(bytes, h->cfg.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) h->allocations.emplace_back(p, bytes);
    return p;
}

void dev_free(lbmp_handle* h, void* p) {
    if (!p) return;
    for (size_t i = 0; i < h->allocations.size(); ++i) {
        if (h->allocations[i].first == p) {
            if (h->cfg.free) h->cfg.free(p, h->allocations[i].second, h->cfg.alloc_ctx);
            else cudaFree(p);
            h->allocations.erase(h->allocations.begin() + (long)i);
            return;
        }
    }
}

double fp16_scale(const lbmp_handle* h, bool inverse) {
    if (h->cfg.precision != LBMP_FP16) return 1.0;
    return std::ldexp(1.0, inverse ? -h->cfg.fp16_scale_log2 : h->cfg.fp16_scale_log2);
}

// Dispatch on the storage type.
template <typename F>
void with_storage(int prec, F&& f) {
    if (prec == LBMP_FP64) f((double*)nullptr);
    else if (prec == LBMP_FP32) f((float*)nullptr);
    else f((__half*)nullptr);
}

// One coupled step (Algorithm 1) on the handle's stream.
void enqueue_step(lbmp_handle* h) {
    const int prec = h->cfg.precision;
    const long long ev_step = profile_mark(h);
    with_storage(prec, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using A = typename Store<S>::A;
        const S* src = (const S*)h->pops[h->cur];
        S* dst = (S*)h->pops[1 - h->cur];
        const CollideParams<A> p = collide_params<A>(h);
        // 1. stream + collide every cell (LBM step)
        const long long ev_bulk = profile_mark(h);
        launch_bulk<S>(src, dst, h->G, p, h->status, h->stream);
        profile_kernel(h, ev_bulk, profile_mark(h), 38.0 * sizeof(S) * (double)h->G.n, (double)h->G.n);
        h->launches += 1;
        if (h->has_particle) {
            // 2. cells next to the sphere: CLI links + momentum-exchange force partials
            int nb = 0;
            launch_boundary<S>(src, dst, h->flags[h->fcur], h->list, h->count, h->list_cap, h->G, p, h->d_ps,
                               h->cfg.boundary == LBMP_CLI ? 1 : 0, h->partials, &nb, h->status, h->stream);
            // 3. force average, gravity, virtual mass, Velocity Verlet
            launch_particle_update(h->d_ps, h->partials, nb, h->G, h->history, h->cfg.history_capacity, h->status,
                                   h->stream);
            // 4. remap: new flags in the box, refill/zero, new boundary list
            uint8_t* fnext = h->flags[1 - h->fcur];
            launch_flags_box(fnext, h->G, h->box, h->d_ps, h->stream);
            launch_refill<S>(dst, h->flags[h->fcur], fnext, h->G, h->box, h->d_ps, (A)fp16_scale(h, false),
                             (A)fp16_scale(h, true), (A)grad_refill_coef(h->cfg.refill, h->tau), h->stream);
            launch_build_links(fnext, h->G, h->box, h->d_ps, h->link_mask, h->link_blocks, h->list, h->count,
                               h->list_cap, h->status, h->stream);
            h->fcur = 1 - h->fcur;
            h->launches += 6;
        }
    });
    profile_step(h, ev_step, profile_mark(h));
    h->cur = 1 - h->cur;
    h->steps += 1;
    h->updates += h->G.n;
}

lbmp_status read_status(lbmp_handle* h) {
    int st = 0;
    LBMP_CK(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    // the particle record comes back with the status word (one synchronisation), so that reading
    // it right after a step costs no second one
    const bool with_ps = h->has_particle && !h->batch;
    if (with_ps) LBMP_CK(h, cudaMemcpyAsync(&h->h_ps, h->d_ps, sizeof(ParticleState), cudaMemcpyDeviceToHost, h->stream));
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    h->d2h += sizeof(int) + (with_ps ? sizeof(ParticleState) : 0);
    h->ps_current = with_ps;
    if (st != 0) {
        int zero = 0;
        LBMP_CK(h, cudaMemcpyAsync(h->status, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
        LBMP_CK(h, cudaStreamSynchronize(h->stream));
        std::string m = "device status:";
        if (st & STATUS_UNSTABLE_FLUID) m += " fluid velocity NaN/Inf or |u|^2 > 0.09;";
        if (st & STATUS_PARTICLE_JUMP) m += " particle moved more than 0.5 cell in one step;";
        if (st & 16) {
            m += " the sphere's neighbourhood left the finest level (regrid more often);";
            return fail(h, LBMP_ERR_PARTICLE_NOT_FINEST, m);
        }
        if (st & 8) {
            m += " a refined-grid pull found no source cell;";
            return fail(h, LBMP_ERR_INVALID_ARG, m);
        }
        if (st & STATUS_LINK_OVERFLOW) {
            m += " boundary list overflow;";
            return fail(h, LBMP_ERR_INVALID_ARG, m);
        }
        return fail(h, LBMP_ERR_UNSTABLE, m);
    }
    return LBMP_OK;
}

lbmp_status upload_particle(lbmp_handle* h) {
    h->frames_stale = true;
    LBMP_CK(h, cudaMemcpyAsync(h->d_ps, &h->h_ps, sizeof(ParticleState), cudaMemcpyHostToDevice, h->stream));
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    h->h2d += sizeof(ParticleState);
    return LBMP_OK;
}

lbmp_status download_particle(lbmp_handle* h) {
    LBMP_CK(h, cudaMemcpyAsync(&h->h_ps, h->d_ps, sizeof(ParticleState), cudaMemcpyDeviceToHost, h->stream));
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    h->d2h += sizeof(ParticleState);
    return LBMP_OK;
}

}  // namespace

namespace lbmp {
long long profile_mark(lbmp_handle* h) {
    if (!h->profiling) return -1;
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        h->ev_pool.push_back(e);
    }
    cudaEventRecord(h->ev_pool[h->ev_used], h->stream);
    return (long long)h->ev_used++;
}

void profile_kernel(lbmp_handle* h, long long start, long long end, double bytes, double updates) {
    if (start < 0 || end < 0) return;
    h->prof_kernel.emplace_back((size_t)start, (size_t)end);
    h->prof_bytes.push_back(bytes);
    h->prof_updates.push_back(updates);
}

void profile_step(lbmp_handle* h, long long start, long long end) {
    if (start < 0 || end < 0) return;
    h->prof_step.emplace_back((size_t)start, (size_t)end);
}

// Error message for entry points that have no handle (read by lbmp_last_error(NULL)).
void set_global_error(const std::string& msg) { g_create_error = msg; }
void* handle_alloc(lbmp_handle* h, size_t bytes) { return dev_alloc(h, bytes); }
void handle_free(lbmp_handle* h, void* p) { dev_free(h, p); }
}  // namespace lbmp

extern "C" {

lbmp_status lbmp_config_default(lbmp_config* c) {
    if (!c) return LBMP_ERR_INVALID_ARG;
    std::memset(c, 0, sizeof(*c));
    c->nx = c->ny = c->nz = 32;
    c->levels = 1;
    c->bc[0] = c->bc[1] = c->bc[2] = LBMP_PERIODIC;
    c->precision = LBMP_FP32;
    c->tau = 0.6;
    c->magic = 3.0 / 16.0;
    c->boundary = LBMP_CLI;
    c->force_average = 1;
    c->rescale_noneq = 0;
    c->regrid_interval = 0;
    c->history_capacity = 4096;
    c->fp16_scale_log2 = 11;
    c->bulk_factor = 1.0;
    c->refill = LBMP_REFILL_EQUILIBRIUM;
    return LBMP_OK;
}

lbmp_status lbmp_create(const lbmp_config* cfg, lbmp_handle** out) {
    if (!cfg || !out) return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: NULL argument");
    *out = nullptr;
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1)
        return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: grid extents must be >= 1");
    const long long n = (long long)cfg->nx * cfg->ny * cfg->nz;
    if (n >= (1LL << 31)) return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: more than 2^31 - 1 cells");
    if (cfg->nz > 65535) return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: nz > 65535");
    if (cfg->levels < 1 || cfg->levels > 6)
        return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: levels must be in [1, 6]");
    if (cfg->levels > 1) {
        if (cfg->nx % 16 || cfg->ny % 16 || cfg->nz % 16)
            return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: refined grids need level-0 extents that are multiples of 16");
        const long long nf = (long long)cfg->nx * cfg->ny * cfg->nz << (3 * (cfg->levels - 1));
        if (nf >= (1LL << 40)) return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: finest lattice too large");
    }
    if (cfg->precision < LBMP_FP64 || cfg->precision > LBMP_FP16)
        return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: unknown precision");
    if (!(cfg->tau > 0.5)) return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: tau must exceed 1/2");
    if (!(cfg->magic > 0.0)) return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: magic parameter must be > 0");
    if (!(cfg->bulk_factor > 0.0) || !std::isfinite(cfg->bulk_factor))
        return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: bulk factor must be > 0 (1 = TRT)");
    if (cfg->refill != LBMP_REFILL_EQUILIBRIUM && cfg->refill != LBMP_REFILL_GRAD)
        return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: unknown refill");
    if (cfg->bulk_factor != 1.0 && cfg->levels > 1 && cfg->rescale_noneq)
        return fail(nullptr, LBMP_ERR_UNSUPPORTED,
                    "lbmp_create: non-equilibrium rescaling is built for TRT only (bulk factor 1)");
    if (cfg->boundary != LBMP_CLI && cfg->boundary != LBMP_SBB)
        return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: unknown boundary scheme");
    for (int a = 0; a < 3; ++a)
        if (cfg->bc[a] != LBMP_PERIODIC && cfg->bc[a] != LBMP_NOSLIP)
            return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: unknown boundary condition");
    if (cfg->history_capacity < 0) return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: history < 0");
    if (cfg->precision == LBMP_FP16 && (cfg->fp16_scale_log2 < 0 || cfg->fp16_scale_log2 > 20))
        return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: fp16_scale_log2 outside [0, 20]");
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
        return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_create: give both alloc and free, or neither");

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(nullptr, LBMP_ERR_CUDA, "lbmp_create: no CUDA device");
    }
    lbmp_handle* h = new (std::nothrow) lbmp_handle();
    if (!h) return fail(nullptr, LBMP_ERR_OOM, "lbmp_create: host allocation failed");
    h->cfg = *cfg;
    h->stream = (cudaStream_t)cfg->cuda_stream;
    h->G.nx = cfg->nx;
    h->G.ny = cfg->ny;
    h->G.nz = cfg->nz;
    for (int a = 0; a < 3; ++a) h->G.periodic[a] = cfg->bc[a] == LBMP_PERIODIC ? 1 : 0;
    h->G.n = n;
    h->tau = cfg->tau;
    h->magic = cfg->magic;
    std::memset(&h->h_ps, 0, sizeof(ParticleState));
    h->h_ps.force_average = cfg->force_average ? 1 : 0;

    const bool refined = cfg->levels > 1;
    const size_t pop_bytes = refined ? 0 : (size_t)19 * (size_t)n * elem_size(cfg->precision);
    if (!refined) {
        h->pops[0] = dev_alloc(h, pop_bytes);
        h->pops[1] = dev_alloc(h, pop_bytes);
        h->flags[0] = (uint8_t*)dev_alloc(h, (size_t)n);
        h->flags[1] = (uint8_t*)dev_alloc(h, (size_t)n);
    }
    h->d_ps = (ParticleState*)dev_alloc(h, sizeof(ParticleState));
    h->status = (int*)dev_alloc(h, sizeof(int));
    h->count = (int*)dev_alloc(h, sizeof(int));
    h->history = (double*)dev_alloc(h, sizeof(double) * 15 * (size_t)std::max(1, cfg->history_capacity));
    if ((!refined && (!h->pops[0] || !h->pops[1] || !h->flags[0] || !h->flags[1])) || !h->d_ps || !h->status ||
        !h->count || !h->history) {
        lbmp_destroy(h);
        return fail(nullptr, LBMP_ERR_OOM, "lbmp_create: device allocation failed");
    }
    cudaError_t e = cudaSuccess;
    if (!refined) {
        if (e == cudaSuccess) e = cudaMemsetAsync(h->pops[0], 0, pop_bytes, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->pops[1], 0, pop_bytes, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->flags[0], 0, (size_t)n, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->flags[1], 0, (size_t)n, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->count, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_ps, &h->h_ps, sizeof(ParticleState), cudaMemcpyHostToDevice,
                                              h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        std::string m = std::string("lbmp_create: ") + cudaGetErrorString(e);
        lbmp_destroy(h);
        return fail(nullptr, LBMP_ERR_CUDA, m);
    }
    if (refined) {
        const lbmp_status st = amr_create(h);
        if (st != LBMP_OK) {
            lbmp_destroy(h);
            return fail(nullptr, st, "lbmp_create: building the refined hierarchy failed");
        }
    }
    *out = h;
    return LBMP_OK;
}

lbmp_status lbmp_destroy(lbmp_handle* h) {
    if (!h) return LBMP_OK;
    cudaStreamSynchronize(h->stream);
    amr_destroy(h);
    batch_destroy(h);
    adjoint_destroy(h);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    h->ev_pool.clear();
    while (!h->allocations.empty()) dev_free(h, h->allocations.back().first);
    delete h;
    return LBMP_OK;
}

lbmp_status lbmp_add_sphere(lbmp_handle* h, const double pos[3], double diameter, double density_ratio, double cv,
                            double cv_omega, int* id) {
    if (!h || !pos) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_add_sphere: NULL argument");
    if (h->has_particle) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_add_sphere: one sphere per handle");
    if (!(diameter > 0.0) || !(density_ratio > 0.0) || cv < 0.0 || cv_omega < 0.0)
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_add_sphere: diameter and density ratio must be > 0, C_v >= 0");
    const int sh = h->cfg.levels - 1;   // positions are in finest-level units
    const int n3[3] = {h->G.nx << sh, h->G.ny << sh, h->G.nz << sh};
    for (int a = 0; a < 3; ++a) {
        if (!(pos[a] >= 0.0 && pos[a] <= (double)n3[a]))
            return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_add_sphere: centre outside the domain");
        if (diameter + 4.0 > (double)n3[a])
            return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_add_sphere: sphere (plus 2 cells) does not fit the domain");
    }
    ParticleState& P = h->h_ps;
    for (int a = 0; a < 3; ++a) P.x[a] = pos[a];
    P.D = diameter;
    P.r = 0.5 * diameter;
    P.rho_p = density_ratio;
    P.cv = cv;
    P.cvw = cv_omega;
    P.V = M_PI * diameter * diameter * diameter / 6.0;
    P.present = 1;
    P.force_average = h->cfg.force_average ? 1 : 0;
    if (h->amr) {
        const lbmp_status st = amr_add_sphere(h);
        if (st != LBMP_OK) return fail(h, st, "lbmp_add_sphere: building the refined hierarchy failed");
        if (id) *id = 0;
        return read_status(h);
    }
    // box around the sphere: half width ceil(r) + 3 cells covers every cell
    // whose flag or boundary status can change in one step (|dx| < 1/2)
    BoxDesc& B = h->box;
    B.R = (int)std::ceil(P.r) + 3;
    B.cells = 1;
    for (int a = 0; a < 3; ++a) {
        B.E[a] = 2 * B.R + 2;
        if (h->G.periodic[a] && B.E[a] >= n3[a]) B.E[a] = n3[a];
        B.cells *= B.E[a];
    }
    // Boundary cells lie in the shell r < |x - x_p| <= r + sqrt(2); cell
    // centres in it are bounded by the volume of the shell widened by the
    // half-diagonal sqrt(3)/2 of a cell on both sides.
    const double h3 = 0.5 * std::sqrt(3.0);
    const double ro = P.r + std::sqrt(2.0) + h3, ri = std::max(0.0, P.r - h3);
    const double shell = 4.0 / 3.0 * M_PI * (ro * ro * ro - ri * ri * ri);
    h->list_cap = (int)std::min<double>((double)B.cells, std::ceil(shell) + 64.0);
    h->list = (int*)dev_alloc(h, sizeof(int) * (size_t)h->list_cap);
    const int max_blocks = boundary_grid(h->list_cap);
    h->partials = (double*)dev_alloc(h, sizeof(double) * 6 * (size_t)max_blocks);
    h->link_mask = (uint8_t*)dev_alloc(h, (size_t)B.cells);
    h->link_blocks = (int*)dev_alloc(h, sizeof(int) * (size_t)((B.cells + 255) / 256));
    if (!h->list || !h->partials || !h->link_mask || !h->link_blocks)
        return fail(h, LBMP_ERR_OOM, "lbmp_add_sphere: device allocation failed");
    lbmp_status s = upload_particle(h);
    if (s != LBMP_OK) return s;
    launch_flags_full(h->flags[h->fcur], h->G, h->d_ps, h->stream);
    launch_flags_full(h->flags[1 - h->fcur], h->G, h->d_ps, h->stream);
    with_storage(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        launch_zero_solid<S>((S*)h->pops[h->cur], h->flags[h->fcur], h->G, h->stream);
    });
    launch_build_links(h->flags[h->fcur], h->G, h->box, h->d_ps, h->link_mask, h->link_blocks, h->list, h->count,
                       h->list_cap, h->status, h->stream);
    LBMP_CK(h, cudaGetLastError());
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    h->has_particle = true;
    if (id) *id = 0;
    return read_status(h);
}

lbmp_status lbmp_set_particle_velocity(lbmp_handle* h, int id, const double u[3], const double w[3]) {
    if (!h || !u || !w) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_particle_velocity: NULL argument");
    if (!h->has_particle || id != 0) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_particle_velocity: no such sphere");
    lbmp_status s = download_particle(h);
    if (s != LBMP_OK) return s;
    for (int a = 0; a < 3; ++a) {
        h->h_ps.u[a] = u[a];
        h->h_ps.w[a] = w[a];
    }
    return upload_particle(h);
}

lbmp_status lbmp_set_particle_fixed(lbmp_handle* h, int id, int fixed) {
    if (!h) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_particle_fixed: NULL handle");
    if (!h->has_particle || id != 0) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_particle_fixed: no such sphere");
    if (fixed < 0 || fixed > 2) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_particle_fixed: fixed must be 0, 1 or 2");
    lbmp_status s = download_particle(h);
    if (s != LBMP_OK) return s;
    h->h_ps.fixed = fixed;
    return upload_particle(h);
}

lbmp_status lbmp_set_wall_velocity(lbmp_handle* h, int axis, int side, const double u[3]) {
    if (!h || !u) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_wall_velocity: NULL argument");
    if (h->amr || h->batch)
        return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_set_wall_velocity: uniform grids only (refined walls are at rest)");
    if (axis < 0 || axis > 2 || side < 0 || side > 1)
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_wall_velocity: axis must be 0..2 and side 0 or 1");
    if (h->G.periodic[axis]) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_wall_velocity: the axis is periodic");
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(u[a]) || std::fabs(u[a]) >= 0.3)
            return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_wall_velocity: need finite |u| < 0.3 (lattice units)");
        h->G.uw[axis][side][a] = u[a];
    }
    int moving = 0;
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 2; ++s)
            for (int k = 0; k < 3; ++k) moving |= h->G.uw[a][s][k] != 0.0;
    h->G.moving = moving;
    return LBMP_OK;
}

lbmp_status lbmp_ga_parameters(double ga, double u_g, double diameter, double density_ratio, double* nu, double* g,
                               double* tau) {
    if (!(ga > 0.0) || !(u_g > 0.0) || !(diameter > 0.0) || !(density_ratio > 0.0) || density_ratio == 1.0)
        return LBMP_ERR_INVALID_ARG;
    // Ga = u_g d_p / nu, u_g = sqrt(|pi_p - 1| g d_p)   (Sec. 3.1)
    const double v = u_g * diameter / ga;
    const double gg = u_g * u_g / (std::fabs(density_ratio - 1.0) * diameter);
    if (nu) *nu = v;
    if (g) *g = gg;
    if (tau) *tau = 3.0 * v + 0.5;   // nu = c_s^2 (tau - 1/2)
    return LBMP_OK;
}

lbmp_status lbmp_set_ga(lbmp_handle* h, double ga, double u_g, const double dir[3]) {
    if (!h || !dir) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_ga: NULL argument");
    if (!h->has_particle) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_ga: add the sphere first");
    double nu, g, tau;
    if (lbmp_ga_parameters(ga, u_g, h->h_ps.D, h->h_ps.rho_p, &nu, &g, &tau) != LBMP_OK)
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_ga: invalid Ga, u_g or density ratio == 1");
    const double norm = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(norm > 0.0)) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_ga: zero direction");
    const double gv[3] = {g * dir[0] / norm, g * dir[1] / norm, g * dir[2] / norm};
    lbmp_status s = lbmp_set_tau(h, tau);
    if (s != LBMP_OK) return s;
    return lbmp_set_gravity(h, gv);
}

lbmp_status lbmp_set_tau(lbmp_handle* h, double tau) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    if (!(tau > 0.5)) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_tau: tau must exceed 1/2");
    h->tau = tau;
    return LBMP_OK;
}

lbmp_status lbmp_set_gravity(lbmp_handle* h, const double g[3]) {
    if (!h || !g) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_gravity: NULL argument");
    if (h->batch) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_set_gravity: gravity is set per simulation of a batch");
    for (int a = 0; a < 3; ++a) h->h_ps.g[a] = g[a];
    // kernels only read the gravity field, so it is written alone, ordered on the
    // stream (the copy from the caller's memory is staged before the call returns)
    LBMP_CK(h, cudaMemcpyAsync(reinterpret_cast<char*>(h->d_ps) + offsetof(ParticleState, g), h->h_ps.g,
                               sizeof(h->h_ps.g), cudaMemcpyHostToDevice, h->stream));
    h->h2d += sizeof(h->h_ps.g);
    return LBMP_OK;
}

lbmp_status lbmp_set_body_force(lbmp_handle* h, const double f[3]) {
    if (!h || !f) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_body_force: NULL argument");
    if (h->amr && (f[0] != 0.0 || f[1] != 0.0 || f[2] != 0.0))
        return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_set_body_force: fluid forcing is implemented on uniform grids");
    for (int a = 0; a < 3; ++a) h->body_force[a] = f[a];
    return LBMP_OK;
}

lbmp_status lbmp_init_fluid(lbmp_handle* h, double rho, const double u[3], const double* u_field,
                            int u_field_on_device) {
    if (!h || !u) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_init_fluid: NULL argument");
    if (h->amr) {
        if (u_field) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_init_fluid: refined grids take lbmp_init_fluid_wave");
        return amr_init_fluid(h, rho, u, 0.0, 0, 0) == LBMP_OK ? LBMP_OK
                                                               : fail(h, LBMP_ERR_CUDA, "lbmp_init_fluid: kernel failed");
    }
    const double* dfield = nullptr;
    double* tmp = nullptr;
    if (u_field && !u_field_on_device) {
        tmp = (double*)dev_alloc(h, sizeof(double) * 3 * (size_t)h->G.n);
        if (!tmp) return fail(h, LBMP_ERR_OOM, "lbmp_init_fluid: staging allocation failed");
        LBMP_CK(h, cudaMemcpyAsync(tmp, u_field, sizeof(double) * 3 * (size_t)h->G.n, cudaMemcpyHostToDevice,
                                   h->stream));
        dfield = tmp;
    } else if (u_field) {
        dfield = u_field;
    }
    with_storage(h->cfg.precision, [&](auto tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        using A = typename Store<S>::A;
        launch_init_equilibrium<S>((S*)h->pops[h->cur], h->flags[h->fcur], h->G, rho, u, dfield,
                                   (A)fp16_scale(h, false), h->stream);
    });
    LBMP_CK(h, cudaGetLastError());
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    dev_free(h, tmp);
    return LBMP_OK;
}

lbmp_status lbmp_set_populations(lbmp_handle* h, const double* g, size_t cap) {
    if (h && h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_set_populations: uniform grids only (refined: lbmp_get_level_cells)");
    if (!h || !g) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_populations: NULL argument");
    const long long total = 19LL * h->G.n;
    if ((long long)cap < total) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_populations: cap < 19*cells");
    const long long chunk = std::min<long long>(total, 1LL << 25);
    double* tmp = (double*)dev_alloc(h, sizeof(double) * (size_t)chunk);
    if (!tmp) return fail(h, LBMP_ERR_OOM, "lbmp_set_populations: staging allocation failed");
    lbmp_status st = LBMP_OK;
    for (long long off = 0; off < total && st == LBMP_OK; off += chunk) {
        const long long m = std::min(chunk, total - off);
        cudaError_t e = cudaMemcpyAsync(tmp, g + off, sizeof(double) * (size_t)m, cudaMemcpyHostToDevice, h->stream);
        h->h2d += (long long)sizeof(double) * m;
        if (e != cudaSuccess) {
            st = cuda_fail(h, e, "lbmp_set_populations");
            break;
        }
        with_storage(h->cfg.precision, [&](auto tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            using A = typename Store<S>::A;
            launch_from_f64<S>(tmp, (S*)h->pops[h->cur] + off, m, (A)fp16_scale(h, false), h->stream);
        });
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "lbmp_set_populations");
    }
    dev_free(h, tmp);
    return st;
}

lbmp_status lbmp_get_populations(lbmp_handle* h, double* g, size_t cap) {
    if (h && h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_get_populations: uniform grids only (refined: lbmp_get_level_cells)");
    if (!h || !g) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_populations: NULL argument");
    const long long total = 19LL * h->G.n;
    if ((long long)cap < total) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_populations: cap < 19*cells");
    const long long chunk = std::min<long long>(total, 1LL << 25);
    double* tmp = (double*)dev_alloc(h, sizeof(double) * (size_t)chunk);
    if (!tmp) return fail(h, LBMP_ERR_OOM, "lbmp_get_populations: staging allocation failed");
    lbmp_status st = LBMP_OK;
    for (long long off = 0; off < total && st == LBMP_OK; off += chunk) {
        const long long m = std::min(chunk, total - off);
        with_storage(h->cfg.precision, [&](auto tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            using A = typename Store<S>::A;
            launch_to_f64<S>((const S*)h->pops[h->cur] + off, tmp, m, (A)fp16_scale(h, true), h->stream);
        });
        cudaError_t e = cudaMemcpyAsync(g + off, tmp, sizeof(double) * (size_t)m, cudaMemcpyDeviceToHost, h->stream);
        h->d2h += (long long)sizeof(double) * m;
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "lbmp_get_populations");
    }
    dev_free(h, tmp);
    return st;
}

lbmp_status lbmp_gather_populations(lbmp_handle* h, const int64_t* cells, size_t n, double* out) {
    if (h && h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_gather_populations: uniform grids only (refined: lbmp_get_level_cells)");
    if (!h || (n > 0 && (!cells || !out))) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_gather_populations: NULL argument");
    if (n == 0) return LBMP_OK;
    for (size_t i = 0; i < n; ++i)
        if (cells[i] < 0 || cells[i] >= h->G.n)
            return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_gather_populations: cell index out of range");
    int64_t* dc = (int64_t*)dev_alloc(h, sizeof(int64_t) * n);
    double* dout = (double*)dev_alloc(h, sizeof(double) * 19 * n);
    if (!dc || !dout) {
        dev_free(h, dc);
        dev_free(h, dout);
        return fail(h, LBMP_ERR_OOM, "lbmp_gather_populations: staging allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(dc, cells, sizeof(int64_t) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        with_storage(h->cfg.precision, [&](auto tag) {
            using S = std::remove_pointer_t<decltype(tag)>;
            using A = typename Store<S>::A;
            launch_gather<S>((const S*)h->pops[h->cur], h->G.n, dc, (long long)n, dout, (A)fp16_scale(h, true),
                             h->stream);
        });
        e = cudaMemcpyAsync(out, dout, sizeof(double) * 19 * n, cudaMemcpyDeviceToHost, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(h, dc);
    dev_free(h, dout);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmp_gather_populations");
    return LBMP_OK;
}

lbmp_status lbmp_step_async(lbmp_handle* h, int n) {
    if (!h || n < 0) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_step: bad argument");
    h->ps_current = false;
    if (h->amr) {
        const lbmp_status st = amr_step(h, n);
        if (st != LBMP_OK) return fail(h, st, "lbmp_step: " + h->err);
        return LBMP_OK;
    }
    if (h->batch) {
        const lbmp_status st = batch_step(h, n);
        if (st != LBMP_OK) return fail(h, st, std::string("lbmp_step: batched step failed: ") +
                                              cudaGetErrorString(cudaGetLastError()));
        return LBMP_OK;
    }
    for (int i = 0; i < n; ++i) enqueue_step(h);
    LBMP_CK(h, cudaGetLastError());
    return LBMP_OK;
}

lbmp_status lbmp_step(lbmp_handle* h, int n) {
    lbmp_status s = lbmp_step_async(h, n);
    if (s != LBMP_OK) return s;
    return read_status(h);
}

lbmp_status lbmp_check_status(lbmp_handle* h) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    return read_status(h);
}

lbmp_status lbmp_synchronize(lbmp_handle* h) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    return LBMP_OK;
}

lbmp_status lbmp_get_particle(lbmp_handle* h, int id, double out[24]) {
    if (!h || !out) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_particle: NULL argument");
    ParticleState tmp;
    if (h->batch) {
        if (batch_get_particle(h, id, &tmp) != LBMP_OK) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_particle: no such simulation");
    } else {
        if (!h->has_particle || id != 0) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_particle: no such sphere");
        if (!h->ps_current) {
            lbmp_status s = download_particle(h);
            if (s != LBMP_OK) return s;
        }
        tmp = h->h_ps;
    }
    const ParticleState& P = tmp;
    for (int a = 0; a < 3; ++a) {
        out[a] = P.Fh[a];
        out[3 + a] = P.Th[a];
        out[6 + a] = P.x[a];
        out[9 + a] = P.u[a];
        out[12 + a] = P.w[a];
        out[15 + a] = P.a[a];
        out[18 + a] = P.b[a];
        out[21 + a] = P.Fp[a];
    }
    return LBMP_OK;
}

lbmp_status lbmp_get_history(lbmp_handle* h, int id, double* out, int max_steps, int* n) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    ParticleState tmp;
    if (h->batch) {
        if (batch_get_particle(h, id, &tmp) != LBMP_OK) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_history: no such simulation");
    } else {
        if (!h->has_particle || id != 0) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_history: no such sphere");
        lbmp_status s = download_particle(h);
        if (s != LBMP_OK) return s;
        tmp = h->h_ps;
    }
    const long long steps = tmp.steps;
    const int cap = h->cfg.history_capacity;
    const long long avail = std::min<long long>(steps, cap);
    if (n) *n = (int)avail;
    if (!out || max_steps <= 0 || avail == 0) return LBMP_OK;
    std::vector<double> ring((size_t)cap * 15);
    if (h->batch) {
        if (batch_history(h, id, ring.data(), cap) != LBMP_OK) return fail(h, LBMP_ERR_CUDA, "lbmp_get_history: copy failed");
    } else {
        LBMP_CK(h, cudaMemcpyAsync(ring.data(), h->history, sizeof(double) * 15 * (size_t)cap, cudaMemcpyDeviceToHost,
                                   h->stream));
        LBMP_CK(h, cudaStreamSynchronize(h->stream));
    }
    const long long m = std::min<long long>(avail, max_steps);
    const long long first = steps - m;   // oldest step returned
    for (long long i = 0; i < m; ++i) {
        const long long st = first + i;
        std::memcpy(out + i * 15, ring.data() + (size_t)(st % cap) * 15, sizeof(double) * 15);
    }
    if (n) *n = (int)m;
    return LBMP_OK;
}

lbmp_status lbmp_get_flags(lbmp_handle* h, uint8_t* out, size_t cap) {
    if (h && h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_get_flags: uniform grids only (refined: lbmp_get_level_cells)");
    if (!h || !out) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_flags: NULL argument");
    if ((long long)cap < h->G.n) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_flags: cap < cells");
    LBMP_CK(h, cudaMemcpyAsync(out, h->flags[h->fcur], (size_t)h->G.n, cudaMemcpyDeviceToHost, h->stream));
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    return LBMP_OK;
}

lbmp_status lbmp_get_links(lbmp_handle* h, int64_t* cell, int32_t* q, double* delta, size_t cap, size_t* n) {
    if (!h || !n) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_links: NULL argument");
    *n = 0;
    if (h->amr) {
        const lbmp_status st = amr_links(h, cell, q, delta, cap, n);
        return st == LBMP_OK ? LBMP_OK : fail(h, st, "lbmp_get_links: failed");
    }
    if (!h->has_particle) return LBMP_OK;
    int cnt = 0;
    LBMP_CK(h, cudaMemcpyAsync(&cnt, h->count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    if (cnt == 0) return LBMP_OK;
    int32_t* dq = (int32_t*)dev_alloc(h, sizeof(int32_t) * 18 * (size_t)cnt);
    double* dd = (double*)dev_alloc(h, sizeof(double) * 18 * (size_t)cnt);
    if (!dq || !dd) {
        dev_free(h, dq);
        dev_free(h, dd);
        return fail(h, LBMP_ERR_OOM, "lbmp_get_links: staging allocation failed");
    }
    launch_export_links(h->flags[h->fcur], h->list, h->count, cnt, h->G, h->d_ps, 1, dq, dd, h->stream);
    std::vector<int32_t> hq((size_t)cnt * 18);
    std::vector<double> hd((size_t)cnt * 18);
    std::vector<int> hl((size_t)cnt);
    cudaError_t e = cudaMemcpyAsync(hq.data(), dq, sizeof(int32_t) * hq.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd.data(), dd, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hl.data(), h->list, sizeof(int) * hl.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(h, dq);
    dev_free(h, dd);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmp_get_links");
    size_t m = 0;
    for (int i = 0; i < cnt; ++i)
        for (int s = 0; s < 18; ++s) {
            const size_t slot = (size_t)i * 18 + s;
            if (hq[slot] < 0) continue;
            if (m < cap) {
                if (cell) cell[m] = hl[i];
                if (q) q[m] = hq[slot];
                if (delta) delta[m] = hd[slot];
            }
            ++m;
        }
    *n = m;
    return LBMP_OK;
}

lbmp_status lbmp_get_counters(lbmp_handle* h, int64_t out[5]) {
    if (!h || !out) return LBMP_ERR_INVALID_ARG;
    out[0] = h->steps;
    out[1] = h->updates;
    out[2] = h->launches;
    out[3] = h->h2d;
    out[4] = h->d2h;
    return LBMP_OK;
}

lbmp_status lbmp_profile(lbmp_handle* h, int enable) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    if (enable) {
        LBMP_CK(h, cudaStreamSynchronize(h->stream));
        h->ev_used = 0;
        h->prof_kernel.clear();
        h->prof_bytes.clear();
        h->prof_updates.clear();
        h->prof_step.clear();
    }
    h->profiling = enable != 0;
    return LBMP_OK;
}

lbmp_status lbmp_get_profile(lbmp_handle* h, double out[6]) {
    if (!h || !out) return LBMP_ERR_INVALID_ARG;
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    double kms = 0.0, sms = 0.0, bytes = 0.0, upd = 0.0;
    for (size_t i = 0; i < h->prof_kernel.size(); ++i) {
        float a = 0.f;
        LBMP_CK(h, cudaEventElapsedTime(&a, h->ev_pool[h->prof_kernel[i].first], h->ev_pool[h->prof_kernel[i].second]));
        kms += a;
        bytes += h->prof_bytes[i];
        upd += h->prof_updates[i];
    }
    for (auto& p : h->prof_step) {
        float a = 0.f;
        LBMP_CK(h, cudaEventElapsedTime(&a, h->ev_pool[p.first], h->ev_pool[p.second]));
        sms += a;
    }
    out[0] = kms;
    out[1] = (double)h->prof_kernel.size();
    out[2] = sms;
    out[3] = (double)h->prof_step.size();
    out[4] = bytes;
    out[5] = upd;
    return LBMP_OK;
}

lbmp_status lbmp_init_fluid_wave(lbmp_handle* h, double rho, const double u[3], double amp, int dir, int axis) {
    if (!h || !u || dir < 0 || dir > 2 || axis < 0 || axis > 2)
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_init_fluid_wave: bad argument");
    if (h->amr) {
        return amr_init_fluid(h, rho, u, amp, dir, axis) == LBMP_OK
                   ? LBMP_OK
                   : fail(h, LBMP_ERR_CUDA, "lbmp_init_fluid_wave: kernel failed");
    }
    const int n3[3] = {h->G.nx, h->G.ny, h->G.nz};
    std::vector<double> f((size_t)3 * h->G.n);
    for (long long c = 0; c < h->G.n; ++c) {
        const long long idx[3] = {c % n3[0], (c / n3[0]) % n3[1], c / ((long long)n3[0] * n3[1])};
        for (int a = 0; a < 3; ++a) f[(size_t)a * h->G.n + c] = u[a];
        f[(size_t)dir * h->G.n + c] += amp * std::sin(2.0 * M_PI * (idx[axis] + 0.5) / n3[axis]);
    }
    const double zero[3] = {0, 0, 0};
    return lbmp_init_fluid(h, rho, zero, f.data(), 0);
}

lbmp_status lbmp_refine_box(lbmp_handle* h, const double lo[3], const double hi[3]) {
    if (!h || !lo || !hi) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_refine_box: NULL argument");
    if (!h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_refine_box: the grid has one level");
    const lbmp_status st = amr_refine_box(h, lo, hi);
    if (st != LBMP_OK) return fail(h, st, "lbmp_refine_box: regrid failed");
    return read_status(h);
}

lbmp_status lbmp_regrid(lbmp_handle* h) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    if (!h->amr) return LBMP_OK;
    const lbmp_status st = amr_regrid(h);
    if (st != LBMP_OK) return fail(h, st, "lbmp_regrid: failed");
    return read_status(h);
}

lbmp_status lbmp_set_refinement_sensor(lbmp_handle* h, double sigma_c, double c) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    if (!h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_set_refinement_sensor: the grid has one level");
    if (!(sigma_c >= 0.0) || !std::isfinite(sigma_c) ||
        (sigma_c > 0.0 && !(c > 0.0 && c < std::pow(2.0, -1.5))))
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_set_refinement_sensor: need sigma_c >= 0 and 0 < c < 2^-1.5");
    return amr_set_sensor(h, sigma_c, c);
}

lbmp_status lbmp_get_block_sensor(lbmp_handle* h, int level, double* out, size_t cap, size_t* n) {
    if (!h || !n) return LBMP_ERR_INVALID_ARG;
    if (!h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_get_block_sensor: the grid has one level");
    const lbmp_status st = amr_block_sensor(h, level, out, cap, n);
    if (st == LBMP_ERR_INVALID_ARG) return fail(h, st, "lbmp_get_block_sensor: no such level");
    return st == LBMP_OK ? LBMP_OK : fail(h, st, "lbmp_get_block_sensor: failed");
}

lbmp_status lbmp_level_shape(lbmp_handle* h, int level, int out[3]) {
    if (!h || !out) return LBMP_ERR_INVALID_ARG;
    if (!h->amr) {
        if (level != 0) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_level_shape: no such level");
        out[0] = h->G.nx;
        out[1] = h->G.ny;
        out[2] = h->G.nz;
        return LBMP_OK;
    }
    return amr_level_shape(h, level, out) == LBMP_OK ? LBMP_OK
                                                     : fail(h, LBMP_ERR_INVALID_ARG, "lbmp_level_shape: no such level");
}

lbmp_status lbmp_get_block_map(lbmp_handle* h, int level, int32_t* out, size_t cap, size_t* n) {
    if (!h || !n) return LBMP_ERR_INVALID_ARG;
    if (!h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_get_block_map: the grid has one level");
    return amr_block_map(h, level, out, cap, n) == LBMP_OK ? LBMP_OK
                                                          : fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_block_map: no such level");
}

lbmp_status lbmp_get_level_cells(lbmp_handle* h, int level, int32_t* xyz, double* g, size_t cap, size_t* n) {
    if (!h || !n) return LBMP_ERR_INVALID_ARG;
    if (!h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_get_level_cells: the grid has one level");
    const lbmp_status st = amr_level_cells(h, level, xyz, g, cap, n);
    return st == LBMP_OK ? LBMP_OK : fail(h, st, "lbmp_get_level_cells: failed");
}

lbmp_status lbmp_get_level_flags(lbmp_handle* h, int level, uint8_t* out, size_t cap, size_t* n) {
    if (!h || !n) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_get_level_flags: NULL argument");
    if (!h->amr) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_get_level_flags: the grid has one level (lbmp_get_flags)");
    const lbmp_status st = amr_level_flags(h, level, out, cap, n);
    return st == LBMP_OK ? LBMP_OK : fail(h, st, "lbmp_get_level_flags: failed");
}

lbmp_status lbmp_updates_per_step(lbmp_handle* h, int64_t* updates, int32_t* launches) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    if (h->amr) {
        if (updates) *updates = amr_cell_updates_per_coarse_step(h);
        if (launches) *launches = amr_launches_per_coarse_step(h);
    } else {
        if (updates) *updates = h->G.n;
        if (launches) *launches = h->has_particle ? 7 : 1;
    }
    return LBMP_OK;
}

lbmp_status lbmp_batch_create(const lbmp_config* cfg, const lbmp_batch_sim* sims, int n, lbmp_handle** out) {
    if (!cfg || !sims || !out || n < 1) return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_batch_create: bad argument");
    *out = nullptr;
    long long cells = 0;
    for (int s = 0; s < n; ++s) {
        const lbmp_batch_sim& b = sims[s];
        if (b.edge < 16 || b.edge % 16 || b.edge > 1024)
            return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_batch_create: edges must be multiples of 16 in [16, 1024]");
        if (!(b.tau > 0.5) || !(b.diameter > 0.0) || !(b.density_ratio > 0.0) || b.cv < 0 || b.cv_omega < 0 ||
            b.diameter + 4.0 > b.edge)
            return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_batch_create: invalid simulation parameters");
        for (int a = 0; a < 3; ++a)
            if (!(b.pos[a] >= 0.0 && b.pos[a] <= (double)b.edge))
                return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_batch_create: centre outside its box");
        cells += (long long)b.edge * b.edge * b.edge;
    }
    if (cells >= (1LL << 31)) return fail(nullptr, LBMP_ERR_INVALID_ARG, "lbmp_batch_create: more than 2^31 - 1 cells");
    lbmp_config c = *cfg;
    c.nx = c.ny = c.nz = 16;
    c.levels = 1;
    c.bc[0] = c.bc[1] = c.bc[2] = LBMP_PERIODIC;
    lbmp_handle* h = nullptr;
    lbmp_status st = lbmp_create(&c, &h);
    if (st != LBMP_OK) return st;
    st = batch_create(h, sims, n);
    if (st != LBMP_OK) {
        lbmp_destroy(h);
        return fail(nullptr, st, "lbmp_batch_create: setting up the batch failed");
    }
    *out = h;
    return LBMP_OK;
}

lbmp_status lbmp_batch_autotune(lbmp_handle* h, int reps) {
    if (!h || !h->batch || reps < 1) return LBMP_ERR_INVALID_ARG;
    const lbmp_status st = batch_autotune(h, reps);
    return st == LBMP_OK ? LBMP_OK : fail(h, st, "lbmp_batch_autotune: failed");
}

lbmp_status lbmp_batch_info(lbmp_handle* h, int64_t out[8]) {
    if (!h || !h->batch || !out) return LBMP_ERR_INVALID_ARG;
    batch_info(h, out);
    return LBMP_OK;
}

lbmp_status lbmp_batch_get_populations(lbmp_handle* h, int sim, double* out, size_t cap) {
    if (!h || !h->batch || !out) return LBMP_ERR_INVALID_ARG;
    const lbmp_status st = batch_populations(h, sim, out, cap);
    return st == LBMP_OK ? LBMP_OK : fail(h, st, "lbmp_batch_get_populations: bad simulation index or capacity");
}

// ------------------------------------------------------------ checkpoint
namespace {

struct CkptHeader {
    char tag[8];              // "LBMPCKPT"
    int32_t version;          // 2
    int32_t nx, ny, nz, levels, precision, bc[3];
    int32_t has_particle, history_capacity, particle_bytes, kind;   // kind: 0 uniform, 1 refined
    double tau, magic, bulk_factor;
    double body_force[3];
    int64_t steps;
    double wall_u[3][2][3];   // domain wall velocities (uniform grids)
};

bool put(FILE* f, const void* p, size_t n) { return n == 0 || fwrite(p, 1, n, f) == n; }
bool get(FILE* f, void* p, size_t n) { return n == 0 || fread(p, 1, n, f) == n; }

}  // namespace

lbmp_status lbmp_save(lbmp_handle* h, const char* path) {
    if (!h || !path) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_save: NULL argument");
    if (h->batch) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_save: batched handles are not checkpointed");
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, cudaGetLastError(), "lbmp_save");
    if (h->has_particle) {
        const lbmp_status s = download_particle(h);
        if (s != LBMP_OK) return s;
    }
    CkptHeader H;
    std::memset(&H, 0, sizeof(H));
    std::memcpy(H.tag, "LBMPCKPT", 8);
    H.version = 2;
    H.nx = h->cfg.nx;
    H.ny = h->cfg.ny;
    H.nz = h->cfg.nz;
    H.levels = h->cfg.levels;
    H.precision = h->cfg.precision;
    for (int a = 0; a < 3; ++a) H.bc[a] = h->cfg.bc[a];
    H.has_particle = h->has_particle ? 1 : 0;
    H.history_capacity = h->history ? h->cfg.history_capacity : 0;
    H.particle_bytes = (int32_t)sizeof(ParticleState);
    H.kind = h->amr ? 1 : 0;
    H.tau = h->tau;
    H.magic = h->magic;
    H.bulk_factor = h->cfg.bulk_factor;
    for (int a = 0; a < 3; ++a) H.body_force[a] = h->body_force[a];
    H.steps = h->steps;
    std::memcpy(H.wall_u, h->G.uw, sizeof(H.wall_u));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(h, LBMP_ERR_INVALID_ARG, std::string("lbmp_save: cannot open ") + path);
    bool ok = put(f, &H, sizeof(H)) && put(f, &h->h_ps, sizeof(ParticleState));
    if (ok && H.history_capacity > 0) {
        std::vector<double> hist((size_t)H.history_capacity * 15);
        ok = cudaMemcpy(hist.data(), h->history, hist.size() * sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess &&
             put(f, hist.data(), hist.size() * sizeof(double));
    }
    if (ok && h->amr) {
        ok = amr_save(h, f) == LBMP_OK;
    } else if (ok) {
        const size_t pb = (size_t)19 * (size_t)h->G.n * elem_size(h->cfg.precision);
        std::vector<unsigned char> buf(pb);
        ok = cudaMemcpy(buf.data(), h->pops[h->cur], pb, cudaMemcpyDeviceToHost) == cudaSuccess && put(f, buf.data(), pb);
        buf.resize((size_t)h->G.n);
        ok = ok && cudaMemcpy(buf.data(), h->flags[h->fcur], (size_t)h->G.n, cudaMemcpyDeviceToHost) == cudaSuccess &&
             put(f, buf.data(), (size_t)h->G.n);
    }
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(h, LBMP_ERR_CUDA, std::string("lbmp_save: writing ") + path + " failed");
    return LBMP_OK;
}

lbmp_status lbmp_load(lbmp_handle* h, const char* path) {
    if (!h || !path) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_load: NULL argument");
    if (h->batch) return fail(h, LBMP_ERR_UNSUPPORTED, "lbmp_load: batched handles are not checkpointed");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(h, LBMP_ERR_INVALID_ARG, std::string("lbmp_load: cannot open ") + path);
    struct Closer {
        FILE* f;
        ~Closer() { std::fclose(f); }
    } closer{f};
    CkptHeader H;
    ParticleState P;
    if (!get(f, &H, sizeof(H)) || std::memcmp(H.tag, "LBMPCKPT", 8) != 0 || H.version != 2 ||
        H.particle_bytes != (int32_t)sizeof(ParticleState) || !get(f, &P, sizeof(P)))
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_load: not a checkpoint of this library version");
    bool same = H.nx == h->cfg.nx && H.ny == h->cfg.ny && H.nz == h->cfg.nz && H.levels == h->cfg.levels &&
                H.precision == h->cfg.precision && H.kind == (h->amr ? 1 : 0);
    for (int a = 0; a < 3; ++a) same = same && H.bc[a] == h->cfg.bc[a];
    if (!same)
        return fail(h, LBMP_ERR_INVALID_ARG,
                    "lbmp_load: the checkpoint's grid, levels, precision or boundary conditions differ from the handle's");
    if (h->has_particle && !H.has_particle)
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_load: the handle has a sphere, the checkpoint none");
    if (h->has_particle && h->h_ps.D != P.D)
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_load: the handle's sphere has another diameter");
    if (H.has_particle && !h->has_particle) {   // buffers and hierarchy for the saved sphere
        const lbmp_status s = lbmp_add_sphere(h, P.x, P.D, P.rho_p, P.cv, P.cvw, nullptr);
        if (s != LBMP_OK) return s;
    }
    std::vector<double> hist((size_t)std::max(H.history_capacity, 0) * 15);
    if (!get(f, hist.data(), hist.size() * sizeof(double)))
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_load: truncated checkpoint");
    h->tau = H.tau;
    for (int a = 0; a < 3; ++a) h->body_force[a] = H.body_force[a];
    h->steps = H.steps;
    if (!h->amr) {
        std::memcpy(h->G.uw, H.wall_u, sizeof(H.wall_u));
        int moving = 0;
        for (const double* v = &H.wall_u[0][0][0]; v < &H.wall_u[0][0][0] + 18; ++v) moving |= *v != 0.0;
        h->G.moving = moving;
    }
    if (H.has_particle) {
        h->h_ps = P;
        const lbmp_status s = upload_particle(h);
        if (s != LBMP_OK) return s;
    }
    if (H.history_capacity > 0 && h->history && H.history_capacity == h->cfg.history_capacity)
        LBMP_CK(h, cudaMemcpy(h->history, hist.data(), hist.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (h->amr) {
        const lbmp_status s = amr_load(h, f);
        if (s != LBMP_OK) return fail(h, s, "lbmp_load: restoring the refined hierarchy failed");
        return read_status(h);
    }
    const size_t pb = (size_t)19 * (size_t)h->G.n * elem_size(h->cfg.precision);
    std::vector<unsigned char> buf(pb);
    if (!get(f, buf.data(), pb)) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_load: truncated checkpoint");
    LBMP_CK(h, cudaMemcpy(h->pops[h->cur], buf.data(), pb, cudaMemcpyHostToDevice));
    buf.resize((size_t)h->G.n);
    if (!get(f, buf.data(), (size_t)h->G.n)) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_load: truncated checkpoint");
    LBMP_CK(h, cudaMemcpy(h->flags[h->fcur], buf.data(), (size_t)h->G.n, cudaMemcpyHostToDevice));
    LBMP_CK(h, cudaMemcpy(h->flags[1 - h->fcur], buf.data(), (size_t)h->G.n, cudaMemcpyHostToDevice));
    h->h2d += (long long)(pb + 2 * (size_t)h->G.n);
    if (h->has_particle)
        launch_build_links(h->flags[h->fcur], h->G, h->box, h->d_ps, h->link_mask, h->link_blocks, h->list, h->count,
                           h->list_cap, h->status, h->stream);
    LBMP_CK(h, cudaStreamSynchronize(h->stream));
    return read_status(h);
}

lbmp_status lbmp_drag_forward(lbmp_handle* h, const double* u0, int nsteps, int checkpoint_interval, int axis,
                              double* J, double* forces) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    h->ps_current = false;
    if (!u0 || !J) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_drag_forward: NULL argument");
    if (nsteps < 1 || checkpoint_interval < 1 || axis < 0 || axis > 2)
        return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_drag_forward: need nsteps >= 1, checkpoint_interval >= 1, axis 0..2");
    lbmp_status s = h->has_particle ? download_particle(h) : LBMP_OK;
    if (s != LBMP_OK) return s;
    std::string why;
    s = adjoint_check(h, &why);
    if (s != LBMP_OK) return fail(h, s, "lbmp_drag_forward: " + why);
    s = adjoint_forward(h, u0, nsteps, checkpoint_interval, axis, J, forces);
    if (s == LBMP_ERR_OOM) return fail(h, s, "lbmp_drag_forward: out of device memory for the checkpoints");
    if (s != LBMP_OK) return fail(h, s, "lbmp_drag_forward: CUDA launch failed");
    return LBMP_OK;
}

lbmp_status lbmp_drag_backward(lbmp_handle* h, const double* dJ, double* grad_tau, double* grad_force,
                               double* grad_u0) {
    if (!h) return LBMP_ERR_INVALID_ARG;
    h->ps_current = false;
    if (!dJ) return fail(h, LBMP_ERR_INVALID_ARG, "lbmp_drag_backward: NULL dJ");
    std::string why;
    lbmp_status s = adjoint_check(h, &why);
    if (s != LBMP_OK) return fail(h, s, "lbmp_drag_backward: " + why);
    s = adjoint_backward(h, dJ, grad_tau, grad_force, grad_u0, &why);
    if (s == LBMP_ERR_CUDA) why = "CUDA launch failed";
    if (s != LBMP_OK) return fail(h, s, "lbmp_drag_backward: " + why);
    return LBMP_OK;
}

const char* lbmp_last_error(const lbmp_handle* h) {
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

}  // extern "C"
