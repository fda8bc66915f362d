// Refined-grid engine (amr.cu): block-structured levels of 16^3 cells with
// 2:1 balance, sub-cycling, explosion and coalescence (Sec. 4.1), the
// particle refinement criterion and regrid (Sec. 4.2.1), and the coupling of
// Algorithm 1 on the finest level.  Used by the C ABI when levels > 1.
#pragma once

#include <cstdio>

#include "internal.h"

namespace lbmp {

lbmp_status amr_cuda_error(lbmp_handle* h, const char* where);   // records the CUDA error text in h->err
lbmp_status amr_create(lbmp_handle* h);   // sets h->amr; starts unrefined (all level 0)
void amr_destroy(lbmp_handle* h);
lbmp_status amr_add_sphere(lbmp_handle* h);            // h->h_ps filled by the caller
lbmp_status amr_refine_box(lbmp_handle* h, const double lo[3], const double hi[3]);
lbmp_status amr_regrid(lbmp_handle* h);                 // with the flow sensor when it is on
lbmp_status amr_set_sensor(lbmp_handle* h, double sigma, double c);   // arguments checked by the caller
lbmp_status amr_block_sensor(lbmp_handle* h, int level, double* out, size_t cap, size_t* n);
lbmp_status amr_init_fluid(lbmp_handle* h, double rho, const double u[3], double amp, int dir, int axis);
lbmp_status amr_step(lbmp_handle* h, int n_coarse);   // enqueues; status read by the caller
lbmp_status amr_level_shape(lbmp_handle* h, int level, int out[3]);
lbmp_status amr_block_map(lbmp_handle* h, int level, int32_t* out, size_t cap, size_t* n);
lbmp_status amr_level_cells(lbmp_handle* h, int level, int32_t* xyz, double* g, size_t cap, size_t* n);
lbmp_status amr_level_flags(lbmp_handle* h, int level, uint8_t* out, size_t cap, size_t* n);
lbmp_status amr_links(lbmp_handle* h, int64_t* cell, int32_t* q, double* delta, size_t cap, size_t* n);
lbmp_status amr_save(lbmp_handle* h, FILE* f);   // refined part of a checkpoint
lbmp_status amr_load(lbmp_handle* h, FILE* f);   // after the particle record is on the device
long long amr_cell_updates_per_coarse_step(const lbmp_handle* h);
int amr_launches_per_coarse_step(const lbmp_handle* h);

}  // namespace lbmp
