// Batched sweep engine (batch.cu): independent uniform periodic simulations
// of different sizes advanced together, one launch per phase for all of them.
#pragma once

#include "internal.h"

namespace lbmp {

lbmp_status batch_create(lbmp_handle* h, const lbmp_batch_sim* sims, int n);
void batch_destroy(lbmp_handle* h);
lbmp_status batch_step(lbmp_handle* h, int n);
lbmp_status batch_autotune(lbmp_handle* h, int reps);
lbmp_status batch_get_particle(lbmp_handle* h, int sim, ParticleState* out);
lbmp_status batch_set_particle(lbmp_handle* h, int sim, const ParticleState* in);
lbmp_status batch_history(lbmp_handle* h, int sim, double* ring, int cap);
lbmp_status batch_populations(lbmp_handle* h, int sim, double* out, size_t cap);
void batch_info(const lbmp_handle* h, int64_t out[8]);

}  // namespace lbmp
