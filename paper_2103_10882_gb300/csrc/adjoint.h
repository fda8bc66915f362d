// Drag adjoint on the uniform grid (adjoint.cu): the C ABI calls
// lbmp_drag_forward and lbmp_drag_backward dispatch here.
#pragma once

#include <string>

#include "internal.h"

namespace lbmp {

// LBMP_OK when the handle is a uniform periodic grid with one sphere held
// fixed at rest in FP32 or FP64 storage; otherwise the reason in *why.
lbmp_status adjoint_check(const lbmp_handle* h, std::string* why);
// J = (1/nsteps) sum_n F_axis^n from the equilibrium of u0 (device [3][cells]);
// keeps every interval-th state for the reverse pass.  J is a device double,
// forces (device [nsteps][3], may be null) receives the force of every step.
lbmp_status adjoint_forward(lbmp_handle* h, const double* u0, int nsteps, int interval, int axis, double* J,
                            double* forces);
// dJ/dtau, dJ/dF (3) and dJ/du0 ([3][cells]) times the device scalar dJ; any output may be null.
lbmp_status adjoint_backward(lbmp_handle* h, const double* dJ, double* grad_tau, double* grad_force, double* grad_u0,
                             std::string* why);
void adjoint_destroy(lbmp_handle* h);

}  // namespace lbmp
