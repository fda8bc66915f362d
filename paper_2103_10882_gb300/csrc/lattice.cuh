// D3Q19 lattice, storage types and small device helpers shared by the
// kernels of this library (Sec. 2.1: D3Q19 velocity set, c_s^2 = 1/3,
// lattice units dx = dt = rho_0 = 1).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmp {

// Direction q: 0 rest, 1..6 faces, 7..18 edges; opposite pairs are (odd, odd+1).
// Components are packed two bits per direction (value + 1), so a run-time q
// costs a shift and a mask instead of a table in local memory.
//   cx: 0, 1,-1, 0, 0, 0, 0, 1,-1, 1,-1, 1,-1, 1,-1, 0, 0, 0, 0
//   cy: 0, 0, 0, 1,-1, 0, 0, 1,-1,-1, 1, 0, 0, 0, 0, 1,-1, 1,-1
//   cz: 0, 0, 0, 0, 0, 1,-1, 0, 0, 0, 0, 1,-1,-1, 1, 1,-1,-1, 1
__host__ __device__ constexpr unsigned long long pack_dirs(const int (&v)[19]) {
    unsigned long long p = 0;
    for (int q = 0; q < 19; ++q) p |= (unsigned long long)(v[q] + 1) << (2 * q);
    return p;
}
constexpr int kCX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
constexpr int kCY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
constexpr int kCZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
constexpr unsigned long long kPX = pack_dirs(kCX), kPY = pack_dirs(kCY), kPZ = pack_dirs(kCZ);
__host__ __device__ constexpr int cx(int q) { return (int)((kPX >> (2 * q)) & 3ull) - 1; }
__host__ __device__ constexpr int cy(int q) { return (int)((kPY >> (2 * q)) & 3ull) - 1; }
__host__ __device__ constexpr int cz(int q) { return (int)((kPZ >> (2 * q)) & 3ull) - 1; }
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
// weights: 1/3 rest, 1/18 faces, 1/36 edges
template <typename T>
__host__ __device__ constexpr T wgt(int q) {
    return q == 0 ? T(1) / T(3) : (q <= 6 ? T(1) / T(18) : T(1) / T(36));
}

// Storage of one population deviation g = f - w.
//   double : FP64 storage, FP64 arithmetic
//   float  : FP32 storage, FP32 arithmetic
//   __half : FP16 storage of g * 2^s, FP32 arithmetic
template <typename S>
struct Store;
template <>
struct Store<double> {
    using A = double;
    __device__ static __forceinline__ A load(const double* p, A) { return __ldg(p); }
    __device__ static __forceinline__ void store(double* p, A v, A) { __stcs(p, v); }
    __device__ static __forceinline__ A load_raw(const double* p) { return __ldg(p); }
    __device__ static __forceinline__ void store_raw(double* p, A v) { __stcs(p, v); }
};
template <>
struct Store<float> {
    using A = float;
    __device__ static __forceinline__ A load(const float* p, A) { return __ldg(p); }
    __device__ static __forceinline__ void store(float* p, A v, A) { __stcs(p, v); }
    __device__ static __forceinline__ A load_raw(const float* p) { return __ldg(p); }
    __device__ static __forceinline__ void store_raw(float* p, A v) { __stcs(p, v); }
};
template <>
struct Store<__half> {
    using A = float;
    // inv_scale = 2^-s on load, scale = 2^s on store (exact power-of-two scaling)
    __device__ static __forceinline__ A load(const __half* p, A inv_scale) {
        return __half2float(__ldg(p)) * inv_scale;
    }
    __device__ static __forceinline__ void store(__half* p, A v, A scale) { *p = __float2half_rn(v * scale); }
    // the stored value g * 2^s itself (kernels that work on the scaled values)
    __device__ static __forceinline__ A load_raw(const __half* p) { return __half2float(__ldg(p)); }
    __device__ static __forceinline__ void store_raw(__half* p, A v) { *p = __float2half_rn(v); }
};

// Device-resident state of the sphere, FP64 throughout (Sec. 2.2, 3.3).
struct ParticleState {
    double x[3];       // centre
    double u[3];       // translational velocity seen by the fluid, u(t + 1/2)
    double w[3];       // angular velocity, omega(t + 1/2)
    double a[3];       // a_p of the previous step
    double b[3];       // beta_p of the previous step
    double Fh[3], Th[3];          // hydrodynamic force/torque of the last step
    double Fh_old[3], Th_old[3];  // and of the step before
    double Fp[3];                 // total force of the last step
    double g[3];                  // gravitational acceleration
    double D, r, rho_p, cv, cvw, V;
    long long steps;
    int present;
    int fixed;         // held degrees of freedom: 0 none, 1 translation and rotation, 2 translation only
    int force_average;
    int prev_fixed;    // the value of fixed in the previous step
};

static_assert(sizeof(ParticleState) % sizeof(int) == 0, "particle record is copied as ints");

// Status bits written by kernels (read by the host after a step).
enum : int { STATUS_UNSTABLE_FLUID = 1, STATUS_PARTICLE_JUMP = 2, STATUS_LINK_OVERFLOW = 4 };

}  // namespace lbmp
