// Boundary-cell list of one sphere computed without allocating anything.
//
// Some callers cannot call cudaMalloc: a time-critical loop in which
// cudaMalloc's possible device-wide synchronisation is not acceptable, or a
// process whose device memory is entirely handed out by another allocator.
// lbmp_boundary_cells_noalloc serves them: the caller passes the flags and
// the output buffers, and the two kernels below keep their scratch (a mask
// byte per box cell and a count per thread block) in one file-scope device
// array of fixed size instead of memory from an allocator.  The call itself
// uses the CUDA runtime (it launches kernels), so it must not be made from a
// host function enqueued on a stream (cudaLaunchHostFunc), where CUDA
// forbids runtime calls.
//
// The array is shared by every call on a device and keeps the last call's
// contents; every entry a call reads has been written earlier in the same
// call, so nothing needs clearing.  Calls that overlap on the GPU (two
// streams, or two host threads) race on it and must be serialised by the
// caller.
//
// The first call on a device looks up the array's device address and
// launches the two kernels for the first time; with lazy module loading
// that loads this file's module, which backs the array and may synchronise
// the device.  A caller that needs every call free of such work makes one
// warm-up call outside its critical loop (and before any stream capture).
// The address is kept for the life of the process: after cudaDeviceReset
// (or any other teardown of the device's primary context) the call must not
// be used again in that process.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "internal.h"

namespace lbmp {
void set_global_error(const std::string& msg);   // defined in api.cu
}

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BOX_CELLS = 1 << 18;                       // 262144 box cells (64^3)
constexpr int NA_MAX_BLOCKS = NA_MAX_BOX_CELLS / NA_THREADS;     // 1024 per-block counts
constexpr size_t NA_SCRATCH_BYTES = (size_t)NA_MAX_BOX_CELLS + sizeof(int) * NA_MAX_BLOCKS;

// Scratch: [0, NA_MAX_BOX_CELLS) mask bytes, then NA_MAX_BLOCKS ints.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

struct Box {
    int o[3];     // first cell per axis (before wrapping)
    int E[3];     // extent per axis
    int n[3];     // domain extent
    int periodic[3];
    int cells;
};

__device__ __forceinline__ bool na_box_cell(int t, const Box& B, int* c) {
    const int tk = t / (B.E[0] * B.E[1]);
    const int r = t - tk * B.E[0] * B.E[1];
    const int tt[3] = {r - (r / B.E[0]) * B.E[0], r / B.E[0], tk};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int v = B.o[a] + tt[a];
        if (v < 0 || v >= B.n[a]) {
            if (!B.periodic[a]) return false;
            v = v < 0 ? v + B.n[a] : v - B.n[a];
            if (v < 0 || v >= B.n[a]) return false;
        }
        c[a] = v;
    }
    return true;
}

__device__ __forceinline__ int na_cx(int q) {
    constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[q];
}
__device__ __forceinline__ int na_cy(int q) {
    constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[q];
}
__device__ __forceinline__ int na_cz(int q) {
    constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[q];
}

__global__ void __launch_bounds__(NA_THREADS)
    k_na_mark(const uint8_t* __restrict__ flags, Box B, unsigned char* __restrict__ scratch) {
    uint8_t* mask = scratch;
    int* block_count = reinterpret_cast<int*>(scratch + NA_MAX_BOX_CELLS);
    const int t = blockIdx.x * NA_THREADS + threadIdx.x;
    int is_b = 0;
    if (t < B.cells) {
        int c[3];
        if (na_box_cell(t, B, c)) {
            const int nx = B.n[0], ny = B.n[1], nz = B.n[2];
            if (flags[c[0] + nx * (c[1] + ny * c[2])] == 0) {
#pragma unroll
                for (int q = 1; q < 19; ++q) {
                    int v[3] = {c[0] + na_cx(q), c[1] + na_cy(q), c[2] + na_cz(q)};
                    bool ok = true;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if (v[a] < 0 || v[a] >= B.n[a]) {
                            if (!B.periodic[a]) ok = false;
                            v[a] = v[a] < 0 ? v[a] + B.n[a] : v[a] - B.n[a];
                        }
                    }
                    if (ok) is_b |= flags[v[0] + nx * (v[1] + ny * v[2])] != 0;
                }
            }
        }
        mask[t] = (uint8_t)is_b;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, is_b);
    __shared__ int wsum[NA_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(ballot);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < NA_THREADS / 32; ++w) s += wsum[w];
        block_count[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(NA_THREADS)
    k_na_emit(Box B, const unsigned char* __restrict__ scratch, int* __restrict__ list, int capacity,
              int* __restrict__ count) {
    const uint8_t* mask = scratch;
    const int* block_count = reinterpret_cast<const int*>(scratch + NA_MAX_BOX_CELLS);
    __shared__ int red[NA_THREADS];
    __shared__ int wsum[NA_THREADS / 32];
    int s = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += NA_THREADS) s += block_count[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = NA_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    const int base = red[0];
    const int t = blockIdx.x * NA_THREADS + threadIdx.x;
    const int is_b = t < B.cells ? mask[t] : 0;
    const unsigned ballot = __ballot_sync(0xffffffffu, is_b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = __popc(ballot);
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += wsum[w];
    if (is_b) {
        int c[3];
        na_box_cell(t, B, c);
        const int pos = base + wbase + __popc(ballot & ((1u << lane) - 1u));
        if (pos < capacity) list[pos] = c[0] + B.n[0] * (c[1] + B.n[1] * c[2]);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        int tot = base;
        for (int w = 0; w < NA_THREADS / 32; ++w) tot += wsum[w];
        *count = tot;   // may exceed capacity: the caller compares
    }
}

// Device address of the scratch array, looked up once per device.
constexpr int NA_MAX_DEVICES = 64;
unsigned char* g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mutex;

lbmp_status scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        lbmp::set_global_error("lbmp_boundary_cells_noalloc: no current CUDA device");
        return LBMP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            lbmp::set_global_error(std::string("lbmp_boundary_cells_noalloc: cudaGetSymbolAddress: ") +
                                   cudaGetErrorString(e));
            return LBMP_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return LBMP_OK;
}

}  // namespace

extern "C" lbmp_status lbmp_boundary_cells_noalloc(const uint8_t* flags, int nx, int ny, int nz,
                                                   const int periodic[3], const double center[3], double diameter,
                                                   int* list, int capacity, int* count, uintptr_t cuda_stream) {
    if (!flags || !periodic || !center || !list || !count || capacity < 0) {
        lbmp::set_global_error("lbmp_boundary_cells_noalloc: NULL argument or negative capacity");
        return LBMP_ERR_INVALID_ARG;
    }
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz >= (1LL << 31) || !(diameter > 0.0)) {
        lbmp::set_global_error("lbmp_boundary_cells_noalloc: bad grid extents or diameter");
        return LBMP_ERR_INVALID_ARG;
    }
    Box B;
    const int n3[3] = {nx, ny, nz};
    const int R = (int)std::ceil(0.5 * diameter) + 3;   // same box as the coupled step's remap
    long long cells = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(center[a] >= 0.0 && center[a] <= (double)n3[a])) {
            lbmp::set_global_error("lbmp_boundary_cells_noalloc: centre outside the domain");
            return LBMP_ERR_INVALID_ARG;
        }
        B.n[a] = n3[a];
        B.periodic[a] = periodic[a] ? 1 : 0;
        B.E[a] = 2 * R + 2;
        B.o[a] = (int)std::floor(center[a] - 0.5) - R;
        if (B.E[a] >= n3[a]) {   // the box spans the axis, periodic or not: the coupled step starts it at 0
            B.E[a] = n3[a];
            B.o[a] = 0;
        }
        cells *= B.E[a];
    }
    if (cells > NA_MAX_BOX_CELLS) {
        lbmp::set_global_error("lbmp_boundary_cells_noalloc: the sphere's box has " + std::to_string(cells) +
                               " cells, more than the fixed scratch holds (" + std::to_string(NA_MAX_BOX_CELLS) +
                               " cells, a sphere diameter of at most 56 cells)");
        return LBMP_ERR_INVALID_ARG;
    }
    B.cells = (int)cells;
    unsigned char* scratch = nullptr;
    const lbmp_status st = scratch_for_current_device(&scratch);
    if (st != LBMP_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int nb = (B.cells + NA_THREADS - 1) / NA_THREADS;
    k_na_mark<<<nb, NA_THREADS, 0, stream>>>(flags, B, scratch);
    k_na_emit<<<nb, NA_THREADS, 0, stream>>>(B, scratch, list, capacity, count);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        lbmp::set_global_error(std::string("lbmp_boundary_cells_noalloc: launch: ") + cudaGetErrorString(e));
        return LBMP_ERR_CUDA;
    }
    return LBMP_OK;
}
