// noalloc.cu -- an allocation-free entry point for the 2D three-stage chain.
//
// The "sweep" schedule of the 2D chain keeps its first stage L in a full
// device array that the plan allocates on first use.  Some callers cannot do
// that: a host application whose own pool owns all of the device's memory,
// a latency-critical loop that must not hit cudaMalloc's implicit device
// synchronisation after start-up, or a caller that has no torch or plan
// object at all.  hfav_chain2d_static runs the same computation with L in a
// file-scope device array that the library carries instead:
//   - capacity HFAV_STATIC_SCRATCH_BYTES (16 MiB), i.e. (nx+2)*(ny+2) doubles;
//     larger grids are rejected with HFAV_EINVAL before any device work;
//   - the array belongs to this file's device module.  With lazy module
//     loading (the CUDA default) the module, and with it the 16 MiB, is loaded
//     on a device by the first call there, which looks the array's device
//     address up with cudaGetSymbolAddress while that device is current (once
//     per device); from then on the device holds the array until the process
//     exits.  Make that first call at start-up, before any stream capture and
//     before a memory pool takes the rest of the device: if the device has no
//     16 MiB left then, the call fails with HFAV_ENOMEM;
//   - the address is cached per device for the life of the process: after a
//     cudaDeviceReset the module is loaded again, possibly elsewhere, so this
//     entry point must not be used across a device reset;
//   - the array is shared by every call: each call overwrites all of L it
//     reads, so nothing has to start at zero, and calls whose device work
//     overlaps (different streams, no ordering) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "common.cuh"

#define HFAV_STATIC_SCRATCH_BYTES (16u << 20)
#define HFAV_STATIC_MAX_DEVICES 64

namespace hfav {

static __device__ __align__(256) double g_chain2d_scratch[HFAV_STATIC_SCRATCH_BYTES / sizeof(double)];

namespace {

std::mutex g_static_mu;
double* g_static_addr[HFAV_STATIC_MAX_DEVICES] = {};
int g_static_blocks[HFAV_STATIC_MAX_DEVICES] = {};   // grid cap: 16 CTAs per SM

// device address of the scratch array for the current device (host code may
// not use the symbol's name as an address) and the grid-size cap there
int static_scratch(double** out, int* blocks) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(HFAV_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= HFAV_STATIC_MAX_DEVICES) return set_error(HFAV_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_chain2d_scratch);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return set_error(HFAV_ENOMEM, "loading the static scratch array (16 MiB) on this device: out of memory");
        }
        if (e != cudaSuccess || !p)
            return set_error(HFAV_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        int n = device_sms();
        g_static_addr[dev] = (double*)p;
        g_static_blocks[dev] = 16 * (n > 0 ? n : 1);
    }
    *out = g_static_addr[dev];
    *blocks = g_static_blocks[dev];
    return HFAV_OK;
}

struct StaticArgs {
    const double* u;
    int64_t pu;       // row pitch of u and out (elements)
    int hu;           // halo of u and out
    int nx, ny, wrap;
    double w[5];      // weights of u(i+1), u(i-1), u(j+1), u(j-1), u(i, j)
    double* L;        // (ny+2) x (nx+2), L(i, j) at (j+1)*(nx+2) + (i+1)
    double* out;
};

__device__ __forceinline__ double ld_static(const StaticArgs& a, int i, int j) {
    if (a.wrap) {
        i %= a.nx; i += i < 0 ? a.nx : 0;
        j %= a.ny; j += j < 0 ? a.ny : 0;
    }
    return a.u[(int64_t)(j + a.hu) * a.pu + (i + a.hu)];
}

// stage 1: L on the halo-1 ring [-1, nx] x [-1, ny]
__global__ void __launch_bounds__(256) static_lap(const StaticArgs a) {
    const int W = a.nx + 2;
    const int64_t n = (int64_t)W * (a.ny + 2);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % W) - 1, j = (int)(k / W) - 1;
        double v = a.w[0] * ld_static(a, i + 1, j);
        v = fma(a.w[1], ld_static(a, i - 1, j), v);
        v = fma(a.w[2], ld_static(a, i, j + 1), v);
        v = fma(a.w[3], ld_static(a, i, j - 1), v);
        a.L[k] = fma(a.w[4], ld_static(a, i, j), v);
    }
}

// stages 2-3: G = |central grad L| / 2, out = G / (1 + G) on the interior
__global__ void __launch_bounds__(256) static_tail(const StaticArgs a) {
    const int W = a.nx + 2;
    const int64_t n = (int64_t)a.nx * a.ny;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % a.nx), j = (int)(k / a.nx);
        const double* L = a.L + (int64_t)(j + 1) * W + (i + 1);
        const double gx = L[1] - L[-1], gy = L[W] - L[-W];
        const double G = sqrt(fma(gx, gx, gy * gy)) * 0.5;
        a.out[(int64_t)(j + a.hu) * a.pu + (i + a.hu)] = G / (1.0 + G);
    }
}

}  // namespace
}  // namespace hfav

using namespace hfav;

extern "C" int hfav_chain2d_static(const double* u, int64_t nx, int64_t ny, int64_t pitch, int halo, int bc,
                                   const double* weights, double* out, void* stream) {
    if (!u || !out) return set_error(HFAV_EINVAL, "null array");
    if (nx < 2 || ny < 2 || nx > (1 << 30) || ny > (1 << 30)) return set_error(HFAV_EINVAL, "bad extents");
    if (bc != HFAV_BC_PERIODIC && bc != HFAV_BC_HALO_GIVEN) return set_error(HFAV_EINVAL, "bad bc");
    if (halo < 0 || (bc == HFAV_BC_HALO_GIVEN && halo < 2)) return set_error(HFAV_EHALO, "halo-given mode needs halo >= 2");
    if (pitch < nx + 2 * halo) return set_error(HFAV_EHALO, "pitch smaller than the padded row");
    {   // u and out span the same padded layout; they must not overlap at all
        const uint64_t span = ((uint64_t)(ny + 2 * halo - 1) * (uint64_t)pitch + (uint64_t)(nx + 2 * halo)) * sizeof(double);
        const uintptr_t a0 = (uintptr_t)u, b0 = (uintptr_t)out;
        if (a0 < b0 + span && b0 < a0 + span) return set_error(HFAV_EINVAL, "out overlaps u");
    }
    const uint64_t need = (uint64_t)(nx + 2) * (uint64_t)(ny + 2) * sizeof(double);
    if (need > HFAV_STATIC_SCRATCH_BYTES)
        return set_error(HFAV_EINVAL, "grid needs " + std::to_string(need) + " bytes of scratch; the static buffer holds " +
                                          std::to_string(HFAV_STATIC_SCRATCH_BYTES) + " ((nx+2)*(ny+2) doubles)");
    double* L = nullptr;
    int cap = 1;
    int rc = static_scratch(&L, &cap);
    if (rc) return rc;
    StaticArgs a;
    a.u = u; a.pu = pitch; a.hu = halo;
    a.nx = (int)nx; a.ny = (int)ny; a.wrap = bc == HFAV_BC_PERIODIC;
    const double def[5] = {1.0, 1.0, 1.0, 1.0, -4.0};
    for (int k = 0; k < 5; ++k) a.w[k] = weights ? weights[k] : def[k];
    a.L = L;
    a.out = out;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n1 = (nx + 2) * (ny + 2);
    const int b1 = (int)((n1 + 255) / 256 < cap ? (n1 + 255) / 256 : cap);
    static_lap<<<b1, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HFAV_ECUDA, std::string("static_lap: ") + cudaGetErrorString(e));
    const int64_t n2 = nx * ny;
    const int b2 = (int)((n2 + 255) / 256 < cap ? (n2 + 255) / 256 : cap);
    static_tail<<<b2, 256, 0, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(HFAV_ECUDA, std::string("static_tail: ") + cudaGetErrorString(e));
    return HFAV_OK;
}
