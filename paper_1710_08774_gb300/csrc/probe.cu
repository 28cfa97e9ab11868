// probe.cu -- measured arithmetic peaks of the current device, the
// denominators of the ALU rooflines of the FP64 workloads.
//
// Each probe kernel runs eight independent dependency chains of one
// operation per thread (enough independent work to keep the pipe busy at
// full occupancy) on 8 CTAs of 256 threads per SM, and is timed with CUDA
// events after a warm-up launch.  The FP64 divide, square root and
// reciprocal square root are CUDA's own (IEEE '/', sqrt, rsqrt); their rates
// divided into the DFMA rate give their cost in DFMA issue slots.
#include <cuda_runtime.h>

#include <string>

#include "common.cuh"

namespace hfav {
namespace {

__device__ double g_probe_sink;
__device__ float g_probe_sinkf;

enum { P_DFMA = 0, P_DDIV = 1, P_DSQRT = 2, P_DRSQRT = 3 };

// the divide, square root and reciprocal square root sequences need more
// registers: four CTAs per SM keep their eight chains out of local memory
template <int OP>
__global__ void __launch_bounds__(256, OP == P_DFMA ? 8 : 4) probe_fp64(int iters, double seed) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = seed + 0.125 * k + 1e-6 * threadIdx.x;
    const double a = 0.9999999, b = 1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if constexpr (OP == P_DFMA) x[k] = fma(x[k], a, b);
            else if constexpr (OP == P_DDIV) x[k] = 1.5 / x[k];
            else if constexpr (OP == P_DSQRT) x[k] = sqrt(x[k]);
            else x[k] = rsqrt(x[k]);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.678) g_probe_sink = s;   // keeps the chains live; never true
}

__global__ void __launch_bounds__(256, 8) probe_ffma(int iters, float seed) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = seed + 0.125f * k + 1e-6f * threadIdx.x;
    const float a = 0.9999999f, b = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.678f) g_probe_sinkf = s;
}

// operations per second of one probe: threads x 8 chains x iters / time
template <typename K, typename S>
int time_probe(K kern, S seed, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double* rate) {
    const int blocks = device_sms() * 8;
    kern<<<blocks, 256, 0, st>>>(iters / 8 > 0 ? iters / 8 : 1, seed);   // warm-up (clocks, module load)
    HFAV_CUDA(cudaGetLastError());
    HFAV_CUDA(cudaEventRecord(e0, st));
    kern<<<blocks, 256, 0, st>>>(iters, seed);
    HFAV_CUDA(cudaGetLastError());
    HFAV_CUDA(cudaEventRecord(e1, st));
    HFAV_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    HFAV_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms <= 0.f) return set_error(HFAV_ECUDA, "probe timing failed");
    *rate = (double)blocks * 256.0 * 8.0 * iters / (ms * 1e-3);
    return HFAV_OK;
}

}  // namespace
}  // namespace hfav

extern "C" int hfav_probe_peaks(double* rates, int n, void* stream) {
    using namespace hfav;
    if (!rates || n < 5) return set_error(HFAV_EINVAL, "rates needs 5 entries");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    HFAV_CUDA(cudaEventCreate(&e0));
    HFAV_CUDA(cudaEventCreate(&e1));
    int rc = time_probe(probe_fp64<P_DFMA>, 1.0, 4096, st, e0, e1, &rates[0]);
    if (!rc) rc = time_probe(probe_fp64<P_DDIV>, 1.0, 512, st, e0, e1, &rates[1]);
    if (!rc) rc = time_probe(probe_fp64<P_DSQRT>, 2.0, 512, st, e0, e1, &rates[2]);
    if (!rc) rc = time_probe(probe_fp64<P_DRSQRT>, 2.0, 512, st, e0, e1, &rates[3]);
    if (!rc) rc = time_probe(probe_ffma, 1.0f, 32768, st, e0, e1, &rates[4]);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
