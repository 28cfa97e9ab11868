// common.cuh -- device helpers and the runtime object shared by the kernel files.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "plan.hpp"

namespace hfav {

#define HFAV_CUDA(call)                                                                       \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return set_error(HFAV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// after every kernel launch: check it, count it and, when per-kernel timing
// is on, record an event so consecutive events bracket each kernel
#define HFAV_LAUNCHED(rt, name, st)                                                           \
    do {                                                                                      \
        cudaError_t e_ = cudaGetLastError();                                                  \
        if (e_ != cudaSuccess)                                                                \
            return set_error(HFAV_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
        (rt)->launches++;                                                                     \
        if ((rt)->timing && !(rt)->capturing) kt_mark((rt), (name), (st));                    \
    } while (0)

// A strided view of a grid function on the device: element (i, j, k) sits at
// p[(k + org[2]) * pitch[2] + (j + org[1]) * pitch[1] + (i + org[0])].
// wrap != 0: indices are first wrapped periodically into [0, ext).
struct GArr {
    void* p;
    int64_t pitch[3];
    int org[3];
    int ext[3];
    int wrap;
};

__host__ __device__ inline int wrap_idx(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// periodic wrap without integer division on the common paths: indices of a
// stencil lie within one period of [0, n); anything further out (the unused
// tail of a CTA tile wider than the grid) takes the general wrap
__device__ __forceinline__ int wrap1(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    if (a < 0 && a >= -n) return a + n;
    if (a >= n && a < 2 * n) return a - n;
    return wrap_idx(a, n);
}

template <typename T>
__device__ __forceinline__ T garr_ld(const GArr& a, int i, int j, int k) {
    if (a.wrap) {
        i = wrap1(i, a.ext[0]);
        j = wrap1(j, a.ext[1]);
        k = wrap1(k, a.ext[2]);
    }
    const T* p = (const T*)a.p;
    return p[(int64_t)(k + a.org[2]) * a.pitch[2] + (int64_t)(j + a.org[1]) * a.pitch[1] + (i + a.org[0])];
}

template <typename T>
__device__ __forceinline__ T* garr_ptr(const GArr& a, int i, int j, int k) {
    T* p = (T*)a.p;
    return p + (int64_t)(k + a.org[2]) * a.pitch[2] + (int64_t)(j + a.org[1]) * a.pitch[1] + (i + a.org[0]);
}

// FP64 reciprocal from the hardware estimate (rcp.approx.ftz.f64) refined
// by Newton-Raphson (a published method)
__device__ __forceinline__ double rcp_est(double b) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
    return r;
}
// reciprocal to within an ulp or two (two Newton-Raphson steps)
__device__ __forceinline__ double rcp_nr(double b) {
    double r = rcp_est(b);
    r = fma(r, fma(-b, r, 1.0), r);
    return fma(r, fma(-b, r, 1.0), r);
}
__device__ __forceinline__ float rcp_nr(float b) { return 1.0f / b; }
// quotient a / b: a * (1/b) with one residual correction
__device__ __forceinline__ double div_nr(double a, double b) {
    const double r = rcp_nr(b);
    const double q = a * r;
    return fma(r, fma(-b, q, a), q);
}
__device__ __forceinline__ float div_nr(float a, float b) { return a / b; }

// atomic max of non-negative doubles through their bit patterns (IEEE order
// of non-negative doubles equals the order of their bits as unsigned ints)
__device__ __forceinline__ void atomic_max_pos(unsigned long long* slot, double v) {
    atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Device-side state owned by a plan.
struct Runtime {
    int device = -1;
    std::vector<void*> allocs;
    std::map<std::string, void*> named;    // scratch buffers by purpose
    std::map<std::string, size_t> named_bytes;
    unsigned long long* counters = nullptr;   // [0] Newton non-converged, [1] non-physical
    unsigned long long* wave = nullptr;       // per grid, wave_cap slots of max wave speed bits
    int wave_cap = 0;
    cudaStream_t last_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int launches = 0;
    int last_launches = 0;
    int last_steps = 0;
    bool capturing = false;   // inside stream capture: no synchronous uploads
    // device tables written from the host (upload()): runs that build a graph
    // keep theirs under this prefix, apart from the plain runs' tables, and
    // copy them from pinned staging that stays fixed after the capture, so a
    // replay re-uploads exactly what was captured
    std::string upload_tag;
    std::map<std::string, std::pair<void*, size_t>> pinned;
    // per-kernel timing (events recorded after each launch of a plain run)
    bool timing = false;
    std::vector<cudaEvent_t> kpool;
    std::vector<std::string> kname;   // name of the kernel ending at event k (k >= 1)
    size_t kused = 0;
    // captured graph
    cudaGraphExec_t gexec = nullptr;
    std::vector<void*> gkey;
    int gsteps = -1;
    std::string gsched;
    cudaStream_t gstream = nullptr;
    cudaEvent_t gdone = nullptr;         // recorded after every graph launch
    cudaStream_t own = nullptr;          // capture stream when the caller passes the legacy stream
    cudaEvent_t join0 = nullptr, join1 = nullptr;
};

// record the next timing event (event 0 is recorded at the start of a run)
void kt_mark(Runtime* rt, const char* name, cudaStream_t st);

// cudaMalloc behind the library's fault injection (hfav_inject_alloc_failure)
cudaError_t dev_malloc(void** ptr, size_t bytes);
extern std::atomic<int> g_fail_alloc;

// streaming multiprocessors of the current device (queried once per device)
int device_sms();

// allocate (or reuse) a named scratch buffer of at least `bytes`; growing a
// buffer drops the plan's captured graph, which holds the old address
int scratch(hfav_plan_t* p, const std::string& name, size_t bytes, void** out);

// copy `bytes` of host data into the named device table, ordered on `st`
// after the work queued before it (the host data may be reused on return)
int upload(hfav_plan_t* p, const std::string& name, const void* host, size_t bytes, cudaStream_t st, void** dev);

// launchers (chain.cu / godunov.cu)
int launch_chain2d(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, cudaStream_t st);
int launch_cosmo(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, cudaStream_t st);
int launch_chain3d(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, cudaStream_t st);
int launch_generic(hfav_plan_t* p, void* const* ax, void* const* go, cudaStream_t st);
// codegen.cu: generated kernels of DAGs with user rule bodies (HFAV_OP_EXPR)
int launch_codegen(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, cudaStream_t st);
// one generated kernel for one rule of the unfused form: ref_slot[r] is the
// entry of `ins` that input r reads; out is written over lo .. lo + n - 1
int launch_cg_rule(hfav_plan_t* p, const Rule& R, const std::vector<int>& ref_slot, const std::vector<GArr>& ins,
                   const GArr& out, const int* lo, const int* n, cudaStream_t st);
int launch_godunov(hfav_plan_t* p, const Schedule& s, void* const* ax, void* const* go, int n_steps,
                   cudaStream_t st);

}  // namespace hfav
