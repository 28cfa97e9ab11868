// mlp.cu -- the learned schedule model: a 3-layer MLP (n_in -> H -> H -> 1,
// ReLU) with hand-written FP32 forward, backward (MSE) and Adam kernels, and
// the host loops that train it and use it to pick a plan's schedule.
//
// Parameter layout (one device array, row-major):
//   W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1]
// The network is tiny (H = 64): one thread per row keeps its activations in
// registers and reads the weights from shared memory; weight gradients are
// row sums (one thread per weight, fixed summation order, no atomics), so a
// gradient is bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace hfav {

#define MLP_HMAX 128
#define MLP_INMAX 32

struct MlpDims {
    int n_in, H;
    int64_t oW1, ob1, oW2, ob2, ow3, ob3, n_params;
};

__host__ __device__ inline MlpDims mlp_dims(int n_in, int H) {
    MlpDims d;
    d.n_in = n_in; d.H = H;
    d.oW1 = 0; d.ob1 = d.oW1 + (int64_t)H * n_in; d.oW2 = d.ob1 + H; d.ob2 = d.oW2 + (int64_t)H * H;
    d.ow3 = d.ob2 + H; d.ob3 = d.ow3 + H; d.n_params = d.ob3 + 1;
    return d;
}

// forward (and, when work != null, the backward activations) of one row per thread
template <bool TRAIN>
__global__ void __launch_bounds__(128) mlp_rows(const float* __restrict__ params, MlpDims d, const float* __restrict__ X,
                                               const float* __restrict__ t, int n, float* __restrict__ y,
                                               float* __restrict__ work) {
    extern __shared__ float sp[];
    for (int64_t k = threadIdx.x; k < d.n_params; k += blockDim.x) sp[k] = params[k];
    __syncthreads();
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int H = d.H, NI = d.n_in;
    float x[MLP_INMAX];
    for (int k = 0; k < NI; ++k) x[k] = X[(int64_t)row * NI + k];
    float h1[MLP_HMAX], h2[MLP_HMAX];
    for (int h = 0; h < H; ++h) {
        float a = sp[d.ob1 + h];
        for (int k = 0; k < NI; ++k) a = fmaf(sp[d.oW1 + h * NI + k], x[k], a);
        h1[h] = fmaxf(a, 0.f);
    }
    float out = sp[d.ob3];
    for (int h = 0; h < H; ++h) {
        float a = sp[d.ob2 + h];
        for (int m = 0; m < H; ++m) a = fmaf(sp[d.oW2 + h * H + m], h1[m], a);
        h2[h] = fmaxf(a, 0.f);
        out = fmaf(sp[d.ow3 + h], h2[h], out);
    }
    if (!TRAIN) { y[row] = out; return; }
    // d loss / d out for loss = mean (out - t)^2
    const float dy = 2.f * (out - t[row]) / (float)n;
    float* w = work + (int64_t)row * (4 * H + 2);   // h1 | h2 | dh1 | dh2 | dy | sq
    float dh2[MLP_HMAX];
    for (int h = 0; h < H; ++h) {
        w[h] = h1[h];
        w[H + h] = h2[h];
        dh2[h] = h2[h] > 0.f ? dy * sp[d.ow3 + h] : 0.f;
        w[3 * H + h] = dh2[h];
    }
    for (int m = 0; m < H; ++m) {
        float a = 0.f;
        for (int h = 0; h < H; ++h) a = fmaf(sp[d.oW2 + h * H + m], dh2[h], a);
        w[2 * H + m] = h1[m] > 0.f ? a : 0.f;
    }
    w[4 * H] = dy;
    w[4 * H + 1] = (out - t[row]) * (out - t[row]);
}

// one thread per parameter: sums over rows in row order
__global__ void __launch_bounds__(256) mlp_grad(MlpDims d, const float* __restrict__ X, int n,
                                                const float* __restrict__ work, float* __restrict__ grad,
                                                float* __restrict__ loss) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int H = d.H, NI = d.n_in, WS = 4 * H + 2;
    if (k == d.n_params) {   // the loss itself
        float s = 0.f;
        for (int r = 0; r < n; ++r) s += work[(int64_t)r * WS + 4 * H + 1];
        *loss = s / (float)n;
        return;
    }
    if (k > d.n_params) return;
    float s = 0.f;
    if (k < d.ob1) {                       // W1[h][i] = sum dh1[h] x[i]
        int h = (int)(k / NI), i = (int)(k % NI);
        for (int r = 0; r < n; ++r) s = fmaf(work[(int64_t)r * WS + 2 * H + h], X[(int64_t)r * NI + i], s);
    } else if (k < d.oW2) {                // b1[h]
        int h = (int)(k - d.ob1);
        for (int r = 0; r < n; ++r) s += work[(int64_t)r * WS + 2 * H + h];
    } else if (k < d.ob2) {                // W2[h][m] = sum dh2[h] h1[m]
        int64_t q = k - d.oW2;
        int h = (int)(q / H), m = (int)(q % H);
        for (int r = 0; r < n; ++r) s = fmaf(work[(int64_t)r * WS + 3 * H + h], work[(int64_t)r * WS + m], s);
    } else if (k < d.ow3) {                // b2[h]
        int h = (int)(k - d.ob2);
        for (int r = 0; r < n; ++r) s += work[(int64_t)r * WS + 3 * H + h];
    } else if (k < d.ob3) {                // w3[h] = sum dy h2[h]
        int h = (int)(k - d.ow3);
        for (int r = 0; r < n; ++r) s = fmaf(work[(int64_t)r * WS + 4 * H], work[(int64_t)r * WS + H + h], s);
    } else {                               // b3
        for (int r = 0; r < n; ++r) s += work[(int64_t)r * WS + 4 * H];
    }
    grad[k] = s;
}

__global__ void mlp_adam_k(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        float gk = g[k];
        float mk = b1 * m[k] + (1.f - b1) * gk;
        float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

namespace {
int mlp_check(int n_in, int hidden) {
    if (n_in < 1 || n_in > MLP_INMAX) return set_error(HFAV_EINVAL, "n_in must be in [1, 32]");
    if (hidden < 1 || hidden > MLP_HMAX) return set_error(HFAV_EINVAL, "hidden must be in [1, 128]");
    return HFAV_OK;
}
size_t mlp_smem(const MlpDims& d) { return (size_t)d.n_params * sizeof(float); }
}  // namespace

}  // namespace hfav

using namespace hfav;

extern "C" {

int64_t hfav_mlp_n_params(int n_in, int hidden) { return mlp_dims(n_in, hidden).n_params; }

int64_t hfav_mlp_work_floats(int n, int hidden) { return (int64_t)n * (4 * hidden + 2); }

int hfav_mlp_forward(const float* params, int n_in, int hidden, const float* X, int n, float* y, void* stream) {
    int rc = mlp_check(n_in, hidden);
    if (rc) return rc;
    if (!params || !X || !y || n < 0) return set_error(HFAV_EINVAL, "bad argument");
    if (n == 0) return HFAV_OK;
    MlpDims d = mlp_dims(n_in, hidden);
    size_t sm = mlp_smem(d);
    if (sm > 200 * 1024) return set_error(HFAV_EINVAL, "network too large");
    HFAV_CUDA(cudaFuncSetAttribute(mlp_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    mlp_rows<false><<<(n + 127) / 128, 128, sm, (cudaStream_t)stream>>>(params, d, X, nullptr, n, y, nullptr);
    HFAV_CUDA(cudaGetLastError());
    return HFAV_OK;
}

int hfav_mlp_loss_grad(const float* params, int n_in, int hidden, const float* X, const float* t, int n, float* grad,
                       float* loss, float* work, void* stream) {
    int rc = mlp_check(n_in, hidden);
    if (rc) return rc;
    if (!params || !X || !t || !grad || !loss || !work || n < 1) return set_error(HFAV_EINVAL, "bad argument");
    MlpDims d = mlp_dims(n_in, hidden);
    size_t sm = mlp_smem(d);
    if (sm > 200 * 1024) return set_error(HFAV_EINVAL, "network too large");
    cudaStream_t st = (cudaStream_t)stream;
    HFAV_CUDA(cudaFuncSetAttribute(mlp_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    mlp_rows<true><<<(n + 127) / 128, 128, sm, st>>>(params, d, X, t, n, nullptr, work);
    HFAV_CUDA(cudaGetLastError());
    mlp_grad<<<(int)((d.n_params + 1 + 255) / 256), 256, 0, st>>>(d, X, n, work, grad, loss);
    HFAV_CUDA(cudaGetLastError());
    return HFAV_OK;
}

int hfav_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t n_params, float lr, float beta1,
                  float beta2, float eps, int step, void* stream) {
    if (!params || !grad || !m || !v || n_params < 1 || step < 1) return set_error(HFAV_EINVAL, "bad argument");
    float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    int blocks = (int)std::min<int64_t>((n_params + 255) / 256, 1024);
    mlp_adam_k<<<blocks, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, n_params, lr, beta1, beta2, eps, c1, c2);
    HFAV_CUDA(cudaGetLastError());
    return HFAV_OK;
}

int hfav_mlp_train(float* params, float* m, float* v, int n_in, int hidden, const float* X, const float* t, int n,
                   int epochs, float lr, float* work, float* grad, float* loss_hist, void* stream) {
    if (epochs < 1 || !loss_hist) return set_error(HFAV_EINVAL, "bad argument");
    const int64_t np = hfav_mlp_n_params(n_in, hidden);
    for (int e = 0; e < epochs; ++e) {
        int rc = hfav_mlp_loss_grad(params, n_in, hidden, X, t, n, grad, loss_hist + e, work, stream);
        if (rc) return rc;
        rc = hfav_mlp_adam(params, grad, m, v, np, lr, 0.9f, 0.999f, 1e-8f, e + 1, stream);
        if (rc) return rc;
    }
    return HFAV_OK;
}

int hfav_model_choose(hfav_plan_t* p, const float* params, int n_models, int hidden, const float* feat_shift,
                      const float* feat_scale, float* pred, int n_pred, char* best, size_t n_best) {
    if (!p || !params || p->analysis_only || n_models < 1) return set_error(HFAV_EINVAL, "bad argument");
    auto vars = valid_schedules(p);
    const int nv = (int)vars.size(), NI = HFAV_N_FEATURES;
    std::vector<float> X((size_t)nv * NI), base(nv);
    for (int k = 0; k < nv; ++k) {
        features(p, vars[k], &X[(size_t)k * NI]);
        base[k] = X[(size_t)k * NI + HFAV_FEATURE_BASE] * 16.f * 0.69314718f;   // ln of the estimate
        for (int f = 0; f < NI; ++f) {
            float sh = feat_shift ? feat_shift[f] : 0.f, sc = feat_scale ? feat_scale[f] : 1.f;
            X[(size_t)k * NI + f] = (X[(size_t)k * NI + f] - sh) * sc;
        }
    }
    float *dX, *dy;
    cudaError_t e = dev_malloc((void**)&dX, X.size() * sizeof(float));
    if (e != cudaSuccess) { cudaGetLastError(); return set_error(HFAV_ENOMEM, "cudaMalloc"); }
    e = dev_malloc((void**)&dy, nv * sizeof(float));
    if (e != cudaSuccess) { cudaFree(dX); return set_error(HFAV_ENOMEM, "cudaMalloc"); }
    std::vector<float> y(nv, 0.f), ym(nv);
    int rc = HFAV_OK;
    if (cudaMemcpy(dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = set_error(HFAV_ECUDA, "upload");
    const int64_t np = hfav_mlp_n_params(NI, hidden);
    for (int m = 0; m < n_models && !rc; ++m) {
        rc = hfav_mlp_forward(params + m * np, NI, hidden, dX, nv, dy, nullptr);
        if (!rc && cudaMemcpy(ym.data(), dy, nv * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = set_error(HFAV_ECUDA, "download");
        for (int k = 0; k < nv && !rc; ++k) y[k] += ym[k] / n_models;
    }
    cudaFree(dX);
    cudaFree(dy);
    if (rc) return rc;
    for (int k = 0; k < nv; ++k) y[k] += base[k];
    int arg = (int)(std::min_element(y.begin(), y.end()) - y.begin());
    for (int k = 0; k < nv && k < n_pred; ++k) pred[k] = y[k];
    p->sched = vars[arg];
    drop_graph(p);
    if (best && n_best) {
        std::string s = vars[arg].str();
        size_t c = std::min(s.size(), n_best - 1);
        memcpy(best, s.data(), c);
        best[c] = 0;
    }
    return HFAV_OK;
}

}  // extern "C"
