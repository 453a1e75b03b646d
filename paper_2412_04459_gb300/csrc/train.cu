// Training-step pieces around the rasterizer (Sec. 3.2.3 objectives, the
// optimizer of the supplementary's implementation details):
//   k_t_concentration  the transmittance-concentration loss L_T, read as the
//                      mean binary entropy of the final transmittance T = 1 -
//                      alpha (T clamped to [1e-6, 1 - 1e-6], no gradient where
//                      the clamp acts), and its gradient with respect to the
//                      alpha image
//   k_weighted_mean    weight * mean of an array added to a loss (the
//                      distortion loss of every ray, rendered by the forward)
//   k_adam             the Adam update with two learning rates by position
//                      (the SH degree-0 coefficients and the rest)
// All are bandwidth-bound element-wise passes with one atomic per block for
// the loss sums.
#include <cmath>

#include "svr_internal.cuh"

namespace svr {

constexpr int kTrainThreads = 256;
constexpr float kTClamp = 1e-6f;

__device__ __forceinline__ void block_add(float acc, float *loss) {
    __shared__ float ws[kTrainThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < kTrainThreads / 32; ++w) s += ws[w];
        atomicAdd(loss, s);
    }
}

__global__ void __launch_bounds__(kTrainThreads) k_t_concentration(const float *__restrict__ alpha, int64_t n,
                                                                   float weight, float *__restrict__ grad,
                                                                   float *__restrict__ loss) {
    const float scale = weight / (float)n;
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float a = alpha[i];
        const float ac = fminf(fmaxf(a, kTClamp), 1.f - kTClamp);   // 1 - T clamped
        const float Tc = 1.f - ac;
        acc -= fmaf(Tc, logf(Tc), ac * logf(ac));
        // dH/dT = ln((1 - T) / T) = ln(a / T), written with x = a - T = 2a - 1
        // so that it keeps its relative precision near T = 1/2 (where the two
        // logarithms would cancel): log1p(x / T) for x >= 0, else
        // -log1p(-x / a); the gradient with respect to alpha is its negative
        if (grad) {
            const float x = fmaf(2.f, ac, -1.f);
            const float dH = x >= 0.f ? log1pf(x / Tc) : -log1pf(-x / ac);
            grad[i] = (a > kTClamp && a < 1.f - kTClamp) ? -scale * dH : 0.f;
        }
    }
    block_add(acc * scale, loss);
}

__global__ void __launch_bounds__(kTrainThreads) k_weighted_mean(const float *__restrict__ x, int64_t n, float weight,
                                                                 float *__restrict__ loss) {
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i];
    block_add(acc * (weight / (float)n), loss);
}

__device__ __forceinline__ float adam_one(float p, float g, float &m, float &v, float lr, float beta1, float beta2,
                                          float eps, float inv_bc1, float inv_bc2) {
    m = fmaf(beta1, m, (1.f - beta1) * g);
    v = fmaf(beta2, v, (1.f - beta2) * g * g);
    return p - lr * (m * inv_bc1) / (sqrtf(v * inv_bc2) + eps);
}

// Four parameters per thread and iteration as float4 (16-byte loads and
// stores of all four arrays); the learning rate of element i is lr_head when
// i mod period < head.  n4 = n / 4 vectors; the tail (n mod 4) is done by the
// first threads in scalar form.
__global__ void __launch_bounds__(kTrainThreads) k_adam(float *__restrict__ param, const float *__restrict__ grad,
                                                        float *__restrict__ m, float *__restrict__ v, int64_t n,
                                                        int period, int head, float lr_head, float lr_rest,
                                                        float beta1, float beta2, float eps, float inv_bc1,
                                                        float inv_bc2) {
    const int64_t n4 = n >> 2;
    float4 *p4 = reinterpret_cast<float4 *>(param);
    const float4 *g4 = reinterpret_cast<const float4 *>(grad);
    float4 *m4 = reinterpret_cast<float4 *>(m);
    float4 *v4 = reinterpret_cast<float4 *>(v);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 g = __ldcs(g4 + i);
        float4 p = __ldcs(p4 + i), mm = __ldcs(m4 + i), vv = __ldcs(v4 + i);
        // position of the first element within its period
        const int r = period == 1 ? 0 : (int)((4 * i) % period);
        const float l0 = (r < head) ? lr_head : lr_rest;
        const float l1 = ((r + 1) % period < head) ? lr_head : lr_rest;
        const float l2 = ((r + 2) % period < head) ? lr_head : lr_rest;
        const float l3 = ((r + 3) % period < head) ? lr_head : lr_rest;
        p.x = adam_one(p.x, g.x, mm.x, vv.x, l0, beta1, beta2, eps, inv_bc1, inv_bc2);
        p.y = adam_one(p.y, g.y, mm.y, vv.y, l1, beta1, beta2, eps, inv_bc1, inv_bc2);
        p.z = adam_one(p.z, g.z, mm.z, vv.z, l2, beta1, beta2, eps, inv_bc1, inv_bc2);
        p.w = adam_one(p.w, g.w, mm.w, vv.w, l3, beta1, beta2, eps, inv_bc1, inv_bc2);
        __stcs(p4 + i, p);
        __stcs(m4 + i, mm);
        __stcs(v4 + i, vv);
    }
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (n & 3)) {
        const int64_t i = 4 * n4 + t;
        float mm = m[i], vv = v[i];
        const float lr = (int)(i % period) < head ? lr_head : lr_rest;
        param[i] = adam_one(param[i], grad[i], mm, vv, lr, beta1, beta2, eps, inv_bc1, inv_bc2);
        m[i] = mm;
        v[i] = vv;
    }
}

static unsigned grid_for(int64_t n) {
    static DeviceCache cache;
    const unsigned sms = device_cached(cache, [] {
        int dev = 0, c = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        return (unsigned)(c > 0 ? c : 1);
    });
    const int64_t want = (n + kTrainThreads - 1) / kTrainThreads;
    return (unsigned)(want < (int64_t)sms * 8 ? (want > 0 ? want : 1) : (int64_t)sms * 8);
}

static int launched(const char *what) {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SVR_OK : set_error(SVR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace svr

extern "C" {

SVR_API int svr_t_concentration_loss(const float *alpha, int64_t n, float weight, float *grad_alpha, float *loss,
                                     void *stream) {
    if (!loss || n < 0 || (n > 0 && !alpha)) return svr::set_error(SVR_ERR_INVALID, "null pointer or n < 0");
    if (n == 0) return SVR_OK;
    svr::k_t_concentration<<<svr::grid_for(n), svr::kTrainThreads, 0, (cudaStream_t)stream>>>(alpha, n, weight,
                                                                                               grad_alpha, loss);
    return svr::launched("t_concentration_loss");
}

SVR_API int svr_weighted_mean(const float *x, int64_t n, float weight, float *loss, void *stream) {
    if (!loss || n < 0 || (n > 0 && !x)) return svr::set_error(SVR_ERR_INVALID, "null pointer or n < 0");
    if (n == 0) return SVR_OK;
    svr::k_weighted_mean<<<svr::grid_for(n), svr::kTrainThreads, 0, (cudaStream_t)stream>>>(x, n, weight, loss);
    return svr::launched("weighted_mean");
}

SVR_API int svr_adam(float *param, const float *grad, float *m, float *v, int64_t n, int32_t period, int32_t head,
                     float lr_head, float lr_rest, float beta1, float beta2, float eps, int64_t step,
                     void *stream) {
    if (n < 0 || (n > 0 && (!param || !grad || !m || !v)))
        return svr::set_error(SVR_ERR_INVALID, "null pointer or n < 0");
    if (period < 1 || head < 0 || head > period || step < 1)
        return svr::set_error(SVR_ERR_INVALID, "adam: period %d, head %d, step %lld", period, head, (long long)step);
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
        return svr::set_error(SVR_ERR_INVALID, "adam: betas %g %g, eps %g", beta1, beta2, eps);
    if (n == 0) return SVR_OK;
    if ((((uintptr_t)param) | ((uintptr_t)grad) | ((uintptr_t)m) | ((uintptr_t)v)) & 15u)
        return svr::set_error(SVR_ERR_INVALID, "adam: arrays must be 16-byte aligned");
    // bias corrections 1 - beta^t in double on the host
    const double bc1 = 1.0 - std::pow((double)beta1, (double)step), bc2 = 1.0 - std::pow((double)beta2, (double)step);
    svr::k_adam<<<svr::grid_for((n + 3) / 4), svr::kTrainThreads, 0, (cudaStream_t)stream>>>(
        param, grad, m, v, n, period, head, lr_head, lr_rest, beta1, beta2, eps, (float)(1.0 / bc1),
        (float)(1.0 / bc2));
    return svr::launched("adam");
}

}  // extern "C"
