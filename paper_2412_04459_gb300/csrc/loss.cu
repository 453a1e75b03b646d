// Mean squared error between a rendered image and a target (the MSE term of
// the paper's photometric loss, Sec. 3.2.3) and its gradient, for training
// steps: loss = sum (p - t)^2 / n, grad = 2 (p - t) / n.
#include "svr_internal.cuh"

namespace svr {

__global__ void __launch_bounds__(256) k_l2_loss(const float *__restrict__ pred, const float *__restrict__ target,
                                                 int64_t n, float *__restrict__ grad, float *__restrict__ loss) {
    __shared__ float ws[8];
    const float inv_n = 1.0f / (float)n;
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = pred[i] - target[i];
        acc = fmaf(d, d, acc);
        if (grad) grad[i] = 2.f * d * inv_n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < 8; ++w) s += ws[w];
        atomicAdd(loss, s * inv_n);
    }
}

}  // namespace svr

extern "C" SVR_API int svr_l2_loss(const float *pred, const float *target, int64_t n, float *grad, float *loss,
                                   void *stream) {
    if (!loss || n < 0 || (n > 0 && (!pred || !target)))
        return svr::set_error(SVR_ERR_INVALID, "null pointer or n < 0");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return svr::set_error(SVR_ERR_CUDA, "l2 loss: %s", cudaGetErrorString(e));
    if (n == 0) return SVR_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const unsigned grid = (unsigned)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
    svr::k_l2_loss<<<grid, 256, 0, s>>>(pred, target, n, grad, loss);
    e = cudaGetLastError();
    if (e != cudaSuccess) return svr::set_error(SVR_ERR_CUDA, "l2 loss: %s", cudaGetErrorString(e));
    return SVR_OK;
}
