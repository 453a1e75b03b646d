// Supersampling anti-aliasing (Sec. 3.1.2 "Anti-aliasing"): an image
// rendered at W_ss x H_ss is averaged down to W x H over each target pixel's
// footprint (area filter, separable).  Target pixel x covers the source
// interval [s x, s (x + 1)), s = W_ss / W, and source pixel X enters with the
// overlap length of [X, X + 1) divided by s.  With integers, the weight is
//     (min((X + 1) W, (x + 1) W_ss) - max(X W, x W_ss)) / W_ss,
// exact up to the one rounding of that division, whatever the image size.
// The backward is the transposed operator, written as a gather: each source
// pixel collects from the (at most two, s >= 1) target pixels per axis that
// overlap it, so no atomics are needed.  Both kernels are bandwidth-bound:
// one thread per output element, consecutive threads on consecutive x.
#include "svr_internal.cuh"

namespace svr {

constexpr int kAaThreads = 256;
constexpr int kAaMaxScale = 4;   // source pixels per target pixel and axis, at most

// Overlap numerator of source pixel X with target pixel x (units of 1/n_ss).
__device__ __forceinline__ long long aa_overlap(long long X, long long x, long long n, long long n_ss) {
    const long long lo = max(X * n, x * n_ss), hi = min((X + 1) * n, (x + 1) * n_ss);
    return hi > lo ? hi - lo : 0;
}

__global__ void __launch_bounds__(kAaThreads) k_downsample(const float *__restrict__ src, int64_t planes, int Hs,
                                                           int Ws, float *__restrict__ dst, int H, int W) {
    const int64_t i = (int64_t)blockIdx.x * kAaThreads + threadIdx.x;
    if (i >= planes * H * W) return;
    const int x = (int)(i % W);
    const int y = (int)((i / W) % H);
    const int64_t pl = i / ((int64_t)W * H);
    const float *s = src + pl * (int64_t)Hs * Ws;
    const int X0 = (int)(((long long)x * Ws) / W), X1 = (int)min((long long)Ws - 1, ((long long)(x + 1) * Ws - 1) / W);
    const int Y0 = (int)(((long long)y * Hs) / H), Y1 = (int)min((long long)Hs - 1, ((long long)(y + 1) * Hs - 1) / H);
    const float inv_x = 1.0f / (float)Ws, inv_y = 1.0f / (float)Hs;
    float acc = 0.f;
    for (int Y = Y0; Y <= Y1; ++Y) {
        const float wy = (float)aa_overlap(Y, y, H, Hs) * inv_y;
        float row = 0.f;
        for (int X = X0; X <= X1; ++X) row = fmaf((float)aa_overlap(X, x, W, Ws) * inv_x, __ldg(s + (int64_t)Y * Ws + X), row);
        acc = fmaf(wy, row, acc);
    }
    dst[i] = acc;
}

__global__ void __launch_bounds__(kAaThreads) k_downsample_bwd(const float *__restrict__ d_dst, int64_t planes, int H,
                                                               int W, float *__restrict__ d_src, int Hs, int Ws) {
    const int64_t i = (int64_t)blockIdx.x * kAaThreads + threadIdx.x;
    if (i >= planes * Hs * Ws) return;
    const int X = (int)(i % Ws);
    const int Y = (int)((i / Ws) % Hs);
    const int64_t pl = i / ((int64_t)Ws * Hs);
    const float *g = d_dst + pl * (int64_t)H * W;
    // target pixels overlapping [X, X + 1): x from floor(X W / W_ss) to
    // floor(((X + 1) W - 1) / W_ss)
    const int x0 = (int)(((long long)X * W) / Ws), x1 = (int)min((long long)W - 1, ((long long)(X + 1) * W - 1) / Ws);
    const int y0 = (int)(((long long)Y * H) / Hs), y1 = (int)min((long long)H - 1, ((long long)(Y + 1) * H - 1) / Hs);
    const float inv_x = 1.0f / (float)Ws, inv_y = 1.0f / (float)Hs;
    float acc = 0.f;
    for (int y = y0; y <= y1; ++y) {
        const float wy = (float)aa_overlap(Y, y, H, Hs) * inv_y;
        float row = 0.f;
        for (int x = x0; x <= x1; ++x) row = fmaf((float)aa_overlap(X, x, W, Ws) * inv_x, __ldg(g + (int64_t)y * W + x), row);
        acc = fmaf(wy, row, acc);
    }
    d_src[i] = acc;
}

static int check_sizes(int64_t planes, int Hs, int Ws, int H, int W) {
    if (planes < 0 || H <= 0 || W <= 0 || Hs <= 0 || Ws <= 0)
        return set_error(SVR_ERR_INVALID, "downsample: sizes %lld x %d x %d -> %d x %d", (long long)planes, Hs, Ws,
                         H, W);
    if (Hs < H || Ws < W || Hs > kAaMaxScale * (int64_t)H || Ws > kAaMaxScale * (int64_t)W)
        return set_error(SVR_ERR_INVALID, "downsample: %d x %d -> %d x %d (ratio must lie in [1, %d])", Hs, Ws, H, W,
                         kAaMaxScale);
    return SVR_OK;
}

}  // namespace svr

extern "C" {

SVR_API int svr_downsample(const float *src, int64_t planes, int height_ss, int width_ss, float *dst, int height,
                           int width, void *stream) {
    int rc = svr::check_sizes(planes, height_ss, width_ss, height, width);
    if (rc != SVR_OK) return rc;
    if (!src || !dst) return svr::set_error(SVR_ERR_INVALID, "downsample: null pointer");
    const int64_t n = planes * height * width;
    if (n == 0) return SVR_OK;
    svr::k_downsample<<<(unsigned)((n + svr::kAaThreads - 1) / svr::kAaThreads), svr::kAaThreads, 0,
                        (cudaStream_t)stream>>>(src, planes, height_ss, width_ss, dst, height, width);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return svr::set_error(SVR_ERR_CUDA, "downsample: %s", cudaGetErrorString(e));
    return SVR_OK;
}

SVR_API int svr_downsample_bwd(const float *d_dst, int64_t planes, int height, int width, float *d_src,
                               int height_ss, int width_ss, void *stream) {
    int rc = svr::check_sizes(planes, height_ss, width_ss, height, width);
    if (rc != SVR_OK) return rc;
    if (!d_dst || !d_src) return svr::set_error(SVR_ERR_INVALID, "downsample_bwd: null pointer");
    const int64_t n = planes * height_ss * width_ss;
    if (n == 0) return SVR_OK;
    svr::k_downsample_bwd<<<(unsigned)((n + svr::kAaThreads - 1) / svr::kAaThreads), svr::kAaThreads, 0,
                            (cudaStream_t)stream>>>(d_dst, planes, height, width, d_src, height_ss, width_ss);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return svr::set_error(SVR_ERR_CUDA, "downsample_bwd: %s", cudaGetErrorString(e));
    return SVR_OK;
}

}  // extern "C"
