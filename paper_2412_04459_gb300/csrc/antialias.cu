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
// 32 x 32 output tiles per block (plane = grid z), each thread four rows of
// one column, consecutive threads on consecutive columns, the tile's windows
// computed once in shared memory; the integer overlap arithmetic is 32-bit
// whenever its products fit.
#include "svr_internal.cuh"

namespace svr {

constexpr int kAaTx = 32, kAaTy = 8;   // threads of a block
constexpr int kAaRows = 4;             // output rows per thread: a block covers 32 x 32 pixels
constexpr int kAaTileY = kAaTy * kAaRows;
constexpr int kAaMaxScale = 4;          // source pixels per target pixel and axis, at most
constexpr int kAaWin = kAaMaxScale + 1;

// Overlap numerator of source pixel X with target pixel x (units of 1/n_ss);
// I is 32-bit when n * n_ss fits, else 64-bit.
template <class I>
__device__ __forceinline__ I aa_overlap(I X, I x, I n, I n_ss) {
    const I lo = max(X * n, x * n_ss), hi = min((X + 1) * n, (x + 1) * n_ss);
    return hi > lo ? hi - lo : I(0);
}

// Source window [X0, X0 + cnt) and weights of target index x along one axis
// (n target, n_ss source pixels).
template <class I>
__device__ __forceinline__ int aa_window(I x, I n, I n_ss, float w[kAaWin], int &cnt) {
    const I X0 = (x * n_ss) / n;
    const I X1 = min(n_ss - 1, ((x + 1) * n_ss - 1) / n);
    const float inv = 1.0f / (float)n_ss;
    cnt = (int)(X1 - X0) + 1;
#pragma unroll
    for (int j = 0; j < kAaWin; ++j) w[j] = (j < cnt) ? (float)aa_overlap<I>(X0 + j, x, n, n_ss) * inv : 0.f;
    return (int)X0;
}

// A block covers a 32 x 32 tile of output pixels (grid z = plane), each
// thread 4 rows of one column.  The tile's 32 column and 32 row windows are
// computed once, by the first 64 threads, into shared memory; then every
// thread does its pixels' loads and multiply-adds, four independent rows at
// once.
template <class I, int WIN>
__global__ void __launch_bounds__(kAaTx * kAaTy) k_downsample(const float *__restrict__ src, int Hs, int Ws,
                                                              float *__restrict__ dst, int H, int W) {
    __shared__ float swx[kAaTx][kAaWin], swy[kAaTileY][kAaWin];
    __shared__ int sx0[kAaTx], sy0[kAaTileY], snx[kAaTx], sny[kAaTileY];
    const int t = threadIdx.y * kAaTx + threadIdx.x;
    if (t < kAaTx) {
        const int x = blockIdx.x * kAaTx + t;
        int cnt = 0;
        float w[kAaWin];
        sx0[t] = x < W ? aa_window<I>(x, W, Ws, w, cnt) : 0;
        snx[t] = x < W ? cnt : 0;
        for (int j = 0; j < kAaWin; ++j) swx[t][j] = x < W ? w[j] : 0.f;
    } else if (t < kAaTx + kAaTileY) {
        const int r = t - kAaTx, y = blockIdx.y * kAaTileY + r;
        int cnt = 0;
        float w[kAaWin];
        sy0[r] = y < H ? aa_window<I>(y, H, Hs, w, cnt) : 0;
        sny[r] = y < H ? cnt : 0;
        for (int j = 0; j < kAaWin; ++j) swy[r][j] = y < H ? w[j] : 0.f;
    }
    __syncthreads();
    const int x = blockIdx.x * kAaTx + threadIdx.x;
    if (x >= W) return;
    const int64_t pl = blockIdx.z;
    const int nx = snx[threadIdx.x];
    const float *s_col = src + pl * Hs * (int64_t)Ws + sx0[threadIdx.x];
#pragma unroll
    for (int q = 0; q < kAaRows; ++q) {
        const int r = threadIdx.y + kAaTy * q, y = blockIdx.y * kAaTileY + r;
        if (y >= H) break;
        const int ny = sny[r];
        const float *s = s_col + (int64_t)sy0[r] * Ws;
        // WIN x WIN window, unrolled with predicated loads so that they are
        // all in flight together (WIN = 3 covers ratios up to 2)
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < WIN; ++j) {
            float rr = 0.f;
#pragma unroll
            for (int i = 0; i < WIN; ++i)
                if (j < ny && i < nx) rr = fmaf(swx[threadIdx.x][i], __ldg(s + (int64_t)j * Ws + i), rr);
            acc = fmaf(j < ny ? swy[r][j] : 0.f, rr, acc);
        }
        dst[(pl * H + y) * (int64_t)W + x] = acc;
    }
}

// The transpose as a gather: source pixel X collects the (at most two, the
// ratio being >= 1) target pixels per axis that overlap it.
template <class I>
__device__ __forceinline__ int aa_window_t(I X, I n, I n_ss, float w[2]) {
    const I x0 = (X * n) / n_ss;
    const I x1 = min(n - 1, ((X + 1) * n - 1) / n_ss);
    const float inv = 1.0f / (float)n_ss;
    w[0] = (float)aa_overlap<I>(X, x0, n, n_ss) * inv;
    w[1] = x1 > x0 ? (float)aa_overlap<I>(X, x0 + 1, n, n_ss) * inv : 0.f;
    return (int)x0;
}

template <class I>
__global__ void __launch_bounds__(kAaTx * kAaTy) k_downsample_bwd(const float *__restrict__ d_dst, int H, int W,
                                                                  float *__restrict__ d_src, int Hs, int Ws) {
    __shared__ float swx[kAaTx][2], swy[kAaTileY][2];
    __shared__ int sx0[kAaTx], sy0[kAaTileY];
    const int t = threadIdx.y * kAaTx + threadIdx.x;
    if (t < kAaTx) {
        const int X = blockIdx.x * kAaTx + t;
        float w[2] = {0.f, 0.f};
        sx0[t] = X < Ws ? aa_window_t<I>(X, W, Ws, w) : 0;
        swx[t][0] = w[0];
        swx[t][1] = w[1];
    } else if (t < kAaTx + kAaTileY) {
        const int r = t - kAaTx, Y = blockIdx.y * kAaTileY + r;
        float w[2] = {0.f, 0.f};
        sy0[r] = Y < Hs ? aa_window_t<I>(Y, H, Hs, w) : 0;
        swy[r][0] = w[0];
        swy[r][1] = w[1];
    }
    __syncthreads();
    const int X = blockIdx.x * kAaTx + threadIdx.x;
    if (X >= Ws) return;
    const int64_t pl = blockIdx.z;
    const float wx0 = swx[threadIdx.x][0], wx1 = swx[threadIdx.x][1];
    const float *g_col = d_dst + pl * H * (int64_t)W + sx0[threadIdx.x];
#pragma unroll
    for (int q = 0; q < kAaRows; ++q) {
        const int r = threadIdx.y + kAaTy * q, Y = blockIdx.y * kAaTileY + r;
        if (Y >= Hs) break;
        const float wy0 = swy[r][0], wy1 = swy[r][1];
        const float *g = g_col + (int64_t)sy0[r] * W;
        float r0 = wx0 * __ldg(g);
        if (wx1 != 0.f) r0 = fmaf(wx1, __ldg(g + 1), r0);
        float acc = wy0 * r0;
        if (wy1 != 0.f) {
            float r1 = wx0 * __ldg(g + W);
            if (wx1 != 0.f) r1 = fmaf(wx1, __ldg(g + W + 1), r1);
            acc = fmaf(wy1, r1, acc);
        }
        d_src[(pl * Hs + Y) * (int64_t)Ws + X] = acc;
    }
}

static int check_sizes(int64_t planes, int Hs, int Ws, int H, int W) {
    if (planes < 0 || H <= 0 || W <= 0 || Hs <= 0 || Ws <= 0)
        return set_error(SVR_ERR_INVALID, "downsample: sizes %lld x %d x %d -> %d x %d", (long long)planes, Hs, Ws,
                         H, W);
    if (Hs < H || Ws < W || Hs > kAaMaxScale * (int64_t)H || Ws > kAaMaxScale * (int64_t)W)
        return set_error(SVR_ERR_INVALID, "downsample: %d x %d -> %d x %d (ratio must lie in [1, %d])", Hs, Ws, H, W,
                         kAaMaxScale);
    if (planes > 65535) return set_error(SVR_ERR_LIMIT, "downsample: %lld planes (65535 at most)", (long long)planes);
    return SVR_OK;
}

}  // namespace svr

extern "C" {

SVR_API int svr_downsample(const float *src, int64_t planes, int height_ss, int width_ss, float *dst, int height,
                           int width, void *stream) {
    int rc = svr::check_sizes(planes, height_ss, width_ss, height, width);
    if (rc != SVR_OK) return rc;
    if (!src || !dst) return svr::set_error(SVR_ERR_INVALID, "downsample: null pointer");
    if (planes == 0) return SVR_OK;
    const dim3 block(svr::kAaTx, svr::kAaTy);
    const dim3 grid((unsigned)((width + svr::kAaTx - 1) / svr::kAaTx),
                    (unsigned)((height + svr::kAaTileY - 1) / svr::kAaTileY), (unsigned)planes);
    // 32-bit index arithmetic when the products of the overlap test fit
    const bool narrow = (int64_t)(width_ss + 1) * width < (1ll << 31) && (int64_t)(height_ss + 1) * height < (1ll << 31);
    // windows of at most 3 source pixels per axis for ratios up to 2
    const bool small = width_ss <= 2 * width && height_ss <= 2 * height;
    cudaStream_t st = (cudaStream_t)stream;
    if (narrow && small)
        svr::k_downsample<int, 3><<<grid, block, 0, st>>>(src, height_ss, width_ss, dst, height, width);
    else if (narrow)
        svr::k_downsample<int, svr::kAaWin><<<grid, block, 0, st>>>(src, height_ss, width_ss, dst, height, width);
    else
        svr::k_downsample<long long, svr::kAaWin><<<grid, block, 0, st>>>(src, height_ss, width_ss, dst, height, width);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return svr::set_error(SVR_ERR_CUDA, "downsample: %s", cudaGetErrorString(e));
    return SVR_OK;
}

SVR_API int svr_downsample_bwd(const float *d_dst, int64_t planes, int height, int width, float *d_src,
                               int height_ss, int width_ss, void *stream) {
    int rc = svr::check_sizes(planes, height_ss, width_ss, height, width);
    if (rc != SVR_OK) return rc;
    if (!d_dst || !d_src) return svr::set_error(SVR_ERR_INVALID, "downsample_bwd: null pointer");
    if (planes == 0) return SVR_OK;
    const dim3 block(svr::kAaTx, svr::kAaTy);
    const dim3 grid((unsigned)((width_ss + svr::kAaTx - 1) / svr::kAaTx),
                    (unsigned)((height_ss + svr::kAaTileY - 1) / svr::kAaTileY), (unsigned)planes);
    const bool narrow = (int64_t)(width_ss + 1) * width < (1ll << 31) && (int64_t)(height_ss + 1) * height < (1ll << 31);
    if (narrow)
        svr::k_downsample_bwd<int><<<grid, block, 0, (cudaStream_t)stream>>>(d_dst, height, width, d_src, height_ss,
                                                                            width_ss);
    else
        svr::k_downsample_bwd<long long><<<grid, block, 0, (cudaStream_t)stream>>>(d_dst, height, width, d_src,
                                                                                  height_ss, width_ss);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return svr::set_error(SVR_ERR_CUDA, "downsample_bwd: %s", cudaGetErrorString(e));
    return SVR_OK;
}

}  // extern "C"
