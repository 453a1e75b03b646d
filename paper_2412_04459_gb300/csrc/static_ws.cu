// Allocation-free forward render: the per-view workspace lives in a fixed
// device array compiled into the library instead of a buffer the caller
// allocates.
//
// Who needs it: code that may not call cudaMalloc or any other allocator
// itself, for example a plugin running inside a host application that owns
// the whole device-memory budget through its own pool, or a render callback
// on a latency-critical path where an allocation (which can synchronise the
// device) is not allowed.  Such callers still own their inputs and outputs;
// only the scratch memory moves into the library.
//
// Cost and limits: the array below is kStaticWorkspaceBytes (16 MiB) of
// device memory that every GPU which loads this library holds until the
// process exits.  It bounds a call to kStaticMaxVoxels voxels and as many
// pairs as fit in the remaining bytes (svr_render_fwd_static reports the
// limit it hit).  All calls share the one array and each call leaves its
// contents behind; the call clears everything that must start at zero.
// Calls whose GPU work overlaps (several host threads, or different streams
// without ordering between them) race on the array and give wrong images.
#include <mutex>

#include "svr_internal.cuh"

namespace {

constexpr size_t kStaticWorkspaceBytes = size_t(16) << 20;
constexpr int64_t kStaticMaxVoxels = 65536;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_ws[kStaticWorkspaceBytes];

std::mutex g_setup_mu;
void *g_static_ptr[kMaxDevices] = {};

// Device address of g_static_ws on the current device.  The host-side name
// of the array is only a stand-in: it must not be passed to a kernel.  The
// address is looked up once per device, with that device current, and kept
// for the life of the process (a device reset would invalidate it: the
// library is not to be used across cudaDeviceReset).
int static_workspace(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return SVR_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SVR_ERR_LIMIT;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess || p == nullptr) return SVR_ERR_CUDA;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return SVR_OK;
}

}  // namespace

extern "C" {

SVR_API int svr_render_fwd_static(const svr_scene *scene, const svr_camera *cam, const svr_params *params,
                                  float *rgb, float *depth, float *alpha, float *T_final, int32_t *last,
                                  int64_t *n_pairs_out, void *stream) {
    if (!scene || !cam || !params) return svr::set_error(SVR_ERR_INVALID, "null scene, camera or params");
    if (scene->n_vox < 0 || scene->n_vox > kStaticMaxVoxels)
        return svr::set_error(SVR_ERR_LIMIT, "static workspace: %lld voxels, at most %lld",
                              (long long)scene->n_vox, (long long)kStaticMaxVoxels);
    // the image's tile count first, so that an oversized image is reported as
    // the limit it breaks (svr_workspace_size returns 0 for it)
    if (params->tile == 8 || params->tile == 16 || params->tile == 32) {
        if (cam->width > 0 && cam->height > 0) {
            const int64_t tiles = (int64_t)((cam->width + params->tile - 1) / params->tile) *
                                  ((cam->height + params->tile - 1) / params->tile);
            if (tiles > 65536)
                return svr::set_error(SVR_ERR_LIMIT, "static workspace: %lld tiles > 2^16 (the key's 16-bit tile id)",
                                      (long long)tiles);
        }
    }
    const size_t base = svr_workspace_size(scene->n_vox, 0, cam, params);
    if (base == 0) return svr::set_error(SVR_ERR_INVALID, "invalid camera or params");
    if (base > kStaticWorkspaceBytes)
        return svr::set_error(SVR_ERR_LIMIT, "static workspace: this image needs %zu bytes, %zu available",
                              base, kStaticWorkspaceBytes);
    // the largest pair capacity whose workspace fits in the array
    int64_t lo = 0, hi = (int64_t)(kStaticWorkspaceBytes / 24) + 1;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) / 2;
        const size_t need = svr_workspace_size(scene->n_vox, mid, cam, params);
        if (need != 0 && need <= kStaticWorkspaceBytes) lo = mid;
        else hi = mid;
    }
    if (lo == 0) return svr::set_error(SVR_ERR_LIMIT, "static workspace: no room left for pairs");
    void *ws = nullptr;
    int rc = static_workspace(&ws);
    if (rc != SVR_OK) return svr::set_error(rc, "static workspace: no device address for the array");
    svr_frame frame;
    rc = svr_preprocess(&frame, scene, cam, params, ws, kStaticWorkspaceBytes, lo, stream);
    if (rc != SVR_OK) return rc;
    int64_t n_pairs = 0;
    rc = svr_bin_sort(&frame, &n_pairs, stream);
    if (n_pairs_out) *n_pairs_out = n_pairs;
    if (rc != SVR_OK) return rc;
    return svr_render_fwd(&frame, rgb, depth, alpha, T_final, last, stream);
}

}  // extern "C"
