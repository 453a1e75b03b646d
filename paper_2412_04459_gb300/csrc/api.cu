// C ABI of the sparse-voxel rasterizer: argument checks, workspace layout and
// launch sequencing.  See include/svr.h for the contract of every call.
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "svr_internal.cuh"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(SVR_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

enum Slot {
    kStatus, kTileMask, kOctpath, kRect, kCount, kTileCount, kRecord, kScanBlocks,
    kKeys0, kKeys1, kVals0, kVals1, kRanges, kDcol, kBox, kTileOrder, kBlockList, kBlockLen,
    kHitMask, kSegment, kTotal, kNumSlots
};

struct Layout {
    size_t off[kNumSlots];
};

// Sub-buffers of the kSegment slot: tile_seg, merge_cnt, seg_len, seg_part.
struct SegBytes {
    size_t tile_seg, merge_cnt, seg_len, seg_part, total;
};

SegBytes seg_bytes(int64_t ntiles, size_t slots, size_t B) {
    SegBytes b;
    b.tile_seg = 0;
    b.merge_cnt = align256(8 * (size_t)ntiles);
    b.seg_len = b.merge_cnt + align256(4 * B * (size_t)ntiles);
    b.seg_part = b.seg_len + align256(4 * B * slots);
    b.total = b.seg_part + 4 * B * slots * svr::kSegFields * 32;
    return b;
}

// n_vox voxels seen by n_views views with ntiles tiles of edge `tile` in all.
Layout make_layout(int64_t n_vox, int n_views, int64_t cap, int64_t ntiles, int tile) {
    Layout L;
    size_t o = 0;
    auto take = [&](Slot s, size_t bytes) {
        L.off[s] = o;
        o = align256(o + bytes);
    };
    const size_t N = (size_t)n_vox, VN = (size_t)n_vox * (size_t)n_views, C = (size_t)cap;
    take(kStatus, sizeof(svr::Status));
    take(kTileMask, (size_t)ntiles * (1 + (size_t)tile * tile / 32));  // tile masks, block sign masks
    take(kOctpath, 8 * N);
    take(kRect, 8 * VN);
    take(kCount, 4 * VN);
    take(kTileCount, 4 * (2 * svr::kTileSub + 1) * (size_t)ntiles);
    take(kRecord, sizeof(svr::Record) * VN);
    take(kScanBlocks, 4 * (((size_t)ntiles * svr::kTileSub + svr::kScanTile - 1) / svr::kScanTile + 1));
    take(kKeys0, 8 * C);
    take(kKeys1, 8 * C);
    take(kVals0, 4 * C);
    take(kVals1, 4 * C);
    take(kRanges, 8 * (size_t)ntiles);
    take(kDcol, 12 * VN);
    take(kBox, 8 * VN);
    const size_t slots = (size_t)svr::seg_slot_capacity(cap);
    take(kTileOrder, 8 * ((size_t)ntiles + slots));
    const size_t B = (size_t)tile * tile / 32;
    take(kBlockList, 8 * B * C);
    take(kBlockLen, 4 * B * (size_t)ntiles);
    take(kHitMask, 4 * B * (C + 32 * (size_t)ntiles));   // the block lists' positions + 32 per (tile, block)
    take(kSegment, seg_bytes(ntiles, slots, B).total);
    L.off[kTotal] = o;
    return L;
}

int tile_bits(int64_t ntiles) {
    int b = 0;
    while (((int64_t)1 << b) < ntiles) ++b;
    return b;
}

int check_params(const svr_params *p) {
    if (!p) return fail(SVR_ERR_INVALID, "null params");
    if (p->tile != 8 && p->tile != 16 && p->tile != 32)
        return fail(SVR_ERR_INVALID, "tile %d (8, 16 or 32 supported)", p->tile);
    if (p->K < 1 || p->K > 3) return fail(SVR_ERR_INVALID, "K = %d (1..3 supported)", p->K);
    if (!(p->t_stop >= 0.f) || !(p->t_stop < 1.f)) return fail(SVR_ERR_INVALID, "t_stop %g", p->t_stop);
    return SVR_OK;
}

int check_camera(const svr_camera *cam, int tile, int *ntx, int *nty) {
    if (!cam) return fail(SVR_ERR_INVALID, "null camera");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 65536 || cam->height > 65536)
        return fail(SVR_ERR_INVALID, "image size %d x %d", cam->width, cam->height);
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
        return fail(SVR_ERR_INVALID, "bad intrinsics");
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(cam->w2c[i])) return fail(SVR_ERR_INVALID, "non-finite w2c");
    *ntx = (cam->width + tile - 1) / tile;
    *nty = (cam->height + tile - 1) / tile;
    return SVR_OK;
}

// Tile count of all views; SVR_OK or an error.
int check_views(const svr_camera *cams, int n_views, const svr_params *p, int64_t *ntiles) {
    int rc = check_params(p);
    if (rc != SVR_OK) return rc;
    if (!cams) return fail(SVR_ERR_INVALID, "null cameras");
    if (n_views < 1 || n_views > SVR_MAX_VIEWS)
        return fail(SVR_ERR_LIMIT, "%d views (1..%d supported)", n_views, SVR_MAX_VIEWS);
    int64_t total = 0;
    for (int v = 0; v < n_views; ++v) {
        int ntx, nty;
        rc = check_camera(cams + v, p->tile, &ntx, &nty);
        if (rc != SVR_OK) return rc;
        total += (int64_t)ntx * nty;
    }
    if (total > INT32_MAX / 64) return fail(SVR_ERR_LIMIT, "%lld tiles", (long long)total);
    *ntiles = total;
    return SVR_OK;
}

}  // namespace

namespace svr {

DebugBlock *debug_block() {
#ifdef SVR_DEBUG
    static std::atomic<DebugBlock *> blocks[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    DebugBlock *b = blocks[dev].load();
    if (b == nullptr) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(DebugBlock)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(DebugBlock)) != cudaSuccess) {
            cudaFree(p);
            return nullptr;
        }
        DebugBlock *expected = nullptr;
        if (!blocks[dev].compare_exchange_strong(expected, (DebugBlock *)p)) {
            cudaFree(p);
            return expected;
        }
        b = (DebugBlock *)p;
    }
    return b;
#else
    return nullptr;
#endif
}

}  // namespace svr

namespace {

svr::FrameDev frame_dev(const svr_frame *f) {
    svr::FrameDev d;
    memset(&d, 0, sizeof(d));
    d.n_views = f->n_views;
    d.total_tiles = (int)f->total_tiles;
    d.key_shift = f->key_shift;
    for (int v = 0; v < f->n_views; ++v) {
        const svr_camera &c = f->cams[v];
        svr::DevCam &dc = d.views[v];
        dc.fx = c.fx;
        dc.fy = c.fy;
        dc.cx = c.cx;
        dc.cy = c.cy;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) dc.R[3 * i + j] = c.w2c[4 * i + j];
        for (int i = 0; i < 3; ++i) dc.t[i] = c.w2c[4 * i + 3];
        for (int i = 0; i < 3; ++i) dc.ro[i] = (float)f->ray_origin[v][i];
        dc.W = c.width;
        dc.H = c.height;
        dc.tile = f->params.tile;
        dc.ntx = (c.width + dc.tile - 1) / dc.tile;
        dc.nty = (c.height + dc.tile - 1) / dc.tile;
        dc.tile_base = f->tile_base[v];
        dc.pix_base = f->pixel_base[v];
    }
    char *ws = (char *)f->ws;
    const uint64_t *o = f->offsets;
    d.status = (svr::Status *)(ws + o[kStatus]);
    d.tile_mask = (uint8_t *)(ws + o[kTileMask]);
    d.block_sign = d.tile_mask + f->total_tiles;
    d.octpath = (uint64_t *)(ws + o[kOctpath]);
    d.rect = (short4 *)(ws + o[kRect]);
    d.count = (uint32_t *)(ws + o[kCount]);
    d.tile_cnt = (uint32_t *)(ws + o[kTileCount]);
    d.cursor = d.tile_cnt + (size_t)svr::kTileSub * f->total_tiles;
    d.tile_end = d.cursor + (size_t)svr::kTileSub * f->total_tiles;
    d.rec = (svr::Record *)(ws + o[kRecord]);
    d.box = (ushort4 *)(ws + o[kBox]);
    d.scan_blocks = (uint32_t *)(ws + o[kScanBlocks]);
    d.keys[0] = (uint64_t *)(ws + o[kKeys0]);
    d.keys[1] = (uint64_t *)(ws + o[kKeys1]);
    d.vals[0] = (uint32_t *)(ws + o[kVals0]);
    d.vals[1] = (uint32_t *)(ws + o[kVals1]);
    d.ranges = (uint2 *)(ws + o[kRanges]);
    d.order = (uint2 *)(ws + o[kTileOrder]);
    d.blist = (uint2 *)(ws + o[kBlockList]);
    d.blen = (uint32_t *)(ws + o[kBlockLen]);
    d.hmask = (uint32_t *)(ws + o[kHitMask]);
    d.blocks_per_tile = f->params.tile * f->params.tile / 32;
    d.seg_slots = svr::seg_slot_capacity(f->pair_capacity);
    const SegBytes sb = seg_bytes(f->total_tiles, (size_t)d.seg_slots, (size_t)d.blocks_per_tile);
    char *seg = ws + o[kSegment];
    d.tile_seg = (uint2 *)(seg + sb.tile_seg);
    d.merge_cnt = (uint32_t *)(seg + sb.merge_cnt);
    d.seg_len = (uint32_t *)(seg + sb.seg_len);
    d.seg_part = (float *)(seg + sb.seg_part);
    d.dcol = (float *)(ws + o[kDcol]);
    d.n_vox = f->scene.n_vox;
    d.n_pts = f->scene.n_pts;
    d.capacity = f->pair_capacity;
    d.world_size = f->scene.world_size;
    for (int i = 0; i < 3; ++i) d.world_min[i] = f->scene.world_center[i] - 0.5f * f->scene.world_size;
    d.max_level = f->scene.max_level;
    d.K = f->params.K;
    d.t_stop = f->params.t_stop;
    for (int i = 0; i < 3; ++i) d.bg[i] = f->params.bg[i];
    d.debug = svr::debug_block();
    d.centre = f->scene.centre;
    d.level = f->scene.level;
    d.corner_idx = f->scene.corner_idx;
    d.grid = f->scene.grid;
    d.sh = f->scene.sh;
    return d;
}

// Shared by svr_preprocess (paper key layout) and svr_preprocess_views
// (compact keys).
int preprocess(svr_frame *frame, const svr_scene *scene, const svr_camera *cams, int n_views,
               const svr_params *params, void *ws, size_t ws_bytes, int64_t pair_capacity, bool paper_keys,
               void *stream) {
    g_err[0] = 0;
    if (!frame || !scene) return fail(SVR_ERR_INVALID, "null frame or scene");
    int64_t ntiles = 0;
    int rc = check_views(cams, n_views, params, &ntiles);
    if (rc != SVR_OK) return rc;
    const int64_t N = scene->n_vox;
    if (N < 0) return fail(SVR_ERR_INVALID, "n_vox %lld", (long long)N);
    if (N > ((int64_t)1 << 29)) return fail(SVR_ERR_LIMIT, "n_vox %lld > 2^29", (long long)N);
    if (scene->max_level < 1 || scene->max_level > 16)
        return fail(SVR_ERR_INVALID, "max_level %d", scene->max_level);
    const int lmax = scene->max_level;
    const int key_shift = paper_keys ? 48 : 3 * (lmax < 16 ? lmax + 1 : 16);
    if (paper_keys && ntiles > 65536)
        return fail(SVR_ERR_LIMIT, "%lld tiles > 2^16 (the key's 16-bit tile id)", (long long)ntiles);
    if (key_shift + tile_bits(ntiles) > 64)
        return fail(SVR_ERR_LIMIT, "%lld tiles and max_level %d do not fit a 64-bit key", (long long)ntiles, lmax);
    if (!(scene->world_size > 0.f) || !std::isfinite(scene->world_size))
        return fail(SVR_ERR_INVALID, "world_size %g", scene->world_size);
    if (N > 0 && (!scene->centre || !scene->level || !scene->corner_idx || !scene->sh ||
                  (!scene->grid && scene->n_pts > 0)))
        return fail(SVR_ERR_INVALID, "null scene array");
    if (N > 0 && (((uintptr_t)scene->sh) & 15u)) return fail(SVR_ERR_INVALID, "sh not 16-byte aligned");
    if (N > 0 && (((uintptr_t)scene->corner_idx) & 15u))
        return fail(SVR_ERR_INVALID, "corner_idx not 16-byte aligned");
    if (pair_capacity < 0 || pair_capacity > INT32_MAX)
        return fail(SVR_ERR_INVALID, "pair_capacity %lld", (long long)pair_capacity);
    if (!ws || (((uintptr_t)ws) & 255u)) return fail(SVR_ERR_INVALID, "workspace null or not 256-byte aligned");
    const Layout L = make_layout(N, n_views, pair_capacity, ntiles, params->tile);
    if (ws_bytes < L.off[kTotal])
        return fail(SVR_ERR_INVALID, "workspace %zu bytes < %zu needed", ws_bytes, (size_t)L.off[kTotal]);

    memset(frame, 0, sizeof(*frame));
    frame->scene = *scene;
    frame->params = *params;
    frame->n_views = n_views;
    frame->key_shift = key_shift;
    frame->total_tiles = ntiles;
    int64_t tb = 0, pb = 0;
    for (int v = 0; v < n_views; ++v) {
        const svr_camera &c = cams[v];
        frame->cams[v] = c;
        frame->tile_base[v] = (int32_t)tb;
        frame->pixel_base[v] = pb;
        tb += (int64_t)((c.width + params->tile - 1) / params->tile) * ((c.height + params->tile - 1) / params->tile);
        pb += (int64_t)c.width * c.height;
        for (int i = 0; i < 3; ++i) {
            double r = 0.0;
            for (int j = 0; j < 3; ++j) r -= (double)c.w2c[4 * j + i] * (double)c.w2c[4 * j + 3];
            frame->ray_origin[v][i] = r;
        }
    }
    frame->tile_base[n_views] = (int32_t)tb;
    frame->pixel_base[n_views] = pb;
    frame->ws = ws;
    frame->ws_bytes = ws_bytes;
    frame->pair_capacity = pair_capacity;
    frame->n_pairs = -1;
    for (int i = 0; i < kNumSlots; ++i) frame->offsets[i] = L.off[i];
    const svr::FrameDev d = frame_dev(frame);
    cudaStream_t s = (cudaStream_t)stream;
    // the tile-mask kernel also clears the status block and the tile counters
    cudaError_t e = svr::launch_tile_mask(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "tile mask");
    e = svr::launch_preprocess(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "preprocess");
    frame->stage = 1;
    return SVR_OK;
}

}  // namespace

namespace svr {
int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}
}  // namespace svr

extern "C" {

SVR_API const char *svr_last_error(void) { return g_err; }

SVR_API int svr_version(void) { return 200; }

SVR_API int svr_debug_build(void) {
#ifdef SVR_DEBUG
    return 1;
#else
    return 0;
#endif
}

SVR_API int svr_debug_report(uint64_t *out) {
    if (!out) return svr::set_error(SVR_ERR_INVALID, "svr_debug_report: null output");
    for (int i = 0; i < 4; ++i) out[i] = 0;
#ifdef SVR_DEBUG
    svr::DebugBlock *b = svr::debug_block();
    if (!b) return svr::set_error(SVR_ERR_CUDA, "svr_debug_report: no debug block on this device");
    svr::DebugBlock h;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, b, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b, 0, sizeof(h));
    if (e != cudaSuccess) return svr::set_error(SVR_ERR_CUDA, "svr_debug_report: %s", cudaGetErrorString(e));
    out[0] = h.count;
    out[1] = h.site;
    out[2] = (uint64_t)h.index;
    out[3] = (uint64_t)h.bound;
#endif
    return SVR_OK;
}

SVR_API size_t svr_workspace_size_views(int64_t n_vox, int64_t pair_capacity, const svr_camera *cams, int n_views,
                                        const svr_params *params) {
    int64_t ntiles = 0;
    if (n_vox < 0 || n_vox > ((int64_t)1 << 29)) return 0;
    if (pair_capacity < 0 || pair_capacity > INT32_MAX) return 0;
    if (check_views(cams, n_views, params, &ntiles) != SVR_OK) return 0;
    return make_layout(n_vox, n_views, pair_capacity, ntiles, params->tile).off[kTotal];
}

SVR_API size_t svr_workspace_size(int64_t n_vox, int64_t pair_capacity, const svr_camera *cam,
                                  const svr_params *params) {
    if (!cam) return 0;
    const size_t n = svr_workspace_size_views(n_vox, pair_capacity, cam, 1, params);
    if (n == 0) return 0;
    int ntx, nty;
    if (check_camera(cam, params->tile, &ntx, &nty) != SVR_OK || (int64_t)ntx * nty > 65536) return 0;
    return n;
}

SVR_API int svr_preprocess(svr_frame *frame, const svr_scene *scene, const svr_camera *cam,
                           const svr_params *params, void *ws, size_t ws_bytes, int64_t pair_capacity,
                           void *stream) {
    return preprocess(frame, scene, cam, 1, params, ws, ws_bytes, pair_capacity, true, stream);
}

SVR_API int svr_preprocess_views(svr_frame *frame, const svr_scene *scene, const svr_camera *cams, int n_views,
                                 const svr_params *params, void *ws, size_t ws_bytes, int64_t pair_capacity,
                                 void *stream) {
    return preprocess(frame, scene, cams, n_views, params, ws, ws_bytes, pair_capacity, false, stream);
}

SVR_API int svr_frame_status(const svr_frame *frame, uint32_t *flags, int64_t *n_pairs, void *stream) {
    if (!frame || frame->stage < 1) return fail(SVR_ERR_INVALID, "frame not preprocessed");
    svr::Status st;
    const svr::FrameDev d = frame_dev(frame);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&st, d.status, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (flags) *flags = st.flags;
    if (n_pairs) *n_pairs = (int64_t)(((uint64_t)st.n_pairs_hi << 32) | st.n_pairs_lo);
    return SVR_OK;
}

SVR_API int svr_bin_sort(svr_frame *frame, int64_t *n_pairs_out, void *stream) {
    g_err[0] = 0;
    if (!frame || frame->stage < 1) return fail(SVR_ERR_INVALID, "frame not preprocessed");
    const svr::FrameDev d = frame_dev(frame);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = svr::launch_scan(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "scan");
    e = svr::launch_order(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "ranges and work order");
    e = svr::launch_emit(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "emit");
    const int lmax = frame->scene.max_level;
    const int morton_bits = 3 * (lmax < 16 ? lmax + 1 : 16);
    e = svr::launch_tile_sort(d, frame->key_shift - morton_bits, morton_bits, lmax == 16, s);
    if (e != cudaSuccess) return cuda_fail(e, "sort");
    frame->sorted_alt = 0;
    e = svr::launch_block_lists(d, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "block lists");
    frame->stage = 2;
    frame->n_pairs = -1;
    if (n_pairs_out) {
        uint32_t flags = 0;
        int64_t P = 0;
        int rc = svr_frame_status(frame, &flags, &P, stream);
        if (rc != SVR_OK) return rc;
        *n_pairs_out = P;
        frame->n_pairs = P;
        if (flags & SVR_FLAG_INVALID_VOXEL)
            return fail(SVR_ERR_INVALID, "a voxel is off its lattice or its level is outside [1, %d]", lmax);
        if (flags & SVR_FLAG_CAPACITY)
            return fail(SVR_ERR_CAPACITY, "%lld pairs > capacity %lld", (long long)P,
                        (long long)frame->pair_capacity);
    }
    return SVR_OK;
}

SVR_API int svr_render_fwd(const svr_frame *frame, float *rgb, float *depth, float *alpha, float *T_final,
                           int32_t *last, void *stream) {
    g_err[0] = 0;
    if (!frame || frame->stage < 2) return fail(SVR_ERR_INVALID, "frame not sorted");
    if (!rgb || !depth || !alpha || !T_final || !last) return fail(SVR_ERR_INVALID, "null output");
    const svr::FrameDev d = frame_dev(frame);
    cudaError_t e = svr::launch_render_fwd(d, rgb, depth, alpha, T_final, last, nullptr, nullptr, nullptr, nullptr,
                                           (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "render_fwd");
    return SVR_OK;
}

SVR_API int svr_render_fwd_ex(const svr_frame *frame, float *rgb, float *depth, float *alpha, float *T_final,
                              int32_t *last, const svr_render_extras *extras, void *stream) {
    g_err[0] = 0;
    if (!frame || frame->stage < 2) return fail(SVR_ERR_INVALID, "frame not sorted");
    if (!rgb || !depth || !alpha || !T_final || !last) return fail(SVR_ERR_INVALID, "null output");
    float *normal = extras ? extras->normal : nullptr;
    float *max_weight = extras ? extras->max_weight : nullptr;
    float *dist = extras ? extras->distortion : nullptr;
    if (max_weight && (((uintptr_t)max_weight) & 3u)) return fail(SVR_ERR_INVALID, "max_weight not 4-byte aligned");
    const svr::FrameDev d = frame_dev(frame);
    cudaError_t e = svr::launch_render_fwd(d, rgb, depth, alpha, T_final, last, nullptr, normal, max_weight, dist,
                                           (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "render_fwd_ex");
    return SVR_OK;
}

SVR_API int svr_render_stats(const svr_frame *frame, float *rgb, float *depth, float *alpha, float *T_final,
                             int32_t *last, int32_t *counts, void *stream) {
    g_err[0] = 0;
    if (!frame || frame->stage < 2) return fail(SVR_ERR_INVALID, "frame not sorted");
    if (!rgb || !depth || !alpha || !T_final || !last || !counts) return fail(SVR_ERR_INVALID, "null output");
    if (((uintptr_t)counts) & 7u) return fail(SVR_ERR_INVALID, "counts not 8-byte aligned");
    const svr::FrameDev d = frame_dev(frame);
    cudaError_t e = svr::launch_render_fwd(d, rgb, depth, alpha, T_final, last, (int2 *)counts, nullptr, nullptr,
                                           nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "render_stats");
    return SVR_OK;
}

SVR_API int svr_render_bwd(const svr_frame *frame, const float *d_rgb, const float *d_depth,
                           const float *d_alpha, const float *T_final, const int32_t *last, float *d_grid,
                           float *d_sh, void *stream) {
    g_err[0] = 0;
    if (!frame || frame->stage < 2) return fail(SVR_ERR_INVALID, "frame not sorted");
    if (!T_final || !last) return fail(SVR_ERR_INVALID, "null T_final or last");
    if (frame->scene.n_vox > 0 && (!d_grid || !d_sh)) return fail(SVR_ERR_INVALID, "null gradient output");
    if (d_sh && (((uintptr_t)d_sh) & 15u)) return fail(SVR_ERR_INVALID, "d_sh not 16-byte aligned");
    const svr::FrameDev d = frame_dev(frame);
    cudaError_t e = svr::launch_render_bwd(d, d_rgb, d_depth, d_alpha, T_final, last, d_grid,
                                           d_sh, nullptr, nullptr, nullptr, nullptr, nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "render_bwd");
    return SVR_OK;
}

SVR_API int svr_render_bwd_ex(const svr_frame *frame, const float *d_rgb, const float *d_depth,
                              const float *d_alpha, const float *T_final, const int32_t *last, float *d_grid,
                              float *d_sh, const svr_render_extras *extras, void *stream) {
    g_err[0] = 0;
    if (!frame || frame->stage < 2) return fail(SVR_ERR_INVALID, "frame not sorted");
    if (!T_final || !last) return fail(SVR_ERR_INVALID, "null T_final or last");
    if (frame->scene.n_vox > 0 && (!d_grid || !d_sh)) return fail(SVR_ERR_INVALID, "null gradient output");
    if (d_sh && (((uintptr_t)d_sh) & 15u)) return fail(SVR_ERR_INVALID, "d_sh not 16-byte aligned");
    const float *d_normal = extras ? extras->d_normal : nullptr;
    float *priority = extras ? extras->priority : nullptr;
    const float *d_dist = extras ? extras->d_distortion : nullptr;
    const float *dist = extras ? extras->distortion : nullptr;
    if (d_dist && !dist) return fail(SVR_ERR_INVALID, "d_distortion needs the forward's distortion output");
    const svr::FrameDev d = frame_dev(frame);
    float *max_weight = extras ? extras->max_weight : nullptr;
    if (max_weight && (((uintptr_t)max_weight) & 3u)) return fail(SVR_ERR_INVALID, "max_weight not 4-byte aligned");
    cudaError_t e = svr::launch_render_bwd(d, d_rgb, d_depth, d_alpha, T_final, last, d_grid, d_sh, d_normal,
                                           priority, d_dist, dist, max_weight, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "render_bwd_ex");
    return SVR_OK;
}

SVR_API int svr_render_batched(svr_frame *frame, const svr_scene *scene, const svr_camera *cams, int n_views,
                               const svr_params *params, void *ws, size_t ws_bytes, int64_t pair_capacity,
                               float *rgb, float *depth, float *alpha, float *T_final, int32_t *last,
                               const float *d_rgb, const float *d_depth, const float *d_alpha, float *d_grid,
                               float *d_sh, void *stream) {
    int rc = svr_preprocess_views(frame, scene, cams, n_views, params, ws, ws_bytes, pair_capacity, stream);
    if (rc != SVR_OK) return rc;
    rc = svr_bin_sort(frame, nullptr, stream);
    if (rc != SVR_OK) return rc;
    rc = svr_render_fwd(frame, rgb, depth, alpha, T_final, last, stream);
    if (rc != SVR_OK) return rc;
    if (d_rgb || d_depth || d_alpha) rc = svr_render_bwd(frame, d_rgb, d_depth, d_alpha, T_final, last, d_grid, d_sh, stream);
    return rc;
}

SVR_API int svr_frame_buffers(const svr_frame *frame, svr_buffers *out) {
    if (!frame || !out || frame->stage < 1) return fail(SVR_ERR_INVALID, "frame not preprocessed");
    const svr::FrameDev d = frame_dev(frame);
    out->status = d.status;
    out->tile_mask = d.tile_mask;
    out->octpath = d.octpath;
    out->rect = (const int16_t *)d.rect;
    out->count = d.count;
    out->offset = nullptr;
    out->record = (const float *)d.rec;
    out->keys = d.keys[frame->sorted_alt];
    out->values = d.vals[frame->sorted_alt];
    out->ranges = (const uint32_t *)d.ranges;
    return SVR_OK;
}

}  // extern "C"
