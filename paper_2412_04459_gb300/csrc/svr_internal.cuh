// Internal declarations of the sparse-voxel rasterizer (sm_103a).
// Shared by the kernel translation units and the C ABI; not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/svr.h"

namespace svr {

template <class T>
__host__ __device__ __forceinline__ T tmin(T a, T b) {
    return a < b ? a : b;
}

constexpr int kMaxLevel = 16;
constexpr int kMaxViews = SVR_MAX_VIEWS;
constexpr float kNear = 1e-3f;             // corners at camera depth <= kNear are "behind"
constexpr uint64_t kTripleOnes = 0x249249249249ull;  // bit 0 of each of the 16 triples
constexpr int kScanTile = 256;             // entries per block of the count scan
// Tile lists longer than kSegLen entries are rendered as segments of kSegLen
// consecutive entries (the last one shorter), each by its own warps, and
// merged afterwards; kSegFields floats per pixel and segment carry the
// partial sums between the warps and on to the backward: colour (0..2),
// depth (3), transmittance after and before (4, 5; 5 holds the stopping
// index until the merge), work counts (6, 7), normal (8..10), distortion
// loss sums (11..13).
constexpr int kSegLen = 1024;
constexpr int kSegFields = 14;
// A tile's pairs are counted and emitted through kTileSub sub-buckets (by
// voxel id), so that the atomics on a busy tile spread over separate cache
// lines; the sub-buckets of a tile are adjacent in its range.
constexpr int kTileSub = 8;

// Segment slots a workspace holds for pair_capacity pairs: a split tile of
// L > kSegLen entries takes ceil(L / kSegLen) < 2 L / kSegLen slots.
__host__ __device__ __forceinline__ int64_t seg_slot_capacity(int64_t capacity) {
    return 2 * capacity / kSegLen + 1;
}

// Camera of one view as the kernels see it: intrinsics, [R | t], the ray
// origin -R^T t (computed in double on the host) and the view's tile grid.
struct DevCam {
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float ro[3];
    int W, H;
    int ntx, nty;
    int tile;
    int tile_base;     // first global tile id of the view
    int64_t pix_base;  // first pixel of the view in the contiguous outputs
};

// Device status block at the start of the workspace (64 bytes).
struct Status {
    unsigned flags;       // SVR_FLAG_*
    unsigned n_pairs_lo;  // total pair count (64-bit, split)
    unsigned n_pairs_hi;
    int bad_voxel;        // smallest invalid voxel id (all bits set: none)
    unsigned fwd_next;    // next work item of the forward render (the last warp of a launch resets it)
    unsigned bwd_next;    // next work item of the backward render (reset before each launch)
    unsigned n_queue;     // (tile, segment) entries of the render work order
    unsigned slots_used;  // segment slots taken by the split tiles
    unsigned fwd_done;    // bit 0: a forward filled the segment sums of the current sort; bit 1: with
                          // the normal image; bit 2: with the distortion loss
    unsigned sort_next;   // next work-order entry of the long-list sort
    unsigned fwd_exit;    // warps of the running forward launch that ran out of work
    unsigned maxw_next;   // next work item of the maximum-weight pass over split lists (reset before it)
    unsigned n_long;      // split tiles: the first n_long work-order entries are their first segments
    unsigned n_listed;    // work-order entries of non-empty lists (the empty tiles' entries come last)
    unsigned pad[2];
};

// Index checks of the SVR_DEBUG build (compiled out otherwise).  A failed
// check counts itself in the device's DebugBlock, keeps the first failure's
// site, index and bound, and the access is skipped (a read takes index 0 or a
// neutral value); nothing traps.  svr_debug_report() reads and clears it.
struct DebugBlock {
    unsigned long long count;
    unsigned site, pad;
    long long index, bound;
};

enum DebugSite : unsigned {
    kDbgTile = 1,        // tile id >= total_tiles (emission)
    kDbgRange = 2,       // tile range end > pair capacity (sort, render)
    kDbgVoxel = 3,       // voxel id of a list entry >= n_vox (block lists, render staging)
    kDbgGradPoint = 4,   // corner index >= n_pts (render backward atomics)
    kDbgRecSlot = 5,     // gradient record slot >= kRecCap (render backward)
    kDbgSegSlot = 6,     // segment slot >= seg_slots (render)
    kDbgBlockList = 7,   // block list longer than its tile list or segment (render)
};

#ifdef SVR_DEBUG
__device__ __forceinline__ bool in_bounds(DebugBlock *d, unsigned site, long long i, long long n) {
    if (i >= 0 && i < n) return true;
    if (d != nullptr && atomicAdd(&d->count, 1ull) == 0ull) {
        d->site = site;
        d->index = i;
        d->bound = n;
    }
    return false;
}
#define SVR_IN_BOUNDS(dbg, site, i, n) ::svr::in_bounds((dbg), (site), (long long)(i), (long long)(n))
#else
#define SVR_IN_BOUNDS(dbg, site, i, n) true
#endif

// Index i if SVR_IN_BOUNDS(i < n) holds, else 0 (the access reads element 0).
template <class I>
__device__ __forceinline__ I checked(DebugBlock *dbg, unsigned site, I i, long long n) {
    return SVR_IN_BOUNDS(dbg, site, i, n) ? i : I(0);
}

// The current device's DebugBlock (allocated on first use; nullptr in
// builds without SVR_DEBUG).
DebugBlock *debug_block();

// Per-voxel record of one view (64 bytes):
//   r0 = (lo - r_o).xyz, size      lo = centre - size / 2, the min corner
//   r1 = corner densities 0..3     (raw, gathered from the grid)
//   r2 = corner densities 4..7
//   r3 = colour rgb, bit c of the w word set if channel c was > 0 before the clamp
// Asynchronous 16-byte global -> shared copy (cp.async, L2 only), its
// commit and the wait for all but the N most recent groups.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

struct Record {
    float4 r0, r1, r2, r3;
};

// Ray direction of pixel (x, y): R^T ((x + .5 - cx) / fx, (y + .5 - cy) / fy, 1),
// written with explicit roundings so every kernel derives the same bits.
__device__ __forceinline__ float3 pixel_dir(const DevCam &c, int x, int y) {
    float dx = __fdiv_rn(__fsub_rn(__fadd_rn((float)x, 0.5f), c.cx), c.fx);
    float dy = __fdiv_rn(__fsub_rn(__fadd_rn((float)y, 0.5f), c.cy), c.fy);
    float3 d;
    d.x = __fadd_rn(__fadd_rn(__fmul_rn(c.R[0], dx), __fmul_rn(c.R[3], dy)), c.R[6]);
    d.y = __fadd_rn(__fadd_rn(__fmul_rn(c.R[1], dx), __fmul_rn(c.R[4], dy)), c.R[7]);
    d.z = __fadd_rn(__fadd_rn(__fmul_rn(c.R[2], dx), __fmul_rn(c.R[5], dy)), c.R[8]);
    return d;
}

// 4 (rd.x < 0) + 2 (rd.y < 0) + (rd.z < 0).
__device__ __forceinline__ int sign_bits(float3 d) {
    return (d.x < 0.f ? 4 : 0) | (d.y < 0.f ? 2 : 0) | (d.z < 0.f ? 1 : 0);
}

// explin (Eq. explin): x above 1.1, else exp(x / 1.1 - 1 + ln 1.1).
__device__ __forceinline__ float explin(float x) {
    return x > 1.1f ? x : __expf(fmaf(x, 0.909090909f, -0.904689820f));
}

// Real SH basis, degree 0..3, index l*l + l + m, no Condon-Shortley phase,
// as polynomials of the unit direction (x, y, z).  Constants are
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the factors of the
// corresponding Legendre / trigonometric polynomial.
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = 0.28209479177387814f;
    Y[1] = 0.4886025119029199f * y;
    Y[2] = 0.4886025119029199f * z;
    Y[3] = 0.4886025119029199f * x;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = 1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (3.f * zz - 1.f);
    Y[7] = 1.0925484305920792f * x * z;
    Y[8] = 0.5462742152960396f * (xx - yy);
    Y[9] = 0.5900435899266435f * y * (3.f * xx - yy);
    Y[10] = 2.890611442640554f * x * y * z;
    Y[11] = 0.4570457994644658f * y * (5.f * zz - 1.f);
    Y[12] = 0.3731763325901154f * z * (5.f * zz - 3.f);
    Y[13] = 0.4570457994644658f * x * (5.f * zz - 1.f);
    Y[14] = 1.445305721320277f * z * (xx - yy);
    Y[15] = 0.5900435899266435f * x * (xx - 3.f * yy);
}

// Everything the kernels need about a frame: the view table, the scene
// arrays and the workspace buffers.  Passed by value as a kernel parameter,
// so launches need no host-to-device copies (CUDA-graph capturable).
// Per-(view, voxel) arrays are indexed view * n_vox + voxel.
struct FrameDev {
    DevCam views[kMaxViews];
    int n_views;
    int total_tiles;         // sum of the views' tile counts
    int key_shift;           // Morton bits kept in the key; the tile id sits above them
    Status *status;
    uint8_t *tile_mask;      // [total_tiles]
    uint8_t *block_sign;     // [total_tiles][B]: sign-bit mask of each 8x4 block's in-image pixels
    uint64_t *octpath;       // [N]
    short4 *rect;            // [V * N] tile rectangle tx0, tx1, ty0, ty1
    uint32_t *count;         // [V * N] pairs of each (view, voxel)
    uint32_t *tile_cnt;      // [kTileSub][total_tiles] pairs of each tile's sub-buckets (k_preprocess)
    uint32_t *cursor;        // [kTileSub][total_tiles] next free slot of each sub-bucket
    uint32_t *tile_end;      // [total_tiles] end of each tile's range (from the scan)
    Record *rec;             // [V * N]
    ushort4 *box;            // [V * N] inclusive pixel range x0, x1, y0, y1 a hit can fall in
    uint32_t *scan_blocks;   // [ceil(total_tiles / kScanTile) + 1]
    uint64_t *keys[2];
    uint32_t *vals[2];
    uint2 *ranges;           // [total_tiles]
    uint2 *order;            // [total_tiles + seg slots] (tile, segment), longest segments first
    uint2 *tile_seg;         // [total_tiles] segments of the tile's list, first segment slot
    uint32_t *merge_cnt;     // [total_tiles * B] segments of a (tile, block) finished by the forward
    uint32_t *seg_len;       // [slots * B] block-list entries of each (segment, block)
    float *seg_part;         // [slots * B][kSegFields][32] per-pixel segment sums
    int64_t seg_slots;       // slots the workspace holds
    uint2 *blist;            // per (tile, 8x4 block) lists of (value, sorted index): block b of a tile
                             // whose list is [beg, end) owns [B beg + b (end - beg), ...)
    uint32_t *blen;          // [total_tiles * B] entries in each block list
    uint32_t *hmask;         // the forward's hit masks: block b of tile g (list [beg, end)) owns the
                             // words from B beg + b (end - beg) + 32 (g B + b); word p of it is, for
                             // p in batch [32 k, 32 k + 32) of the block's walk, the mask of the
                             // batch's entries (bit i: position 32 k + i) that pixel p mod 32 hit
    int blocks_per_tile;     // B = tile * tile / 32
    float *dcol;             // [V * N][3] colour gradient accumulator
    int64_t n_vox;
    int64_t n_pts;
    int64_t capacity;
    float world_size;
    float world_min[3];      // w_c - w_s / 2
    int max_level;
    int K;
    float t_stop;
    float bg[3];
    const float *centre;
    const uint8_t *level;
    const int32_t *corner_idx;
    const float *grid;
    const float *sh;
    DebugBlock *debug;       // index-check report of the SVR_DEBUG build (else nullptr)
};

// View that owns global tile g.
__device__ __forceinline__ int view_of_tile(const FrameDev &f, int g) {
    int v = 0;
    while (v + 1 < f.n_views && g >= f.views[v + 1].tile_base) ++v;
    return v;
}

// A launch constant (a persistent grid size, an SM count) kept per device,
// so that a process driving several GPUs in turn launches each with its
// own; 0 means not computed yet.  Concurrent first calls may both compute
// it and store the same value.
constexpr int kMaxDevices = 64;
struct DeviceCache {
    std::atomic<unsigned> v[kMaxDevices];
};

template <class F>
unsigned device_cached(DeviceCache &c, F compute) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return compute();
    unsigned x = c.v[dev].load(std::memory_order_relaxed);
    if (x == 0) {
        x = compute();
        c.v[dev].store(x, std::memory_order_relaxed);
    }
    return x;
}

// Records a printf-style message for svr_last_error() and returns code.
int set_error(int code, const char *fmt, ...);

cudaError_t launch_tile_mask(const FrameDev &f, cudaStream_t s);
cudaError_t launch_preprocess(const FrameDev &f, cudaStream_t s);
cudaError_t launch_scan(const FrameDev &f, cudaStream_t s);
cudaError_t launch_order(const FrameDev &f, cudaStream_t s);
cudaError_t launch_emit(const FrameDev &f, cudaStream_t s);
cudaError_t launch_tile_sort(const FrameDev &f, int lo_bit, int nbits, bool ties, cudaStream_t s);
cudaError_t launch_block_lists(const FrameDev &f, int sorted_alt, cudaStream_t s);
cudaError_t launch_render_fwd(const FrameDev &f, float *rgb, float *depth,
                              float *alpha, float *T_final, int32_t *last, int2 *stats, float *normal,
                              float *max_weight, float *dist, cudaStream_t s);
cudaError_t launch_render_bwd(const FrameDev &f, const float *d_rgb,
                              const float *d_depth, const float *d_alpha, const float *T_final,
                              const int32_t *last, float *d_grid, float *d_sh, const float *d_normal,
                              float *priority, const float *d_dist, const float *dist, float *max_weight,
                              cudaStream_t s);

}  // namespace svr
